"""Replica sharding and the cross-rank timing reduction with two gloo ranks (CPU)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2012_08238_gb300 import replicas  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ids = replicas.shard(rank, world, per_rank=8)
    gathered = [None] * world
    dist.all_gather_object(gathered, ids)
    elapsed = 1.0 + rank  # rank 1 is the slowest
    mx = replicas.max_over_ranks(elapsed, dist)
    units = replicas.sum_over_ranks(len(ids), dist)
    if rank == 0:
        out.put((gathered, mx, units, replicas.throughput(units, mx)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_and_max_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    gathered, mx, units, rate = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    flat = [i for ids in gathered for i in ids]
    assert sorted(flat) == list(range(16)) and len(set(flat)) == 16  # disjoint and complete
    assert mx == 2.0 and units == 16
    assert rate == pytest.approx(8.0)


def test_single_process_fallbacks():
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.shard(0, 1, 3) == [0, 1, 2]
    with pytest.raises(ValueError):
        replicas.shard(2, 2, 3)
