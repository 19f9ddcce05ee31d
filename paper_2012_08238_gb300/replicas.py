"""Replica execution over several GPUs: signals are independent, so each rank
runs its own shard and no collective touches the data path.  Only the timing
and the throughput total cross ranks (one scalar all-reduce each)."""
from __future__ import annotations


def shard(rank: int, world: int, per_rank: int) -> list[int]:
    """Signal ids of one rank: disjoint contiguous blocks of per_rank ids."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return [rank * per_rank + i for i in range(per_rank)]


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest value over all ranks (the job's elapsed time)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, dist=None, device=None) -> float:
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def throughput(units_all_ranks: float, elapsed_max_s: float) -> float:
    """Whole-job rate: every rank's units over the slowest rank's time."""
    return units_all_ranks / elapsed_max_s
