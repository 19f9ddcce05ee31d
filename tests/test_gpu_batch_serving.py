"""Batched execution and the serving loop against the plain per-signal path.

Votes, selections and medians are integer or comparison-only work, but a
batch may split a job's gather into a different number of chunks than a plain
call, which reorders FP32 additions.  So the recovered frequencies must be
identical and the values equal within relative L2 1e-5 (the bucket-value
tolerance of the parity tests); a batch replayed with the same job list is
bit-for-bit deterministic.
"""
import time

import numpy as np
import pytest

from gpu_helpers import run_execute
from paper_2012_08238_gb300 import configs, sfft, signals

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# (N, K, B, w, L, seed, snr): shuffle-table, shared-table and generic-L jobs mixed
MIX = [
    (1 << 16, 10, 64, 2368, 8, 0, None),
    (1 << 14, 6, 1024, 2048, 4, 1, 15.0),
    (1 << 15, 12, 128, 128 * 36, 12, 2, 20.0),
    (1 << 13, 5, 32, 32 * 34, 5, 3, 10.0),
    (1 << 16, 10, 64, 2368, 8, 4, 30.0),
]


def _setup(mix):
    plans, xs, idxs, vals, sigs = [], [], [], [], []
    for N, K, B, w, L, seed, snr in mix:
        sig = signals.make_signal(N, K, seed, snr)
        sigs.append(sig)
        plans.append(sfft.sfft_plan_create(N, K, B, w, L, seed))
        xs.append(torch.from_numpy(sig.x).cuda())
        idxs.append(torch.full((K,), -1, dtype=torch.int32, device="cuda"))
        vals.append(torch.zeros(K, dtype=torch.complex64, device="cuda"))
    kout = torch.zeros(len(mix), dtype=torch.int32, device="cuda")
    return plans, xs, idxs, vals, kout, sigs


def _collect(idxs, vals, kout):
    torch.cuda.synchronize()
    k = kout.cpu().numpy()
    return [(idxs[i].cpu().numpy()[: k[i]], vals[i].cpu().numpy()[: k[i]]) for i in range(len(idxs))]


def _same(a, b):
    """Identical support; values within relative L2 1e-5."""
    if not np.array_equal(a[0], b[0]):
        return False
    va, vb = np.asarray(a[1], np.complex128), np.asarray(b[1], np.complex128)
    return np.linalg.norm(va - vb) <= 1e-5 * max(np.linalg.norm(vb), 1e-30)


def _identical(a, b):
    return np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_batch_of_mixed_plans_equals_plain_execute():
    plans, xs, idxs, vals, kout, sigs = _setup(MIX)
    ref = [run_execute(p, s.x)[:2] for p, s in zip(plans, sigs)]
    sfft.sfft_execute_batch(plans, xs, idxs, vals, kout)
    got = _collect(idxs, vals, kout)
    for r, g in zip(ref, got):
        assert _same(r, g)


def test_batch_graph_replay_reads_current_inputs():
    plans, xs, idxs, vals, kout, sigs = _setup(MIX)
    ref = [run_execute(p, s.x)[:2] for p, s in zip(plans, sigs)]
    first = None
    for _ in range(3):  # staging run, graph capture, graph replay
        for t in idxs:
            t.fill_(-1)
        sfft.sfft_execute_batch(plans, xs, idxs, vals, kout)
        got = _collect(idxs, vals, kout)
        for r, g in zip(ref, got):
            assert _same(r, g)
        if first is None:
            first = got
        for a, b in zip(first, got):
            assert _identical(a, b)  # same job list: same arithmetic
    # new contents in the same buffers: the replayed graph must see them
    new = [signals.make_signal(N, K, seed + 100, snr) for (N, K, B, w, L, seed, snr) in MIX]
    for t, s in zip(xs, new):
        t.copy_(torch.from_numpy(s.x).cuda())
    ref2 = [run_execute(p, s.x)[:2] for p, s in zip(plans, new)]
    sfft.sfft_execute_batch(plans, xs, idxs, vals, kout)
    got = _collect(idxs, vals, kout)
    for r, g in zip(ref2, got):
        assert _same(r, g)


def test_batch_rejects_repeated_plan():
    plans, xs, idxs, vals, kout, sigs = _setup(MIX[:2])
    with pytest.raises(sfft.SfftError) as ei:
        sfft.sfft_execute_batch([plans[0], plans[0]], xs, idxs, vals, kout)
    assert ei.value.status == sfft.SFFT_EINVAL


def test_host_buffer_paths_equal_device_paths():
    plans, xs, idxs, vals, kout, sigs = _setup(MIX)
    ref = [run_execute(p, s.x)[:2] for p, s in zip(plans, sigs)]
    # single plan, host buffers
    N, K = MIX[0][0], MIX[0][1]
    ih = np.zeros(K, np.int32)
    vh = np.zeros(K, np.complex64)
    kh = np.zeros(1, np.int32)
    sfft.sfft_execute_host(plans[0], np.ascontiguousarray(sigs[0].x), ih, vh, kh)
    assert _same(ref[0], (ih[: kh[0]], vh[: kh[0]]))
    # batch, pinned host buffers
    xh = [torch.from_numpy(s.x).pin_memory() for s in sigs]
    ihs = [torch.zeros(m[1], dtype=torch.int32).pin_memory() for m in MIX]
    vhs = [torch.zeros(m[1], dtype=torch.complex64).pin_memory() for m in MIX]
    khs = torch.zeros(len(MIX), dtype=torch.int32).pin_memory()
    sfft.sfft_execute_batch_host(plans, xh, ihs, vhs, khs)
    for i, r in enumerate(ref):
        k = int(khs[i])
        assert _same(r, (ihs[i].numpy()[:k], vhs[i].numpy()[:k]))


def test_host_buffer_batches_across_signals_and_reseeds():
    # host-buffer batches of voting plans (one with the stream gather) and of
    # comb plans (a batch of their own method): every result equals its
    # device-path call, across signals and a reseed.
    voting = [(1 << 16, 10, 64, 2368, 8, 0, sfft.SFFT_METHOD_VOTING, 0),
              (1 << 18, 40, 256, 256 * 39, 12, 1, sfft.SFFT_METHOD_VOTING, 0),
              (1 << 17, 20, 128, 128 * 38, 12, 2, sfft.SFFT_METHOD_VOTING, sfft.SFFT_GATHER_STREAM)]
    comb = [(1 << 16, 10, 64, 2368, 8, 3, sfft.SFFT_METHOD_COMB, 0),
            (1 << 16, 12, 64, 2368, 8, 4, sfft.SFFT_METHOD_COMB, 0)]
    for specs in (voting, comb):
        plans = [sfft.sfft_plan_create_ex(N, K, B, w, L, seed, method=m, mode=mode)
                 for N, K, B, w, L, seed, m, mode in specs]
        for round_ in range(3):
            if round_ == 2:
                sfft.sfft_plan_reseed(plans[1], 77)
                torch.cuda.synchronize()
            sigs = [signals.make_signal(sp[0], sp[1], 40 + 10 * round_ + i, 20.0).x for i, sp in enumerate(specs)]
            xh = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory() for x in sigs]
            ihs = [torch.zeros(sp[1], dtype=torch.int32).pin_memory() for sp in specs]
            vhs = [torch.zeros(sp[1], dtype=torch.complex64).pin_memory() for sp in specs]
            khs = torch.zeros(len(specs), dtype=torch.int32).pin_memory()
            sfft.sfft_execute_batch_host(plans, xh, ihs, vhs, khs)
            for i, (p, x) in enumerate(zip(plans, sigs)):
                k = int(khs[i])
                assert _same(run_execute(p, x)[:2], (ihs[i].numpy()[:k], vhs[i].numpy()[:k])), (round_, i)


def test_timed_batch_reports_stage_times():
    plans, xs, idxs, vals, kout, sigs = _setup(MIX)
    ref = [run_execute(p, s.x)[:2] for p, s in zip(plans, sigs)]
    total, stages = sfft.sfft_execute_batch_timed(plans, xs, idxs, vals, kout, 3)
    assert total > 0 and all(v >= 0 for v in stages.values())
    assert sum(stages.values()) <= total * 1.01
    got = _collect(idxs, vals, kout)
    for r, g in zip(ref, got):
        assert _same(r, g)


# ------------------------------------------------------------------ serving
def _request_buffers(N, K, seed, snr):
    sig = signals.make_signal(N, K, seed, snr)
    x = torch.from_numpy(sig.x).cuda()
    idx = torch.full((K,), -1, dtype=torch.int32, device="cuda")
    val = torch.zeros(K, dtype=torch.complex64, device="cuda")
    return sig, x, idx, val


def _serve(srv, reqs):
    """Submit every request, wait for all; returns [(idx, val, result)]."""
    bufs, tickets = [], []
    for (N, K, B, w, L, seed, snr) in reqs:
        sig, x, idx, val = _request_buffers(N, K, seed, snr)
        bufs.append((x, idx, val))
        tickets.append(sfft.sfft_submit(srv, N, K, B, w, L, seed, x, idx, val))
    out = []
    for t, (x, idx, val) in zip(tickets, bufs):
        res = sfft.sfft_wait(srv, t, 60000)
        torch.cuda.synchronize()
        out.append((idx.cpu().numpy()[: res.k_out], val.cpu().numpy()[: res.k_out], res))
    return out


def test_server_results_equal_alone_and_in_the_mix():
    srv = sfft.sfft_server_create(4 << 30, 16)
    probe = (1 << 16, 10, 64, 2368, 8, 77, 20.0)
    alone = _serve(srv, [probe])[0]
    rng = np.random.default_rng(0)
    mix = [MIX[i % len(MIX)][:5] + (1000 + i, float(rng.uniform(0, 40))) for i in range(30)]
    mix.insert(13, probe)
    served = _serve(srv, mix)
    in_mix = served[13]
    assert _same((alone[0], alone[1]), (in_mix[0], in_mix[1]))
    # every served result equals the plain path
    for (N, K, B, w, L, seed, snr), (idx, val, res) in zip(mix, served):
        assert res.status == sfft.SFFT_OK and res.latency_ns > 0
        plan = sfft.sfft_plan_create(N, K, B, w, L, seed)
        ref = run_execute(plan, signals.make_signal(N, K, seed, snr).x)
        assert _same(ref[:2], (idx, val))
        assert res.samples_touched == plan.info.samples_touched
    srv.destroy()


def test_server_pause_wait_timeout_and_resume():
    srv = sfft.sfft_server_create(1 << 30, 4)
    sfft.sfft_server_set_paused(srv, True)
    N, K, B, w, L = 1 << 14, 5, 64, 64 * 35, 6
    sig, x, idx, val = _request_buffers(N, K, 5, None)
    t = sfft.sfft_submit(srv, N, K, B, w, L, 5, x, idx, val)
    assert sfft.sfft_poll(srv, t) is None  # pending
    with pytest.raises(sfft.SfftError) as ei:
        sfft.sfft_wait(srv, t, 100)
    assert ei.value.status == sfft.SFFT_ETIMEDOUT
    sfft.sfft_server_set_paused(srv, False)
    res = sfft.sfft_wait(srv, t, 60000)
    assert res.status == sfft.SFFT_OK and res.k_out == K
    torch.cuda.synchronize()
    assert np.array_equal(idx.cpu().numpy(), sig.freqs)
    srv.destroy()


def test_server_rejects_request_beyond_budget_and_evicts_idle_plans():
    small = sfft.sfft_server_create(1 << 20, 4)  # 1 MiB: no N=2^20 plan fits
    W = configs.GENERAL_N20
    sig, x, idx, val = _request_buffers(1 << 12, 4, 1, None)
    with pytest.raises(sfft.SfftError) as ei:
        sfft.sfft_submit(small, W.N, W.K, W.B, W.window, W.L, 0, x, idx, val)
    assert ei.value.status == sfft.SFFT_EBUSY
    small.destroy()
    # room for about two N=2^16 plans: four different plans must still all be served
    srv = sfft.sfft_server_create(5 << 20, 2)
    reqs = [(1 << 16, 10, 64, 2368, 8, s, 20.0) for s in range(4)]
    out = []
    for r in reqs:  # one at a time, so each new plan must evict an idle one
        out += _serve(srv, [r])
    for (N, K, B, w, L, seed, snr), (i, v, res) in zip(reqs, out):
        assert res.status == sfft.SFFT_OK
        plan = sfft.sfft_plan_create(N, K, B, w, L, seed)
        ref = run_execute(plan, signals.make_signal(N, K, seed, snr).x)
        assert np.array_equal(ref[0], i)
    srv.destroy()


def test_server_destroy_drains_outstanding_work():
    srv = sfft.sfft_server_create(2 << 30, 8)
    bufs = []
    for s in range(12):
        sig, x, idx, val = _request_buffers(1 << 14, 5, s, None)
        bufs.append((sig, x, idx, val))  # buffers stay alive until the server is done
        sfft.sfft_submit(srv, 1 << 14, 5, 64, 64 * 35, 6, s, x, idx, val)
    srv.destroy()  # must finish every queued request before returning
    torch.cuda.synchronize()
    for sig, x, idx, val in bufs:
        assert np.array_equal(idx.cpu().numpy(), sig.freqs)


# ------------------------------------------------- reseeding and shared tables
def test_reseeded_plan_equals_a_fresh_plan_also_under_graph_replay():
    N, K, B, L = 1 << 16, 10, 64, 8
    w = configs.default_window(N, B)
    sigs = [signals.make_signal(N, K, s, 20.0) for s in (21, 22)]
    plans = [sfft.sfft_plan_create(N, K, B, w, L, s) for s in (1, 2)]
    xs = [torch.from_numpy(g.x).cuda() for g in sigs]
    idxs = [torch.zeros(K, dtype=torch.int32, device="cuda") for _ in range(2)]
    vals = [torch.zeros(K, dtype=torch.complex64, device="cuda") for _ in range(2)]
    kout = torch.zeros(2, dtype=torch.int32, device="cuda")
    for _ in range(3):  # staging run, capture, replay: the graph now exists
        sfft.sfft_execute_batch(plans, xs, idxs, vals, kout)
    for p, s in zip(plans, (21, 22)):
        sfft.sfft_plan_reseed(p, s)
    assert plans[0].info.seed == 21
    assert sfft.sfft_plan_get_loops(plans[0]) == sfft.sfft_loop_params(N, L, 21)
    sfft.sfft_execute_batch(plans, xs, idxs, vals, kout)  # replays the cached graph
    got = _collect(idxs, vals, kout)
    for i, s in enumerate((21, 22)):
        fresh = sfft.sfft_plan_create(N, K, B, w, L, s)
        ref = run_execute(fresh, sigs[i].x)
        assert _same(ref[:2], got[i])  # (a batch may split the gather differently)
        assert plans[i].info.samples_touched == fresh.info.samples_touched


def test_plans_sharing_tables_outlive_each_other():
    N, K, B, L = 1 << 15, 8, 128, 8
    w = configs.default_window(N, B)
    sig = signals.make_signal(N, K, 3, 30.0)
    a = sfft.sfft_plan_create(N, K, B, w, L, 3)
    ref = run_execute(a, sig.x)
    b = sfft.sfft_plan_create(N, K, B, w, L, 3)  # same shape: the tables of a
    a.destroy()
    assert _identical(ref[:2], run_execute(b, sig.x)[:2])
    c = sfft.sfft_plan_create(N, K, B, w, L, 3)
    b.destroy()
    assert _identical(ref[:2], run_execute(c, sig.x)[:2])


def test_server_rebinds_cached_plans_to_each_seed_and_K():
    # one voting shape (K up to 128 share a plan), 40 requests of distinct seeds and K
    N, B, L = 1 << 16, 512, 8
    w = configs.default_window(N, B)
    srv = sfft.sfft_server_create(2 << 30, 8)
    Ks = [65 + (37 * i) % 64 for i in range(40)]
    reqs = [(N, Ks[i], B, w, L, 300 + i, 20.0) for i in range(40)]
    served = _serve(srv, reqs)
    for (N_, K, B_, w_, L_, seed, snr), (idx, val, res) in zip(reqs, served):
        assert res.status == sfft.SFFT_OK and res.k_out == K
        ref = run_execute(sfft.sfft_plan_create(N, K, B, w, L, seed), signals.make_signal(N, K, seed, snr).x)
        assert _same(ref[:2], (idx, val))
    srv.destroy()


def test_one_slot_server_is_the_plain_path():
    srv = sfft.sfft_server_create(1 << 30, 1)
    reqs = [(1 << 14, 5, 64, 64 * 35, 6, 900 + i, 20.0) for i in range(6)]
    for (N, K, B, w, L, seed, snr), (idx, val, res) in zip(reqs, _serve(srv, reqs)):
        ref = run_execute(sfft.sfft_plan_create(N, K, B, w, L, seed), signals.make_signal(N, K, seed, snr).x)
        assert res.status == sfft.SFFT_OK and _identical(ref[:2], (idx, val))
    srv.destroy()
