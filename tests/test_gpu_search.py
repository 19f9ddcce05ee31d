"""Location by binary or multi-scale search (SFFT_METHOD_SEARCH) on the GPU against the FP64 oracle.

Noiseless inputs: supports identical to the oracle's and to the planted
spectrum, values within relative L2 1e-4 of the oracle's, iterations equal
to the oracle's.  Noisy inputs (the variant's advantage over phase
encoding): supports agree with the oracle's up to near-tie decisions, values
on the common support within relative L2 1e-4 of the oracle's (the FP32
tolerance; measured ~2e-7 on these cases and on the 2^20 workload), and the
planted support is recovered.  Batches give the plain path's answers.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import rel_l2, run_execute
from paper_2012_08238_gb300 import configs, metrics, sfft, signals

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SEARCH = sfft.SFFT_METHOD_SEARCH


def _pair(N, K, B, R, seed, b=1):
    w = configs.default_window(N, B)
    plan = sfft.sfft_plan_create_ex(N, K, B, w, R, seed, method=SEARCH, search_bits=b)
    return plan, oracle.PlanBS(N, K, B, w, R, seed, b=b)


@pytest.mark.parametrize("N,K,B,b,seed", [(1 << 16, 10, 64, 1, s) for s in range(4)] +
                         [(1 << 16, 10, 64, 2, 4), (1 << 14, 30, 128, 3, 1), (1 << 12, 5, 32, 1, 2),
                          (1 << 18, 100, 512, 1, 0), (1 << 18, 100, 512, 2, 3)])
def test_noiseless_matches_oracle(N, K, B, b, seed):
    sig = signals.make_signal(N, K, seed)
    plan, op = _pair(N, K, B, 8, seed, b)
    ref = oracle.sfft_bs(op, sig.x)
    idx, val, k = run_execute(plan, sig.x)
    st = sfft.sfft_plan_last_stats(plan)
    assert k == ref["k_out"] == K
    assert np.array_equal(idx, ref["idx"]) and np.array_equal(idx, np.sort(sig.freqs))
    assert rel_l2(val, ref["val"]) <= 1e-4
    assert st.iterations == ref["iters"]


@pytest.mark.parametrize("N,K,B,b,snr,seed", [
    (1 << 16, 10, 64, 1, 20.0, 3),
    (1 << 16, 10, 64, 1, 10.0, 5),
    (1 << 16, 10, 64, 2, 20.0, 6),
])
def test_noisy_matches_oracle(N, K, B, b, snr, seed):
    sig = signals.make_signal(N, K, seed, snr)
    plan, op = _pair(N, K, B, 8, seed, b)
    ref = oracle.sfft_bs(op, sig.x)
    idx, val, k = run_execute(plan, sig.x)
    common, gi, oi = np.intersect1d(idx, ref["idx"], return_indices=True)
    assert len(common) >= k - 1
    assert rel_l2(val[gi], ref["val"][oi]) <= 1e-4
    assert len(np.intersect1d(idx, sig.freqs)) == K


def test_general_workload_search():
    # N = 2^20, K = 100, 20 dB, B = 512: phase encoding finds nothing here
    W = configs.GENERAL_N20
    sig = signals.make_signal(W.N, W.K, 0, W.snr_db)
    plan, op = _pair(W.N, W.K, W.B, 8, 0)
    ref = oracle.sfft_bs(op, sig.x)
    idx, val, k = run_execute(plan, sig.x)
    common, gi, oi = np.intersect1d(idx, ref["idx"], return_indices=True)
    assert len(common) >= 0.99 * len(ref["idx"])
    # element by element on the common support
    assert rel_l2(val[gi], ref["val"][oi]) <= 1e-4
    assert np.max(np.abs(val[gi] - ref["val"][oi])) <= 1e-4 * np.max(np.abs(ref["val"]))
    assert sfft.sfft_plan_last_stats(plan).iterations == ref["iters"]
    e = metrics.errors(sig.xhat, W.K, idx, val)
    assert e["L0"] <= 1


def test_zero_and_one_sparse():
    N, B = 1 << 14, 64
    plan, op = _pair(N, 4, B, 8, 0)
    idx, val, k = run_execute(plan, np.zeros(N, np.complex64))
    assert k == 0 and sfft.sfft_plan_last_stats(plan).iterations == 1
    plan, op = _pair(N, 1, B, 8, 2)
    j = np.arange(N)
    x = ((0.3 + 0.4j) * np.exp(2j * np.pi * j * 12345 / N)).astype(np.complex64)
    idx, val, k = run_execute(plan, x)
    assert list(idx) == [12345] and abs(val[0] - (0.3 + 0.4j)) < 1e-4


def test_batch_equals_plain():
    specs = [(1 << 16, 10, 64, 1, s) for s in range(3)] + [(1 << 14, 20, 128, 2, 9)]
    plans, xs, idxs, vals, ref = [], [], [], [], []
    for N, K, B, b, seed in specs:
        sig = signals.make_signal(N, K, seed, 20.0)
        plan, _ = _pair(N, K, B, 8, seed, b)
        plans.append(plan)
        ref.append(run_execute(plan, sig.x)[:2])
        xs.append(torch.from_numpy(sig.x).cuda())
        idxs.append(torch.full((K,), -1, dtype=torch.int32, device="cuda"))
        vals.append(torch.zeros(K, dtype=torch.complex64, device="cuda"))
    kout = torch.zeros(len(specs), dtype=torch.int32, device="cuda")
    for _ in range(3):
        sfft.sfft_execute_batch(plans, xs, idxs, vals, kout)
        torch.cuda.synchronize()
        k = kout.cpu().numpy()
        for i, (ri, rv) in enumerate(ref):
            assert np.array_equal(idxs[i].cpu().numpy()[: k[i]], ri)
            assert rel_l2(vals[i].cpu().numpy()[: k[i]], rv) <= 1e-5


def test_search_option_checks():
    N, K, B = 1 << 16, 8, 64
    w = configs.default_window(N, B)
    with pytest.raises(sfft.SfftError):
        sfft.sfft_plan_create_ex(N, K, B, w, 8, 0, method=SEARCH, search_bits=5)
    with pytest.raises(sfft.SfftError):  # search_bits is for the search method only
        sfft.sfft_plan_create_ex(N, K, B, w, 8, 0, search_bits=1)
    with pytest.raises(sfft.SfftError):  # bucket buffers beyond one CTA's shared memory
        sfft.sfft_plan_create_ex(1 << 24, K, 8192, configs.default_window(1 << 24, 8192), 8, 0, method=SEARCH)
    info = sfft.sfft_plan_create_ex(N, K, B, w, 8, 0, method=SEARCH).info
    assert info.method == SEARCH


def test_server_serves_every_method_and_option():
    # requests of every location method and estimator option through one
    # server: each equals the same plan executed alone (batches are formed
    # per method; plans are keyed by every option)
    srv = sfft.sfft_server_create(2 << 30, 16)
    N, K, B = 1 << 16, 10, 64
    w = configs.default_window(N, B)
    kinds = [dict(), dict(method=sfft.SFFT_METHOD_PHASE), dict(method=sfft.SFFT_METHOD_COMB, comb=256),
             dict(method=SEARCH), dict(method=SEARCH, search_bits=2), dict(estimator=sfft.SFFT_ESTIMATOR_MEAN),
             dict(refine=2), dict(estimator=sfft.SFFT_ESTIMATOR_MEAN, refine=1)]
    reqs, bufs = [], []
    for i in range(2 * len(kinds)):
        kind = kinds[i % len(kinds)]
        sig = signals.make_signal(N, K, 70 + i, 30.0)
        x = torch.from_numpy(sig.x).cuda()
        idx = torch.full((K,), -1, dtype=torch.int32, device="cuda")
        val = torch.zeros(K, dtype=torch.complex64, device="cuda")
        bufs.append((sig, kind, x, idx, val))
        reqs.append(sfft.sfft_submit(srv, N, K, B, w, 8, 70 + i, x, idx, val, **kind))
    for i, (t, (sig, kind, x, idx, val)) in enumerate(zip(reqs, bufs)):
        res = sfft.sfft_wait(srv, t, 60000)
        assert res.status == sfft.SFFT_OK
        torch.cuda.synchronize()
        plan = sfft.sfft_plan_create_ex(N, K, B, w, 8, 70 + i, **kind)
        ri, rv, rk = run_execute(plan, sig.x)
        assert res.k_out == rk
        assert np.array_equal(idx.cpu().numpy()[:rk], ri)
        assert rel_l2(val.cpu().numpy()[:rk], rv) <= 1e-5
    srv.destroy()
