"""The averaging estimator (SFFT_ESTIMATOR_MEAN) on the GPU against the FP64 oracle.

Step a6 combines a candidate's L per-loop estimates by their mean instead of
the coordinate-wise median; no bound on a mean prunes the candidates, so the
scans hand every candidate to the estimate kernels.  Shapes cover the
register-table scan (32 <= B <= 512, T = ceil(L/2)), the table scans (T other
than ceil(L/2), B > 512, B < 32, odd L), the comb pre-filter, the fallback
pass, the single-stage estimate entry point and batches that mix both
estimators.  Supports must match the oracle's outside near ties of the K-th
rank; values stay within relative L2 1e-4 on the common support.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import rel_l2, run_estimate, run_execute
from paper_2012_08238_gb300 import configs, metrics, sfft, signals

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MEAN = sfft.SFFT_ESTIMATOR_MEAN


def _pair(N, K, B, L, seed, T=None, method=sfft.SFFT_METHOD_VOTING, comb=0):
    w = configs.default_window(N, B)
    plan = sfft.sfft_plan_create_ex(N, K, B, w, L, seed, T=T or 0, method=method, comb=comb, estimator=MEAN)
    return plan, oracle.Plan(N, K, B, w, L, seed, T=T, estimator=oracle.MEAN)


def _check(idx, val, k, ref):
    assert k == ref["k_out"]
    common, gi, oi = np.intersect1d(idx, ref["idx"], return_indices=True)
    assert k - len(common) <= 1  # a disagreement only at a near tie of the K-th rank
    assert rel_l2(val[gi], ref["val"][oi]) <= 1e-4


@pytest.mark.parametrize("N,K,B,L,T,snr,seed", [
    (1 << 14, 10, 64, 8, None, None, 0),    # register table of kept bits
    (1 << 16, 20, 256, 12, None, 20.0, 1),  # register table, noisy
    (1 << 14, 10, 64, 8, 3, 20.0, 2),       # T != ceil(L/2): table scan
    (1 << 16, 16, 1024, 8, None, 30.0, 3),  # shared-table scan
    (1 << 12, 5, 16, 5, None, 30.0, 4),     # B < 32, odd L (generic estimate)
])
def test_mean_matches_oracle(N, K, B, L, T, snr, seed):
    sig = signals.make_signal(N, K, seed, snr)
    plan, op = _pair(N, K, B, L, seed, T)
    assert plan.info.estimator == MEAN
    ref = oracle.sfft(op, sig.x)
    idx, val, k = run_execute(plan, sig.x)
    _check(idx, val, k, ref)
    st = sfft.sfft_plan_last_stats(plan)
    if st.fallback == 0:
        # every candidate was estimated: the survivors are the candidates (the
        # counts agree up to kept sets that differ at near ties of the select
        # rank, FP32 against FP64, e.g. among the leakage-floor buckets of a
        # noiseless signal)
        full = oracle.sfft(op, sig.x, intermediates=True)
        assert abs(st.estimated - len(full["cand"])) <= 0.01 * len(full["cand"])


def test_general_workload_mean():
    W = configs.GENERAL_N20
    sig = signals.make_signal(W.N, W.K, 0, W.snr_db)
    plan, op = _pair(W.N, W.K, W.B, W.L, 0)
    ref = oracle.sfft(op, sig.x)
    idx, val, k = run_execute(plan, sig.x)
    _check(idx, val, k, ref)
    e = metrics.errors(sig.xhat, W.K, idx, val)
    assert e["L0"] <= 1


def test_mean_behind_comb():
    N, K, B, L, Bc, seed = 1 << 16, 10, 64, 8, 256, 5
    sig = signals.make_signal(N, K, seed, 20.0)
    plan, op = _pair(N, K, B, L, seed, method=sfft.SFFT_METHOD_COMB, comb=Bc)
    ref = oracle.sfft2(op, sig.x, Bc)
    idx, val, k = run_execute(plan, sig.x)
    _check(idx, val, k, ref)


def test_mean_fallback_pass():
    # four strong coefficients, K = 16: fewer than K estimates reach theta,
    # so the fallback pass estimates (by the mean) every candidate
    N, K, B, L = 1 << 14, 16, 64, 6
    plan, op = _pair(N, K, B, L, 5, T=3)
    rng = np.random.default_rng(5)
    j = np.arange(N)
    x = sum(a * np.exp(2j * np.pi * j * f / N) for f, a in zip([101, 2000, 7777, 12001], [1.0, -0.8j, 0.9, 0.7 + 0.7j]))
    x = (x + 1e-3 * (rng.standard_normal(N) + 1j * rng.standard_normal(N))).astype(np.complex64)
    ref = oracle.sfft(op, x, intermediates=True)
    idx, val, k = run_execute(plan, x)
    st = sfft.sfft_plan_last_stats(plan)
    assert st.fallback == 1 and st.candidates == len(ref["cand"])
    _check(idx, val, k, ref)


def test_estimate_entry_point_mean():
    N, K, B, L, seed = 1 << 14, 10, 64, 8, 6
    sig = signals.make_signal(N, K, seed, 20.0)
    plan, op = _pair(N, K, B, L, seed)
    ref = oracle.sfft(op, sig.x, intermediates=True)
    est = run_estimate(plan, ref["zhat"].astype(np.complex64), ref["cand"])
    assert rel_l2(est, ref["est"]) <= 1e-4
    assert np.max(np.abs(est - ref["est"])) <= 1e-4 * np.max(np.abs(ref["est"]))


def test_batch_mixes_estimators():
    specs = [(1 << 16, 10, 64, 8, s, e) for s, e in ((0, 0), (1, MEAN), (2, MEAN), (3, 0))]
    plans, xs, idxs, vals, ref = [], [], [], [], []
    for N, K, B, L, seed, est in specs:
        sig = signals.make_signal(N, K, seed, 20.0)
        w = configs.default_window(N, B)
        plan = sfft.sfft_plan_create_ex(N, K, B, w, L, seed, estimator=est)
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


def test_estimator_option_checks():
    N, K, B = 1 << 14, 8, 64
    w = configs.default_window(N, B)
    with pytest.raises(sfft.SfftError):
        sfft.sfft_plan_create_ex(N, K, B, w, 8, 0, estimator=2)
    with pytest.raises(sfft.SfftError):  # phase encoding has its own estimate
        sfft.sfft_plan_create_ex(N, K, B, w, 8, 0, method=sfft.SFFT_METHOD_PHASE, estimator=MEAN)
