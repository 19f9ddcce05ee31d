"""Iterative-framework refinement (sfft_opts.refine) on the GPU against the FP64 oracle.

After the top K, each pass re-estimates every found coefficient in every
loop after subtracting the other found coefficients of the same or a
neighbouring bucket, and combines the loops as the plan does.  The oracle
subtracts every other found coefficient by the exact bucket identity; the
GPU's three-bucket table leaves out gains below the flat window's stop-band
floor.  Supports are those of the unrefined run; values stay within relative
L2 1e-4 of the oracle's.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import rel_l2, run_execute
from paper_2012_08238_gb300 import configs, metrics, sfft, signals
from test_oracle_refine_pins import _colliding
from test_oracle_pins import _sparse_signal

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MEAN, MEDIAN = sfft.SFFT_ESTIMATOR_MEAN, sfft.SFFT_ESTIMATOR_MEDIAN


def _pair(N, K, B, L, seed, est, passes, method=sfft.SFFT_METHOD_VOTING, comb=0):
    w = configs.default_window(N, B)
    plan = sfft.sfft_plan_create_ex(N, K, B, w, L, seed, method=method, comb=comb, estimator=est, refine=passes)
    return plan, oracle.Plan(N, K, B, w, L, seed, estimator=est, refine=passes)


@pytest.mark.parametrize("N,K,B,L,est,passes,snr,seed", [
    (1 << 14, 10, 64, 8, MEDIAN, 2, 20.0, 0),
    (1 << 16, 20, 256, 12, MEAN, 3, 20.0, 1),
    (1 << 12, 5, 16, 5, MEAN, 2, 30.0, 2),     # B < 32, odd L
    (1 << 16, 16, 1024, 8, MEDIAN, 1, 30.0, 3),  # B > 512
])
def test_refine_matches_oracle(N, K, B, L, est, passes, snr, seed):
    sig = signals.make_signal(N, K, seed, snr)
    plan, op = _pair(N, K, B, L, seed, est, passes)
    assert plan.info.refine == passes
    ref = oracle.sfft(op, sig.x)
    idx, val, k = run_execute(plan, sig.x)
    assert k == ref["k_out"]
    common, gi, oi = np.intersect1d(idx, ref["idx"], return_indices=True)
    assert k - len(common) <= 1
    assert rel_l2(val[gi], ref["val"][oi]) <= 1e-4


def test_refine_removes_collisions_noiseless():
    # coefficients placed to collide with one another in every loop: the
    # refined values equal the planted ones to FP32 rounding
    N, B, L, seed = 1 << 14, 32, 6, 4
    freqs, _ = _colliding(N, B, L, seed)
    coefs = np.exp(2j * np.pi * np.random.default_rng(1).random(len(freqs)))
    x = _sparse_signal(N, freqs, coefs).astype(np.complex64)
    w = configs.default_window(N, B)
    plain = sfft.sfft_plan_create_ex(N, len(freqs), B, w, L, seed)
    refined = sfft.sfft_plan_create_ex(N, len(freqs), B, w, L, seed, refine=4)
    i0, v0, _ = run_execute(plain, x)
    i1, v1, _ = run_execute(refined, x)
    assert np.array_equal(i0, freqs) and np.array_equal(i1, freqs)
    assert np.max(np.abs(v0 - coefs)) > 0.1
    assert np.max(np.abs(v1 - coefs)) < 1e-4


def test_refine_behind_comb():
    N, K, B, L, Bc, seed = 1 << 16, 10, 64, 8, 256, 5
    sig = signals.make_signal(N, K, seed, 20.0)
    plan, op = _pair(N, K, B, L, seed, MEAN, 2, method=sfft.SFFT_METHOD_COMB, comb=Bc)
    ref = oracle.sfft2(op, sig.x, Bc)
    idx, val, k = run_execute(plan, sig.x)
    common, gi, oi = np.intersect1d(idx, ref["idx"], return_indices=True)
    assert k == ref["k_out"] and k - len(common) <= 1
    assert rel_l2(val[gi], ref["val"][oi]) <= 1e-4


def test_general_workload_mean_refined():
    W = configs.GENERAL_N20
    sig = signals.make_signal(W.N, W.K, 0, W.snr_db)
    plan, op = _pair(W.N, W.K, W.B, W.L, 0, MEAN, 2)
    ref = oracle.sfft(op, sig.x)
    idx, val, k = run_execute(plan, sig.x)
    common, gi, oi = np.intersect1d(idx, ref["idx"], return_indices=True)
    assert k - len(common) <= 1
    assert rel_l2(val[gi], ref["val"][oi]) <= 1e-4
    e = metrics.errors(sig.xhat, W.K, idx, val)
    assert e["L0"] <= 1


def test_batch_mixes_refining_plans():
    specs = [(1 << 16, 10, 64, 8, s, e, r) for s, e, r in ((0, MEDIAN, 0), (1, MEAN, 2), (2, MEDIAN, 1), (3, MEAN, 0))]
    plans, xs, idxs, vals, ref = [], [], [], [], []
    for N, K, B, L, seed, est, passes in specs:
        sig = signals.make_signal(N, K, seed, 20.0)
        w = configs.default_window(N, B)
        plan = sfft.sfft_plan_create_ex(N, K, B, w, L, seed, estimator=est, refine=passes)
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


def test_refine_option_checks():
    N, K, B = 1 << 14, 8, 64
    w = configs.default_window(N, B)
    with pytest.raises(sfft.SfftError):
        sfft.sfft_plan_create_ex(N, K, B, w, 8, 0, refine=sfft.SFFT_MAX_REFINE + 1)
    with pytest.raises(sfft.SfftError):
        sfft.sfft_plan_create_ex(N, K, B, w, 8, 0, method=sfft.SFFT_METHOD_PHASE, refine=1)
    with pytest.raises(sfft.SfftError):  # the found set must fit shared memory
        sfft.sfft_plan_create_ex(1 << 20, 5000, 8192, configs.default_window(1 << 20, 8192), 8, 0, refine=1)
