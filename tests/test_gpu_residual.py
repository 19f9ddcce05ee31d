"""Final residual-energy check (sfft_opts.residual) on the GPU against the FP64 oracle.

The GPU subtracts its output from the L loops' buckets in FP64 (own and
neighbouring buckets) and sums the energy left; the oracle does the same with
the exact identity over every bucket, on its own pipeline's buckets and
output.  Bucket energies agree within 1e-5 (FP32 bucket values), residual
energies within 1e-4 of each other where they are large (noise left in the
buckets, a planted miss) and within 1e-9 of the bucket energy where exact
recovery leaves only rounding.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import run_execute
from paper_2012_08238_gb300 import configs, sfft, signals

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _pair(N, K, B, L, seed, **kw):
    w = configs.default_window(N, B)
    plan = sfft.sfft_plan_create_ex(N, K, B, w, L, seed, residual=1, **kw)
    return plan, oracle.Plan(N, K, B, w, L, seed, residual=True, **kw)


def _gpu_residual(plan, x):
    idx, val, k = run_execute(plan, x)
    st = sfft.sfft_plan_last_stats(plan)
    return idx, val, st.residual_energy, st.bucket_energy


def test_exact_recovery_leaves_rounding_only():
    W = configs.EXACT_N16
    sig = signals.make_signal(W.N, W.K, 5)
    plan, op = _pair(W.N, W.K, W.B, W.L, 5)
    ref = oracle.sfft(op, sig.x)
    idx, val, er, et = _gpu_residual(plan, sig.x)
    er_o, et_o = ref["residual"]
    assert np.array_equal(idx, ref["idx"])
    assert et == pytest.approx(et_o, rel=1e-5)
    assert 0.0 <= er <= 1e-9 * et
    assert abs(er - er_o) <= 1e-9 * et_o


@pytest.mark.parametrize("N,K,B,L,snr,seed", [(1 << 18, 50, 256, 12, 20.0, 1), (1 << 16, 10, 64, 8, 10.0, 2),
                                              (1 << 20, 100, 512, 12, 20.0, 0)])
def test_noisy_residual_matches_oracle(N, K, B, L, snr, seed):
    sig = signals.make_signal(N, K, seed, snr)
    plan, op = _pair(N, K, B, L, seed)
    ref = oracle.sfft(op, sig.x)
    idx, val, er, et = _gpu_residual(plan, sig.x)
    assert np.array_equal(idx, ref["idx"])
    er_o, et_o = ref["residual"]
    assert et == pytest.approx(et_o, rel=1e-5)
    assert er == pytest.approx(er_o, rel=1e-4)
    assert er < et  # the output explains most of the bucket energy


def test_planted_miss_leaves_its_energy():
    # nine coefficients of magnitude 1 and one of 0.5: a plan for K = 9 leaves out the 0.5
    N, B, L, seed = 1 << 16, 64, 8, 11
    rng = np.random.default_rng(4)
    freqs = rng.choice(N, size=10, replace=False)
    xhat = np.zeros(N, np.complex128)
    mags = np.ones(10)
    mags[9] = 0.5
    xhat[freqs] = mags * np.exp(2j * np.pi * rng.uniform(size=10))
    x = (np.fft.ifft(xhat) * N).astype(np.complex64)
    plan, op = _pair(N, 9, B, L, seed)
    ref = oracle.sfft(op, x)
    idx, val, er, et = _gpu_residual(plan, x)
    assert np.array_equal(idx, np.sort(freqs[:9])) and np.array_equal(idx, ref["idx"])
    er_o, _ = ref["residual"]
    assert er == pytest.approx(er_o, rel=1e-4)
    # the miss is far above rounding: about 0.25 of a unit coefficient's share
    assert er > 0.01 * et


def test_batch_mixes_checking_and_plain_plans():
    N, K, B, L = 1 << 16, 10, 64, 8
    w = configs.default_window(N, B)
    plans, xs, idxs, vals, refs = [], [], [], [], []
    for i in range(4):
        sig = signals.make_signal(N, K, 40 + i, 20.0)
        plans.append(sfft.sfft_plan_create_ex(N, K, B, w, L, 40 + i, residual=i % 2))
        _, _, _ = run_execute(plans[-1], sig.x)
        refs.append(sfft.sfft_plan_last_stats(plans[-1]))
        xs.append(torch.from_numpy(sig.x).cuda())
        idxs.append(torch.zeros(K, dtype=torch.int32, device="cuda"))
        vals.append(torch.zeros(K, dtype=torch.complex64, device="cuda"))
    kout = torch.zeros(4, dtype=torch.int32, device="cuda")
    for _ in range(3):  # staging run, graph capture, replay
        sfft.sfft_execute_batch(plans, xs, idxs, vals, kout)
        torch.cuda.synchronize()
        for i, p in enumerate(plans):
            st = sfft.sfft_plan_last_stats(p)
            if i % 2:
                # (the batch may split the gather into other chunks: FP32 sums in another order)
                assert st.residual_energy == pytest.approx(refs[i].residual_energy, rel=1e-5)
                assert st.bucket_energy == pytest.approx(refs[i].bucket_energy, rel=1e-6)
            else:
                assert st.residual_energy == -1.0 and st.bucket_energy == -1.0


def test_residual_option_checks():
    N, K = 1 << 16, 8
    with pytest.raises(sfft.SfftError):  # iterative methods: no residual check
        sfft.sfft_plan_create_ex(N, K, 64, configs.default_window(N, 64), 8, 0, residual=1,
                                 method=sfft.SFFT_METHOD_PHASE)
    with pytest.raises(sfft.SfftError):  # B beyond the shared-memory residuals
        sfft.sfft_plan_create_ex(1 << 20, K, 16384, 16384 * 41, 8, 0, residual=1)
    with pytest.raises(sfft.SfftError):  # B = 2: the neighbours would be one bucket
        sfft.sfft_plan_create_ex(N, 1, 2, 2 * 37, 8, 0, residual=1)
