"""Split-BF16 tensor-core DFT (sfft_opts.precision = 1) against the FP64 oracle.

The B-point transform of step a2 runs as a tcgen05 GEMM with hi/lo BF16
splits and FP32 accumulation; the tolerance stated for it is relative L2
1e-3 (the splits leave ~2^-16).  Bucket values are compared with the
oracle's directly; end to end, supports must agree (exactly on exactly
sparse inputs, up to near ties on noisy ones) and values stay within 1e-3.
A batch mixing FP32 and split-BF16 plans gives each plan its plain answer.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import rel_l2, run_bucketize, run_execute
from paper_2012_08238_gb300 import configs, sfft, signals

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("N,K,B,L,snr", [(1 << 14, 10, 64, 8, None), (1 << 16, 20, 128, 12, 20.0),
                                         (1 << 18, 60, 512, 12, 10.0), (1 << 20, 100, 512, 12, 20.0),
                                         (1 << 18, 200, 1024, 16, 30.0), (1 << 12, 4, 64, 5, 0.0),
                                         (1 << 20, 1000, 4096, 12, 20.0)])
def test_bucket_values_within_split_bf16_tolerance(N, K, B, L, snr):
    w = configs.default_window(N, B)
    seed = 3
    plan = sfft.sfft_plan_create_ex(N, K, B, w, L, seed, precision=1)
    op = oracle.Plan(N, K, B, w, L, seed)
    x = signals.make_signal(N, K, seed, snr).x
    _, zo = oracle.bucketize(N, B, w, op.sigma, op.tau, op.g, x)
    zg = run_bucketize(plan, x)
    err = rel_l2(zg, zo)
    assert err <= 1e-3, err
    assert sfft.sfft_plan_last_stats(plan).device_error == 0
    # and consistent with the FP32 path
    z32 = run_bucketize(sfft.sfft_plan_create(N, K, B, w, L, seed), x)
    assert rel_l2(zg, z32) <= 1e-3


@pytest.mark.parametrize("N,K,B,L,snr,seed", [(1 << 16, 10, 64, 8, None, 0), (1 << 16, 10, 64, 8, None, 1),
                                              (1 << 20, 100, 512, 12, 20.0, 0), (1 << 18, 50, 256, 12, 15.0, 2)])
def test_execute_matches_oracle(N, K, B, L, snr, seed):
    w = configs.default_window(N, B)
    plan = sfft.sfft_plan_create_ex(N, K, B, w, L, seed, precision=1)
    sig = signals.make_signal(N, K, seed, snr)
    ref = oracle.sfft(oracle.Plan(N, K, B, w, L, seed), sig.x)
    idx, val, k = run_execute(plan, sig.x)
    assert k == ref["k_out"]
    common, gi, oi = np.intersect1d(idx, ref["idx"], return_indices=True)
    if snr is None:
        assert np.array_equal(idx, ref["idx"]) and np.array_equal(idx, sig.freqs)
    else:
        assert len(common) >= 0.999 * len(ref["idx"]) - 1
    assert rel_l2(val[gi], ref["val"][oi]) <= 1e-3
    assert sfft.sfft_plan_last_stats(plan).device_error == 0


def test_batch_mixes_fp32_and_split_bf16_plans():
    N, K, B, L = 1 << 16, 10, 64, 8
    w = configs.default_window(N, B)
    specs = [(s, s % 2) for s in range(6)] + [(9, 1)]
    plans, xs, idxs, vals, refs = [], [], [], [], []
    for seed, prec in specs:
        sig = signals.make_signal(N, K, 100 + seed, 25.0)
        plans.append(sfft.sfft_plan_create_ex(N, K, B, w, L, 100 + seed, precision=prec))
        refs.append(run_execute(plans[-1], sig.x)[:2])
        xs.append(torch.from_numpy(sig.x).cuda())
        idxs.append(torch.full((K,), -1, dtype=torch.int32, device="cuda"))
        vals.append(torch.zeros(K, dtype=torch.complex64, device="cuda"))
    kout = torch.zeros(len(specs), dtype=torch.int32, device="cuda")
    for _ in range(3):  # staging run, capture, replay
        sfft.sfft_execute_batch(plans, xs, idxs, vals, kout)
        torch.cuda.synchronize()
        k = kout.cpu().numpy()
        for i, (ri, rv) in enumerate(refs):
            assert np.array_equal(idxs[i].cpu().numpy()[: k[i]], ri)
            assert rel_l2(vals[i].cpu().numpy()[: k[i]], rv) <= 1e-5


def test_precision_option_checks():
    N, K = 1 << 16, 8
    w = configs.default_window(N, 64)
    for bad in (dict(precision=2), dict(precision=1, method=sfft.SFFT_METHOD_PHASE)):
        with pytest.raises(sfft.SfftError):
            sfft.sfft_plan_create_ex(N, K, 64, w, 8, 0, **bad)
    with pytest.raises(sfft.SfftError):  # B below the tensor-core tile
        sfft.sfft_plan_create_ex(N, K, 32, 32 * 37, 8, 0, precision=1)
    with pytest.raises(sfft.SfftError):  # B above the W tables kept
        sfft.sfft_plan_create_ex(1 << 20, K, 8192, 8192 * 41, 8, 0, precision=1)
