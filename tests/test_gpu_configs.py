"""The other workload shapes as parity and property tests on the GPU.

* Mixed batch (the batched shape: N log-uniform over 2^14..2^22, K uniform
  in [10, 1000] with K <= N/256, SNR uniform in [0, 40] dB, one plan per
  signal with B from the library's size-class rule sfft_suggest_params,
  which keeps the window B (log2 N + 21) below N, L = 12): the batch gives every signal the answer of its plain execution,
  and three small signals match the FP64 oracle.
* Precision sweep (N = 2^24, K = 1000, B = 4096, L = 12, SNR in
  {-10, 0, 10, 20, 40} dB, two seeds each): properties that hold at any
  size.  The support is recovered at 20 and 40 dB, and the L1 error falls as
  the SNR rises from 0 dB (the oracle comparison at this size is in
  test_gpu_fullsize.py).
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import rel_l2, run_execute
from paper_2012_08238_gb300 import configs, metrics, sfft, signals

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _size_class_B(N, K):
    return sfft.sfft_suggest_params(N, K, 20.0)[0]


def _mixed_specs(n, seed=0):
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(n):
        N = 1 << int(rng.integers(14, 23))
        K = int(rng.integers(10, min(1000, N // 256) + 1))
        snr = float(rng.uniform(0.0, 40.0))
        specs.append((N, K, _size_class_B(N, K), 12, 500 + i, snr))
    return specs


@pytest.mark.slow
def test_mixed_size_batch_equals_plain_and_oracle():
    specs = _mixed_specs(96)
    plans, xs, idxs, vals, ref, sigs = [], [], [], [], [], []
    for N, K, B, L, seed, snr in specs:
        sig = signals.make_signal(N, K, seed, snr, keep_xhat=False)
        plan = sfft.sfft_plan_create(N, K, B, configs.default_window(N, B), L, seed)
        plans.append(plan)
        ref.append(run_execute(plan, sig.x)[:2])
        xs.append(torch.from_numpy(sig.x).cuda())
        idxs.append(torch.full((K,), -1, dtype=torch.int32, device="cuda"))
        vals.append(torch.zeros(K, dtype=torch.complex64, device="cuda"))
        sigs.append(sig if N <= (1 << 17) else None)
    kout = torch.zeros(len(specs), dtype=torch.int32, device="cuda")
    for _ in range(2):  # staging run, then graph capture and replay
        sfft.sfft_execute_batch(plans, xs, idxs, vals, kout)
    torch.cuda.synchronize()
    k = kout.cpu().numpy()
    for i, (ri, rv) in enumerate(ref):
        assert np.array_equal(idxs[i].cpu().numpy()[: k[i]], ri)
        assert rel_l2(vals[i].cpu().numpy()[: k[i]], rv) <= 1e-5
    small = [i for i, s in enumerate(sigs) if s is not None][:3]
    assert len(small) == 3
    for i in small:
        N, K, B, L, seed, snr = specs[i]
        op = oracle.Plan(N, K, B, configs.default_window(N, B), L, seed)
        o = oracle.sfft(op, sigs[i].x)
        common, gi, oi = np.intersect1d(ref[i][0], o["idx"], return_indices=True)
        assert len(common) >= len(o["idx"]) - 1
        assert rel_l2(ref[i][1][gi], o["val"][oi]) <= 1e-4


@pytest.mark.slow
def test_precision_sweep_at_2p24():
    W = configs.SWEEP_N24
    plan_cache = {}
    l1, recall = {}, {}
    for snr in (-10.0, 0.0, 10.0, 20.0, 40.0):
        e1, rc = [], []
        for seed in (0, 1):
            sig = signals.make_signal(W.N, W.K, seed, snr)
            if seed not in plan_cache:
                plan_cache[seed] = sfft.sfft_plan_create(W.N, W.K, W.B, W.window, W.L, seed)
            idx, val, k = run_execute(plan_cache[seed], sig.x)
            assert k == W.K
            e = metrics.errors(sig.xhat, W.K, idx, val)
            e1.append(e["L1"])
            rc.append(1.0 - e["L0"] / W.K)
            del sig
        l1[snr], recall[snr] = float(np.mean(e1)), float(np.mean(rc))
    assert recall[20.0] >= 0.99 and recall[40.0] >= 0.99
    assert l1[0.0] > l1[10.0] > l1[20.0] > l1[40.0]
