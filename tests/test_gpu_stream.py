"""Stream gather (sfft_opts.mode = SFFT_GATHER_STREAM) against the FP64 oracle.

Step a1 read once in sample order must give the permuted gather's bucket sums
(the same reads and taps, added in another order): bucket values within
relative L2 1e-5 of the oracle's, over shapes that cover one and several loop
groups (L B > 6144), walkers per loop from 8 to 64, segments of one to many
pieces, dense windows (w = N), odd L, the comb method and signals that are
only 8-byte aligned (the kernel's 8-byte copy path).  End to end the stream
plans match the oracle like the permuted ones; a batch mixing both modes gives
each plan its plain answer; a reseeded stream plan equals a fresh plan of the
new seed.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import rel_l2, run_bucketize, run_execute
from paper_2012_08238_gb300 import configs, sfft, signals

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

STREAM = sfft.SFFT_GATHER_STREAM

# (N, K, B, w, L, kind): kind None = exactly sparse, else an SNR in dB
SHAPES = [
    (1 << 12, 4, 64, 64 * 33, 5, None),          # smallest N; 2 clusters of one-piece segments
    (1 << 12, 8, 64, 1 << 12, 8, 10.0),          # w = N: every sample read in every loop
    (1 << 14, 10, 64, 64 * 35, 8, None),
    (1 << 16, 20, 128, 128 * 37, 12, 20.0),
    (1 << 16, 64, 256, 256 * 37, 16, 15.0),      # L B = 4096, 16 walkers per loop
    (1 << 18, 60, 512, 512 * 39, 12, 10.0),      # L B = 6144: one group
    (1 << 18, 50, 512, 512 * 39, 7, 25.0),       # odd L
    (1 << 20, 100, 512, 512 * 41, 12, 20.0),     # the headline shape
    (1 << 20, 200, 1024, 1024 * 41, 12, 20.0),   # two loop groups
    (1 << 19, 500, 2048, 2048 * 40, 8, 30.0),    # four groups of two loops
    (1 << 18, 800, 4096, 4096 * 39, 12, None),   # one loop per group, 64 walkers
    (1 << 21, 30, 128, 128 * 42, 32, 15.0),      # L = 32
]


def _x(N, K, seed, kind):
    return signals.make_signal(N, K, seed, kind).x


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"N{s[0]}_B{s[2]}_w{s[3]}_L{s[4]}")
def test_bucket_values_match_oracle(shape):
    N, K, B, w, L, kind = shape
    seed = 17
    plan = sfft.sfft_plan_create_ex(N, K, B, w, L, seed, mode=STREAM)
    op = oracle.Plan(N, K, B, w, L, seed)
    x = _x(N, K, seed, kind)
    _, zo = oracle.bucketize(N, B, w, op.sigma, op.tau, op.g, x)
    zs = run_bucketize(plan, x)
    assert rel_l2(zs, zo) <= 1e-5
    # and the permuted gather's
    zp = run_bucketize(sfft.sfft_plan_create_ex(N, K, B, w, L, seed, mode=sfft.SFFT_GATHER_PERMUTED), x)
    assert rel_l2(zs, zp) <= 1e-5


def test_eight_byte_aligned_signal():
    N, K, B, L = 1 << 18, 40, 512, 12
    w = configs.default_window(N, B)
    plan = sfft.sfft_plan_create_ex(N, K, B, w, L, 5, mode=STREAM)
    op = oracle.Plan(N, K, B, w, L, 5)
    x = _x(N, K, 5, 20.0)
    buf = torch.zeros(N + 1, dtype=torch.complex64, device="cuda")
    buf[1:] = torch.from_numpy(x.astype(np.complex64)).cuda()
    xd = buf[1:]
    assert xd.data_ptr() % 16 == 8
    zhat = torch.zeros((L, B), dtype=torch.complex64, device="cuda")
    sfft.sfft_bucketize(plan, xd, zhat)
    torch.cuda.synchronize()
    _, zo = oracle.bucketize(N, B, w, op.sigma, op.tau, op.g, x)
    assert rel_l2(zhat.cpu().numpy(), zo) <= 1e-5


@pytest.mark.parametrize("N,K,B,L,kind,seed", [(1 << 16, 10, 64, 8, None, 0), (1 << 18, 50, 256, 12, None, 1),
                                               (1 << 20, 100, 512, 12, 20.0, 0), (1 << 18, 50, 256, 12, 15.0, 2),
                                               (1 << 20, 300, 1024, 12, 25.0, 3)])
def test_execute_matches_oracle(N, K, B, L, kind, seed):
    w = configs.default_window(N, B)
    plan = sfft.sfft_plan_create_ex(N, K, B, w, L, seed, mode=STREAM)
    sig = signals.make_signal(N, K, seed, kind)
    ref = oracle.sfft(oracle.Plan(N, K, B, w, L, seed), sig.x)
    idx, val, k = run_execute(plan, sig.x)
    assert k == ref["k_out"]
    common, gi, oi = np.intersect1d(idx, ref["idx"], return_indices=True)
    if kind is None:
        assert np.array_equal(idx, ref["idx"]) and np.array_equal(idx, sig.freqs)
    else:
        # (rounding-order differences may swap near ties at the K-th place)
        assert len(common) >= 0.999 * len(ref["idx"]) - 1
    assert rel_l2(val[gi], ref["val"][oi]) <= 1e-4


def test_comb_method_with_stream_gather():
    N, K, B, L = 1 << 18, 20, 256, 8
    w = configs.default_window(N, B)
    COMB = sfft.SFFT_METHOD_COMB
    sig = signals.make_signal(N, K, 8)
    plan = sfft.sfft_plan_create_ex(N, K, B, w, L, 8, method=COMB, comb=1024, mode=STREAM)
    ref = oracle.sfft2(oracle.Plan(N, K, B, w, L, 8), sig.x, 1024)
    idx, val, k = run_execute(plan, sig.x)
    assert k == ref["k_out"] and np.array_equal(idx, ref["idx"])
    assert rel_l2(val, ref["val"]) <= 1e-4


def _close(a, b, tol=1e-5):
    if not np.array_equal(a[0], b[0]):
        return False
    va, vb = np.asarray(a[1], np.complex128), np.asarray(b[1], np.complex128)
    return np.linalg.norm(va - vb) <= tol * max(np.linalg.norm(vb), 1e-30)


def test_batch_mixes_gather_modes():
    specs = [(1 << 16, 10, 64, s % 2, 0) for s in range(4)] + [(1 << 18, 30, 256, 1, 0), (1 << 18, 30, 256, 0, 0),
                                                               (1 << 20, 100, 512, 1, 0), (1 << 20, 100, 512, 1, 1),
                                                               (1 << 17, 40, 1024, 1, 0)]
    plans, xs, idxs, vals, refs = [], [], [], [], []
    for i, (N, K, B, stream, prec) in enumerate(specs):
        w = configs.default_window(N, B)
        sig = signals.make_signal(N, K, 300 + i, 25.0)
        plans.append(sfft.sfft_plan_create_ex(N, K, B, w, 12, 300 + i, precision=prec,
                                              mode=STREAM if stream else sfft.SFFT_GATHER_PERMUTED))
        refs.append(run_execute(plans[-1], sig.x)[:2])
        xs.append(torch.from_numpy(sig.x).cuda())
        idxs.append(torch.full((K,), -1, dtype=torch.int32, device="cuda"))
        vals.append(torch.zeros(K, dtype=torch.complex64, device="cuda"))
    kout = torch.zeros(len(specs), dtype=torch.int32, device="cuda")
    for _ in range(3):  # staging run, capture, replay
        sfft.sfft_execute_batch(plans, xs, idxs, vals, kout)
        torch.cuda.synchronize()
        k = kout.cpu().numpy()
        for i, ref in enumerate(refs):
            got = (idxs[i].cpu().numpy()[: k[i]], vals[i].cpu().numpy()[: k[i]])
            assert _close(got, ref), i


def test_reseeded_stream_plan_equals_fresh_plan():
    N, K, B, L = 1 << 18, 40, 256, 12
    w = configs.default_window(N, B)
    sig = signals.make_signal(N, K, 77)
    plan = sfft.sfft_plan_create_ex(N, K, B, w, L, 1, mode=STREAM)
    run_execute(plan, sig.x)
    sfft.sfft_plan_reseed(plan, 77)
    got = run_execute(plan, sig.x)
    fresh = run_execute(sfft.sfft_plan_create_ex(N, K, B, w, L, 77, mode=STREAM), sig.x)
    assert _close(got[:2], fresh[:2])
    ref = oracle.sfft(oracle.Plan(N, K, B, w, L, 77), sig.x)
    assert np.array_equal(got[0], ref["idx"])


def test_large_signal_bucket_values():
    # N = 2^24, B = 4096 (one loop per group), against the oracle's bucket sums
    N, K, B, L = 1 << 24, 1000, 4096, 12
    w = configs.default_window(N, B)
    plan = sfft.sfft_plan_create_ex(N, K, B, w, L, 9, mode=STREAM)
    op = oracle.Plan(N, K, B, w, L, 9)
    x = _x(N, K, 9, 20.0)
    _, zo = oracle.bucketize(N, B, w, op.sigma, op.tau, op.g, x)
    assert rel_l2(run_bucketize(plan, x), zo) <= 1e-5
