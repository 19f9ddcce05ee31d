"""sfft_bucketize_noalloc: bucket values without any device allocation.

This entry point serves callers that cannot call cudaMalloc while running
(their device memory belongs to another allocator, or an allocation that may
block is not allowed in their steady state), so they cannot create a plan.
It keeps its scratch in a static device array shared by all calls.  The test
calls it through the C ABI and compares it with sfft_bucketize on a plan,
within the bucket-value tolerance of the parity tests, on two calls in a row,
and with the FP64 oracle's bucket values on the small shape;
it is collected last so that a failure here stops a run only after every
other test has run, and it holds alone in a fresh process.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import rel_l2, run_bucketize
from paper_2012_08238_gb300 import configs, sfft, signals

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _noalloc(N, B, w, L, seed, x):
    xd = torch.from_numpy(np.ascontiguousarray(x, np.complex64)).cuda()
    z = torch.full((L, B), complex(np.nan, np.nan), dtype=torch.complex64, device="cuda")
    sfft.sfft_bucketize_noalloc(N, B, w, L, seed, xd, z)
    torch.cuda.synchronize()
    return z.cpu().numpy()


def test_noalloc_matches_plan_bucketize_on_consecutive_calls():
    W = configs.GENERAL_N20
    small = (1 << 12, 32, 32 * 33, 5)  # B < 256: threads share a bucket
    cases = [(W.N, W.B, W.window, W.L, 3, signals.make_signal(W.N, W.K, 3, W.snr_db).x),
             (*small, 4, signals.make_signal(small[0], 4, 4, 10.0).x)]
    refs = []
    for N, B, w, L, seed, x in cases:
        plan = sfft.sfft_plan_create(N, 4, B, w, L, seed)
        refs.append(run_bucketize(plan, x))
        plan.destroy()
    # two calls in a row on the first shape, then the other shape, then back
    for i in (0, 0, 1, 0):
        N, B, w, L, seed, x = cases[i]
        z = _noalloc(N, B, w, L, seed, x)
        assert np.isfinite(z).all()
        assert rel_l2(z, refs[i]) <= 1e-5


def test_noalloc_matches_oracle_bucket_values():
    # the same quantity from the FP64 oracle (Eq. 11 fold + Eq. 2 DFT), no plan involved
    N, B, w, L, seed = 1 << 12, 32, 32 * 33, 5, 4
    x = signals.make_signal(N, 4, seed, 10.0).x
    sigma, tau, _ = oracle.loop_params(N, L, seed)
    _, zo = oracle.bucketize(N, B, w, sigma, tau, oracle.window_taps(N, B, w), x)
    for _ in range(2):
        assert rel_l2(_noalloc(N, B, w, L, seed, x), zo) <= 1e-5


def test_noalloc_rejects_sizes_beyond_its_scratch():
    N, B, w, L = 1 << 16, 16384, 16384, 32  # L*B = 2^19 > 2^18 partial sums
    x = torch.zeros(N, dtype=torch.complex64, device="cuda")
    z = torch.zeros((L, B), dtype=torch.complex64, device="cuda")
    with pytest.raises(sfft.SfftError) as ei:
        sfft.sfft_bucketize_noalloc(N, B, w, L, 0, x, z)
    assert ei.value.status == sfft.SFFT_EINVAL
    assert "static scratch" in str(ei.value)
