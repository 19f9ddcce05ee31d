"""The stream gather's sampling geometry (sfft_window_walk) against brute force.

Loop (sigma, tau) reads sample p with tap q(p) = (sigma^-1 (p - tau) + w/2)
mod N when q(p) < w; these are exactly the samples (sigma m + tau) mod N,
m = q - w/2, of the permuted gather (step a1).  The return map (three-distance
theorem) must step from each read to the next one in sample order, and the
first read at or after p0 must be the first such sample.  Host only.
"""
import numpy as np
import pytest

from paper_2012_08238_gb300 import sfft


def reads_brute(N, w, sigma, tau):
    """Sorted samples the window reads and their taps, from the gather's definition."""
    q = np.arange(w, dtype=np.int64)
    p = (sigma * (q - w // 2) + tau) % N
    order = np.argsort(p)
    return p[order], q[order]


def check_walk(N, w, sigma, tau, p0):
    p_s, q_s = reads_brute(N, w, sigma, tau)
    first, q1, kp, alpha, km, beta = sfft.sfft_window_walk(N, w, sigma, tau, p0)
    # first read at or after p0, cyclically
    i = int(np.searchsorted(p_s, p0))
    i = i % len(p_s)
    assert (first, q1) == (int(p_s[i]), int(q_s[i]))
    # minimality of the return times and their displacements
    s = pow(sigma, -1, N) if N > 1 else 1
    assert 0 < alpha < w or (w == N and alpha == s % N)
    assert (kp * s) % N == alpha and (N - (km * s) % N) == beta
    if N <= 4096:
        k = np.arange(1, N, dtype=np.int64)
        d = (k * s) % N
        up = k[(d > 0) & (d < w)]
        down = k[(d > N - w) & (d < N)]
        assert kp == int(up[0]) and km == int(down[0])
    # walking the return map from the first read visits every read in order
    p, q = first, q1
    n = len(p_s)
    for step in range(min(n, 5000)):
        j = (i + step) % n
        assert (p % N, q) == (int(p_s[j]), int(q_s[j])), (step, p, q)
        if q + alpha < w:
            p, q = p + kp, q + alpha
        elif q >= beta:
            p, q = p + km, q - beta
        else:
            p, q = p + kp + km, q + alpha - beta


@pytest.mark.parametrize("N", [2, 4, 16, 64, 256, 1024, 4096])
def test_walk_small_exhaustive_sigmas(N):
    rng = np.random.default_rng(N)
    sigmas = range(1, N, 2) if N <= 256 else [1, N - 1, 3, N // 2 + 1] + [int(v) | 1 for v in rng.integers(0, N, 24)]
    for sigma in sigmas:
        for w in sorted({2, min(N, 3), min(N, N // 8 + 2), N // 2, N}):
            if w < 2:
                continue
            tau = int(rng.integers(0, N))
            p0 = int(rng.integers(0, N))
            check_walk(N, w, sigma, tau, p0)


@pytest.mark.parametrize("logN,B,extra", [(12, 64, 33), (14, 256, 35), (16, 512, 37), (20, 512, 41),
                                          (24, 4096, 45), (30, 16384, 51)])
def test_walk_plan_shapes(logN, B, extra):
    N = 1 << logN
    w = min(N, B * extra) // B * B
    sig, tau, _ = sfft.sfft_loop_params(N, 6, 1234 + logN)
    rng = np.random.default_rng(logN)
    for l in range(6):
        for p0 in (0, N - 1, int(rng.integers(0, N))):
            first, q1, kp, alpha, km, beta = sfft.sfft_window_walk(N, w, sig[l], tau[l], p0)
            # the first read: a read, and no read in [p0, first)
            s = pow(sig[l], -1, N)
            qp = lambda p: (s * (p - tau[l]) + w // 2) % N  # noqa: E731
            assert qp(first) == q1 < w
            gap = (first - p0) % N
            if gap <= 1 << 20:
                ps = (p0 + np.arange(gap, dtype=np.int64)) % N
                qs = (s * (ps - tau[l]) + w // 2) % N
                assert not np.any(qs < w)
            # the return map from it lands on reads, with no read skipped
            p, q = first, q1
            for _ in range(200):
                d = kp if q + alpha < w else (km if q >= beta else kp + km)
                q2 = q + alpha if q + alpha < w else (q - beta if q >= beta else q + alpha - beta)
                if d <= 1 << 16:
                    ps = (p + 1 + np.arange(d - 1, dtype=np.int64)) % N
                    assert not np.any((s * (ps - tau[l]) + w // 2) % N < w)
                p = (p + d) % N
                q = q2
                assert qp(p) == q < w


def test_walk_rejects_bad_arguments():
    for args in [(3, 2, 1, 0, 0), (16, 1, 1, 0, 0), (16, 17, 1, 0, 0), (16, 8, 2, 0, 0), (16, 8, 1, 16, 0),
                 (16, 8, 1, 0, 16), (16, 8, 17, 0, 0)]:
        with pytest.raises(sfft.SfftError):
            sfft.sfft_window_walk(*args)


def test_stream_mode_option_checks():
    # (refused before any device work: EINVAL here too, without a GPU)
    N, K = 1 << 16, 8
    w = 64 * 37
    bad = [(N, 64, w, dict(mode=3)),  # unknown mode
           # the iterative methods read with their own gathers
           (N, 64, w, dict(mode=sfft.SFFT_GATHER_STREAM, method=sfft.SFFT_METHOD_PHASE)),
           (1 << 11, 64, 64 * 16, dict(mode=sfft.SFFT_GATHER_STREAM)),  # N below 2^12
           (1 << 22, 8192, 8192 * 43, dict(mode=sfft.SFFT_GATHER_STREAM))]  # B above 4096
    for n, b, ww, kw in bad:
        with pytest.raises(sfft.SfftError) as e:
            sfft.sfft_plan_create_ex(n, K, b, ww, 8, 0, **kw)
        assert e.value.status == 1, str(e.value)
