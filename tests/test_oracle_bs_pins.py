"""Pins of the oracle's location by binary or multi-scale search (CPU only).

sFFT4.0 / MPFFT-style location (§ "The method of binary search or
multi-scale search"): a time shift of N / 2^m turns a coefficient f by
exp(2 pi i f / 2^m), so the shifted buckets decide the digits of f one at a
time (b bits each); log2(N/B) + 1 bits and the bucket fix sigma f.  The pins
check the shift schedule against its closed form, exact location of lone
coefficients (also next to a bucket edge), agreement with an exhaustive
search over the 2N/B candidates of the search window under noise, rejection of a bucket shared by two coefficients,
exact recovery of noiseless signals, and recovery where phase encoding
fails (the robustness the paper ranks above it).
"""
import numpy as np
import pytest

import oracle
from paper_2012_08238_gb300 import configs, signals
from test_oracle_pins import _sparse_signal


def _zhat(N, B, w, g, sigma, tau, shifts, x):
    rows = []
    for s in shifts:
        _, z = oracle.bucketize(N, B, w, np.array([sigma]), np.array([(tau + s) % N]), g, x)
        rows.append(z[0])
    return np.array(rows)


@pytest.mark.parametrize("N,B,b,want", [
    (1 << 16, 64, 1, [0] + [(1 << 16) >> m for m in range(1, 12)]),   # log2(N/B) + 1 = 11 bits
    (1 << 16, 64, 2, [0] + [(1 << 16) >> m for m in (2, 4, 6, 8, 10, 11)]),
    (1 << 16, 64, 3, [0] + [(1 << 16) >> m for m in (3, 6, 9, 11)]),
    (256, 256, 1, [0, 128]),  # B = N: one bit
    (256, 1, 1, [0] + [256 >> m for m in range(1, 9)]),  # B = 1: capped at log2 N
])
def test_shift_schedule(N, B, b, want):
    np.testing.assert_array_equal(oracle.bs_shifts(N, B, b), want)


@pytest.mark.parametrize("N,B,b", [(1 << 12, 16, 1), (1 << 16, 64, 1), (1 << 16, 64, 2), (1 << 14, 32, 3)])
def test_lone_coefficient_located_exactly(N, B, b):
    w = configs.default_window(N, B)
    g = oracle.window_taps(N, B, w)
    Gfull = oracle.filter_gain_full(N, w, g)
    sigma, tau, sinv = oracle.loop_params(N, 3, 8)
    shifts = oracle.bs_shifts(N, B, b)
    rng = np.random.default_rng(N + b)
    for f in rng.choice(N, 6, replace=False):
        c = np.exp(2j * np.pi * rng.random())
        for l in range(3):
            z = _zhat(N, B, w, g, sigma[l], tau[l], shifts, _sparse_signal(N, [f], [c]))
            fl, vl, act = oracle.bs_locate(N, B, b, sigma[l], sinv[l], tau[l], Gfull, z, 1e-9)
            # (near a bucket edge the neighbour holds leakage too: active, but
            # its location hashes back to the coefficient's own bucket)
            assert act >= 1 and list(fl) == [f]
            assert abs(vl[0] - c) < 1e-9


def test_matches_exhaustive_search_under_noise():
    # greedy digit decisions equal the best of all N/B candidates of the
    # bucket (smallest residual over the shifted buckets) at moderate noise
    N, B, b = 1 << 14, 32, 1
    w = configs.default_window(N, B)
    g = oracle.window_taps(N, B, w)
    Gfull = oracle.filter_gain_full(N, w, g)
    sigma, tau, sinv = oracle.loop_params(N, 1, 5)
    shifts = oracle.bs_shifts(N, B, b)
    rng = np.random.default_rng(1)
    NB = N // B
    for trial in range(5):
        f = int(rng.integers(N))
        x = _sparse_signal(N, [f], [1.0]) + 0.02 * (rng.standard_normal(N) + 1j * rng.standard_normal(N))
        z = _zhat(N, B, w, g, sigma[0], tau[0], shifts, x)
        k = int(np.argmax(np.abs(z[0])))
        cands = [(int(sinv[0]) * p) % N for p in range(k * NB - NB, k * NB + NB)]  # the search window
        res = [np.sum(np.abs(z[1:, k] - z[0, k] * np.exp(2j * np.pi * shifts[1:] * c / N)) ** 2) for c in cands]
        best = cands[int(np.argmin(res))]
        fl, _, _ = oracle.bs_locate(N, B, b, sigma[0], sinv[0], tau[0], Gfull, z, np.abs(z[0, k]) ** 2 * 0.5)
        assert best == f and list(fl) == [best]


def test_shared_bucket_rejected():
    N, B, b = 1 << 14, 32, 1
    w = configs.default_window(N, B)
    g = oracle.window_taps(N, B, w)
    Gfull = oracle.filter_gain_full(N, w, g)
    sigma, tau, sinv = oracle.loop_params(N, 1, 6)
    f = 3000
    f2 = int((f + sinv[0] * 5) % N)  # sigma f2 = sigma f + 5: the same bucket
    x = _sparse_signal(N, [f, f2], [1.0, 0.8j])
    z = _zhat(N, B, w, g, sigma[0], tau[0], oracle.bs_shifts(N, B, b), x)
    fl, _, act = oracle.bs_locate(N, B, b, sigma[0], sinv[0], tau[0], Gfull, z, 1e-6)
    assert act >= 1 and f not in fl and f2 not in fl


@pytest.mark.parametrize("b", [1, 2])
@pytest.mark.parametrize("N,K,B", [(1 << 12, 5, 32), (1 << 16, 10, 64)])
def test_exact_recovery_noiseless(N, K, B, b):
    for seed in range(3):
        sig = signals.make_signal(N, K, seed)
        out = oracle.sfft_bs(oracle.PlanBS(N, K, B, configs.default_window(N, B), 8, seed, b=b), sig.x)
        np.testing.assert_array_equal(out["idx"], np.sort(sig.freqs))
        np.testing.assert_allclose(out["val"], sig.xhat[np.sort(sig.freqs)], atol=1e-6)


def test_zero_signal():
    N, B = 1 << 12, 32
    out = oracle.sfft_bs(oracle.PlanBS(N, 4, B, configs.default_window(N, B), 8, 0), np.zeros(N, np.complex128))
    assert out["k_out"] == 0 and out["iters"] == 1


def test_recovers_where_phase_encoding_fails():
    # 20 dB noise: the phase of a one-sample shift cannot resolve f to one of
    # N bins, the sign decisions of the search can
    N, K, B = 1 << 16, 10, 64
    w = configs.default_window(N, B)
    sig = signals.make_signal(N, K, 3, 20.0)
    bs = oracle.sfft_bs(oracle.PlanBS(N, K, B, w, 8, 3), sig.x)
    pe = oracle.sfft_pe(oracle.PlanPE(N, K, B, w, 8, 3), sig.x)
    assert len(np.intersect1d(bs["idx"], sig.freqs)) == K
    assert len(np.intersect1d(pe["idx"], sig.freqs)) < K // 2


def test_pure_noise_stops_after_one_iteration():
    # the threshold's noise-floor term (20 times the median bucket energy): no
    # bucket of white noise reaches it, so nothing is located and the loop stops
    N, B = 1 << 14, 64
    rng = np.random.default_rng(7)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    out = oracle.sfft_bs(oracle.PlanBS(N, 8, B, configs.default_window(N, B), 8, 1), x)
    assert out["iters"] == 1 and out["nfound"] == 0


def test_noisy_signal_stops_early():
    # 20 dB: the planted support is found within a few iterations, then
    # nothing above the noise floor remains
    N, K, B = 1 << 16, 10, 64
    sig = signals.make_signal(N, K, 4, 20.0)
    out = oracle.sfft_bs(oracle.PlanBS(N, K, B, configs.default_window(N, B), 8, 4), sig.x)
    assert out["iters"] < 8 and len(np.intersect1d(out["idx"], sig.freqs)) == K
