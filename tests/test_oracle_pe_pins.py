"""Pins of the oracle's phase-encoding, iterative variant (CPU only).

sFFT3.0-style location ("Phase encoding method": a one-sample time shift
turns a lone coefficient f by exp(+2 pi i f / N) in our sign convention, so
f = arg(zhat' / zhat) N / 2 pi) inside the iterative framework ("The
iterative framework": found coefficients are subtracted before each new
bucketization).  Each pin checks the oracle against something other than
itself: numpy's FFT, the closed-form bucket identity, or the planted
spectrum of a noiseless signal.
"""
import numpy as np
import pytest

import oracle
from paper_2012_08238_gb300 import configs, signals
from test_oracle_pins import _gain_by_fft, _sparse_signal


@pytest.mark.parametrize("N,B", [(1 << 12, 16), (1 << 14, 64)])
def test_gain_full_against_numpy_fft(N, B):
    w = configs.default_window(N, B)
    g = oracle.window_taps(N, B, w)
    np.testing.assert_allclose(oracle.filter_gain_full(N, w, g), _gain_by_fft(N, w, g), atol=1e-12)


@pytest.mark.parametrize("N,B,f", [(1 << 12, 32, 777), (1 << 16, 64, 40001)])
def test_unit_shift_turns_lone_coefficient(N, B, f):
    # bucket values at tau and tau + 1 of a one-sparse signal: their ratio at
    # the coefficient's bucket is exp(+2 pi i f / N)
    w = configs.default_window(N, B)
    g = oracle.window_taps(N, B, w)
    x = _sparse_signal(N, [f], [0.6 - 0.8j])
    sigma, tau, _ = oracle.loop_params(N, 3, 7)
    for l in range(3):
        _, z0 = oracle.bucketize(N, B, w, sigma[l:l + 1], tau[l:l + 1], g, x)
        _, z1 = oracle.bucketize(N, B, w, sigma[l:l + 1], (tau[l:l + 1] + 1) % N, g, x)
        h, _ = oracle.hash_(N, B, int(sigma[l]), f)
        assert abs(z1[0][h] / z0[0][h] - np.exp(2j * np.pi * f / N)) < 1e-10


@pytest.mark.parametrize("N,B,K", [(1 << 12, 32, 6), (1 << 14, 64, 12)])
def test_subtraction_removes_known_coefficients(N, B, K):
    # the closed-form identity zhat[k] = sum_f x^_f e^{2 pi i tau f/N} G~(sigma f - kN/B):
    # subtracting every planted coefficient leaves nothing
    w = configs.default_window(N, B)
    g = oracle.window_taps(N, B, w)
    Gfull = oracle.filter_gain_full(N, w, g)
    rng = np.random.default_rng(N + K)
    freqs = rng.choice(N, K, replace=False)
    coefs = np.exp(2j * np.pi * rng.random(K))
    x = _sparse_signal(N, freqs, coefs)
    sigma, tau, _ = oracle.loop_params(N, 2, 3)
    for l in range(2):
        for t in (int(tau[l]), int(tau[l] + 1) % N):
            _, zhat = oracle.bucketize(N, B, w, sigma[l:l + 1], np.array([t], np.int64), g, x)
            z = np.array(zhat[0], dtype=np.complex128, copy=True)
            scale = np.max(np.abs(z))
            oracle.pe_subtract(N, B, sigma[l], t, Gfull, freqs, coefs, z)
            assert np.max(np.abs(z)) < 1e-10 * scale
            # and subtracting half of each leaves half of the bucket values
            _, zhat = oracle.bucketize(N, B, w, sigma[l:l + 1], np.array([t], np.int64), g, x)
            z = np.array(zhat[0], dtype=np.complex128, copy=True)
            oracle.pe_subtract(N, B, sigma[l], t, Gfull, freqs, 0.5 * coefs, z)
            np.testing.assert_allclose(z, 0.5 * zhat[0], atol=1e-10 * scale)


def test_locate_finds_lone_coefficients():
    N, B = 1 << 14, 64
    w = configs.default_window(N, B)
    g = oracle.window_taps(N, B, w)
    Gfull = oracle.filter_gain_full(N, w, g)
    sigma, tau, _ = oracle.loop_params(N, 1, 11)
    # coefficients in distinct buckets of this loop
    rng = np.random.default_rng(5)
    freqs, used = [], set()
    while len(freqs) < 8:
        f = int(rng.integers(N))
        h, _ = oracle.hash_(N, B, int(sigma[0]), f)
        if h not in used and (h + 1) % B not in used and (h - 1) % B not in used:
            used.add(h)
            freqs.append(f)
    coefs = np.exp(2j * np.pi * rng.random(8))
    x = _sparse_signal(N, freqs, coefs)
    _, z0 = oracle.bucketize(N, B, w, sigma, tau, g, x)
    _, z1 = oracle.bucketize(N, B, w, sigma, (tau + 1) % N, g, x)
    f, v, active = oracle.pe_locate(N, B, sigma[0], tau[0], Gfull, z0[0], z1[0], 1e-6 * np.max(np.abs(z0)) ** 2)
    order = np.argsort(f)
    assert sorted(freqs) == f[order].tolist()
    want = dict(zip(freqs, coefs))
    assert max(abs(vv - want[ff]) for ff, vv in zip(f, v)) < 1e-4
    assert active >= 8


@pytest.mark.parametrize("N,K,B,seeds", [(1 << 12, 5, 32, range(6)), (1 << 16, 10, 64, range(4)),
                                         (1 << 16, 50, 256, range(2))])
def test_exact_recovery_noiseless(N, K, B, seeds):
    # exactly sparse signals (Table 1: sFFT3.0 targets them): every planted
    # frequency is found and valued
    w = configs.default_window(N, B)
    for seed in seeds:
        sig = signals.make_signal(N, K, seed)
        out = oracle.sfft_pe(oracle.PlanPE(N, K, B, w, 8, seed), sig.x)
        assert out["k_out"] == K
        assert np.array_equal(out["idx"], np.sort(sig.freqs))
        assert np.max(np.abs(out["val"] - sig.xhat[out["idx"]])) < 1e-4


def test_one_sparse_is_exact_and_stops():
    N, B = 1 << 14, 64
    w = configs.default_window(N, B)
    x = _sparse_signal(N, [12345], [0.3 + 0.4j])
    out = oracle.sfft_pe(oracle.PlanPE(N, 1, B, w, 8, 2), x)
    assert out["idx"].tolist() == [12345]
    assert abs(out["val"][0] - (0.3 + 0.4j)) < 1e-9
    assert out["iters"] == 2  # found in the first iteration, nothing left in the second


def test_iterations_resolve_a_collision():
    # two coefficients that share a bucket in iteration 0: the first
    # iteration cannot place them, a later one (new permutation) does
    N, B = 1 << 14, 32
    w = configs.default_window(N, B)
    sigma, _, _ = oracle.loop_params(N, 1, 4)
    f1 = 1000
    h1, _ = oracle.hash_(N, B, int(sigma[0]), f1)
    f2 = next(f for f in range(2000, N) if oracle.hash_(N, B, int(sigma[0]), f)[0] == h1)
    x = _sparse_signal(N, [f1, f2], [1.0, -1.0j])
    out = oracle.sfft_pe(oracle.PlanPE(N, 2, B, w, 8, 4), x)
    assert out["idx"].tolist() == sorted([f1, f2])
    assert out["iters"] >= 3
    np.testing.assert_allclose(out["val"], [1.0, -1.0j] if f1 < f2 else [-1.0j, 1.0], atol=1e-6)


def test_zero_signal():
    N, B = 1 << 12, 32
    out = oracle.sfft_pe(oracle.PlanPE(N, 4, B, configs.default_window(N, B), 8, 0), np.zeros(N))
    assert out["k_out"] == 0 and out["iters"] == 1
