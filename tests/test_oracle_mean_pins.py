"""Pins of the oracle's averaging estimator (CPU only).

Step a6 may combine the L per-loop estimates by their mean, the paper's
remark that averaging several buckets is more accurate (§ "The method of
estimating the value"), instead of the coordinate-wise median.  The pins hold
the oracle to what fixes a mean: it is exact on one-sparse signals (every
loop then estimates the coefficient itself, so a wrong scale shows), it is
linear in the signal (the median is not, which the test also shows), and on
two coefficients its value is 1/L of the summed per-loop values written out
from the closed-form bucket identity with numpy's FFT of the window.
"""
import numpy as np
import pytest

import oracle
from paper_2012_08238_gb300 import configs
from test_oracle_pins import _gain_by_fft, _sparse_signal


def _setup(N, B, L, seed):
    w = configs.default_window(N, B)
    g = oracle.window_taps(N, B, w)
    Gt = oracle.filter_gain(N, B, w, g)
    sigma, tau, sinv = oracle.loop_params(N, L, seed)
    return w, g, Gt, sigma, tau, sinv


def _mean_of(N, B, w, g, Gt, sigma, tau, x, cand):
    _, zhat = oracle.bucketize(N, B, w, sigma, tau, g, x)
    est, per = oracle.estimate(N, B, sigma, tau, Gt, zhat, cand, combine=oracle.MEAN)
    return est, per, zhat


@pytest.mark.parametrize("N,B,L,f", [(1 << 12, 16, 5, 1234), (1 << 14, 64, 8, 9999)])
def test_mean_exact_on_one_sparse(N, B, L, f):
    w, g, Gt, sigma, tau, _ = _setup(N, B, L, 3)
    c = 0.3 - 1.1j
    est, per, _ = _mean_of(N, B, w, g, Gt, sigma, tau, _sparse_signal(N, [f], [c]), np.array([f]))
    assert abs(est[0] - c) < 1e-10
    np.testing.assert_allclose(per[0], np.full(L, c), atol=1e-10)


def test_mean_is_linear_and_median_is_not():
    N, B, L = 1 << 12, 32, 7
    w, g, Gt, sigma, tau, _ = _setup(N, B, L, 11)
    rng = np.random.default_rng(0)
    f1 = rng.choice(N, 6, replace=False)
    f2 = rng.choice(N, 6, replace=False)
    x1 = _sparse_signal(N, f1, rng.standard_normal(6) + 1j * rng.standard_normal(6))
    x2 = _sparse_signal(N, f2, rng.standard_normal(6) + 1j * rng.standard_normal(6))
    x2 = x2 + 0.05 * (rng.standard_normal(N) + 1j * rng.standard_normal(N))
    cand = np.unique(np.concatenate([f1, f2, rng.choice(N, 20, replace=False)])).astype(np.int32)
    m1, _, z1 = _mean_of(N, B, w, g, Gt, sigma, tau, x1, cand)
    m2, _, z2 = _mean_of(N, B, w, g, Gt, sigma, tau, x2, cand)
    m12, _, z12 = _mean_of(N, B, w, g, Gt, sigma, tau, x1 + x2, cand)
    np.testing.assert_allclose(m12, m1 + m2, atol=1e-10)
    med = [oracle.estimate(N, B, sigma, tau, Gt, z, cand)[0] for z in (z1, z2, z12)]
    assert np.max(np.abs(med[2] - med[0] - med[1])) > 1e-3


def test_two_coefficients_closed_form():
    # a second coefficient placed to share f's bucket in loop 0 biases the
    # mean by about |c_g| / L, while the median stays at c_f
    N, B, L = 1 << 14, 32, 6
    w, g, Gt, sigma, tau, sinv = _setup(N, B, L, 5)
    f = 4321
    gq = int((f + sinv[0] * 3) % N)
    cf, cg = 1.0 + 0.5j, -0.8 + 0.6j
    x = _sparse_signal(N, [f, gq], [cf, cg])
    est, per, _ = _mean_of(N, B, w, g, Gt, sigma, tau, x, np.array([f]))
    full = _gain_by_fft(N, w, g)
    NB = N // B
    want = 0.0
    for l in range(L):
        h = (((int(sigma[l]) * f) % N + NB // 2) // NB) % B  # round half up of sigma f B / N
        gain_f = full[(int(sigma[l]) * f - h * NB) % N]
        zb = (cf * np.exp(2j * np.pi * int(tau[l]) * f / N) * gain_f
              + cg * np.exp(2j * np.pi * int(tau[l]) * gq / N) * full[(int(sigma[l]) * gq - h * NB) % N])
        want += zb * np.exp(-2j * np.pi * int(tau[l]) * f / N) / gain_f
    want /= L
    assert abs(est[0] - want) < 1e-10
    assert abs(est[0] - cf) > 0.5 * abs(cg) / L
    med = oracle.estimate(N, B, sigma, tau, Gt, oracle.bucketize(N, B, w, sigma, tau, g, x)[1], np.array([f]))[0]
    assert abs(med[0] - cf) < 1e-3


def test_mean_pipeline_recovers_noiseless():
    # the whole pipeline with the mean: exact supports and values on a
    # noiseless signal whose coefficients share no bucket and no neighbouring
    # bucket in any loop (a collision would bias the mean by 1/L of it)
    N, K, B, L, seed = 1 << 14, 8, 64, 8, 9
    sigma, _, _ = oracle.loop_params(N, L, seed)
    NB = N // B
    rng = np.random.default_rng(2)
    while True:
        freqs = np.sort(rng.choice(N, K, replace=False))
        h = np.array([[(((int(s) * int(f)) % N + NB // 2) // NB) % B for f in freqs] for s in sigma])
        d = np.abs(h[:, :, None] - h[:, None, :]) % B
        d = np.minimum(d, B - d) + 2 * np.eye(K, dtype=np.int64)[None]
        if d.min() >= 2:
            break
    coefs = np.exp(2j * np.pi * rng.random(K))
    x = _sparse_signal(N, freqs, coefs)
    w = configs.default_window(N, B)
    out = oracle.sfft(oracle.Plan(N, K, B, w, L, seed, estimator=oracle.MEAN), x)
    np.testing.assert_array_equal(out["idx"], freqs)
    np.testing.assert_allclose(out["val"], coefs, atol=1e-4)
