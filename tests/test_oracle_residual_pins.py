"""Pins of the oracle's final residual-energy check (CPU only).

The check (Problem Statement of sFFT, Eq. 5: the error left after recovery)
subtracts the recovered coefficients from every bucket of every loop by the
bucket identity zhat_l[k] = sum_f xhat_f e^{+2 pi i tau_l f / N}
G~(sigma_l f - k N/B) and sums the energy left.  Pinned here against facts
computed without that identity:

* exact recovery of a noiseless signal leaves nothing (to FP64 rounding);
* with one planted coefficient f0 left out, the residual is the bucket
  energy of the lone tone at f0, folded and transformed directly in numpy
  (Eq. 11 fold of the windowed permuted samples, then numpy's FFT);
* the value of f0 with its sign flipped leaves four times that energy;
* an empty found set leaves all of it: the energy of the bucket values.
"""
import numpy as np
import pytest

import oracle
from paper_2012_08238_gb300 import signals


def _tone(N, f, v):
    j = np.arange(N)
    return v * np.exp(2j * np.pi * j * f / N)


def _numpy_bucket_energy(N, B, w, L, seed, x):
    """sum_l sum_k |FFT_B(fold of g(m) x[(sigma_l m + tau_l) mod N])|^2, written out with numpy."""
    sigma, tau, _ = oracle.loop_params(N, L, seed)
    g = oracle.window_taps(N, B, w)
    m = np.arange(w) - w // 2
    e = 0.0
    for l in range(L):
        samples = g * x[(int(sigma[l]) * m + int(tau[l])) % N]
        z = np.zeros(B, np.complex128)
        np.add.at(z, m % B, samples)
        e += float(np.sum(np.abs(np.fft.fft(z)) ** 2))
    return e


def _case(N=1 << 12, K=6, B=32, L=5, seed=3):
    w = B * 33
    sig = signals.make_signal(N, K, seed)
    x = N * np.fft.ifft(sig.xhat)  # complex128: no float32 rounding of the input
    plan = oracle.Plan(N, K, B, w, L, seed)
    _, zhat = oracle.bucketize(N, B, w, plan.sigma, plan.tau, plan.g, x)
    return plan, sig, x, zhat


def test_exact_recovery_leaves_nothing():
    plan, sig, x, zhat = _case()
    er, et = oracle.residual_energy(plan, zhat, sig.freqs, sig.coefs)
    assert et > 0 and er <= 1e-24 * et


@pytest.mark.parametrize("drop", [0, 3])
def test_planted_miss_closed_form(drop):
    plan, sig, x, zhat = _case()
    keep = np.arange(len(sig.freqs)) != drop
    er, _ = oracle.residual_energy(plan, zhat, sig.freqs[keep], sig.coefs[keep])
    f0, v0 = int(sig.freqs[drop]), sig.coefs[drop]
    want = _numpy_bucket_energy(plan.N, plan.B, plan.w, plan.L, plan.seed, _tone(plan.N, f0, v0))
    assert er == pytest.approx(want, rel=1e-9)


def test_flipped_value_leaves_four_times_the_tone():
    plan, sig, x, zhat = _case()
    v = sig.coefs.copy()
    v[2] = -v[2]
    er, _ = oracle.residual_energy(plan, zhat, sig.freqs, v)
    tone = _numpy_bucket_energy(plan.N, plan.B, plan.w, plan.L, plan.seed,
                                _tone(plan.N, int(sig.freqs[2]), sig.coefs[2]))
    assert er == pytest.approx(4.0 * tone, rel=1e-9)


def test_empty_set_leaves_the_bucket_energy():
    plan, sig, x, zhat = _case()
    er, et = oracle.residual_energy(plan, zhat, np.zeros(0, np.int32), np.zeros(0, np.complex128))
    want = _numpy_bucket_energy(plan.N, plan.B, plan.w, plan.L, plan.seed, x)
    assert er == et and et == pytest.approx(want, rel=1e-9)


def test_pipeline_reports_residual_of_its_output():
    # noiseless signal through the whole oracle: its exact recovery leaves ~nothing
    N, K, B, L, seed = 1 << 12, 5, 32, 6, 2
    sig = signals.make_signal(N, K, seed)
    out = oracle.sfft(oracle.Plan(N, K, B, B * 33, L, seed, residual=True), sig.x)
    er, et = out["residual"]
    assert np.array_equal(out["idx"], sig.freqs)
    assert er <= 1e-10 * et  # the complex64 input's rounding, not the method
