"""Pins of the oracle's iterative-framework refinement (CPU only).

The voting output's values are refined by the iterative framework's
subtraction (§ "Four algorithmic frameworks"): each found coefficient is
re-estimated in every loop from its bucket after the other found
coefficients are subtracted by the bucket identity.  The pins: given the
true values of a noiseless signal whose coefficients collide in several
loops, one pass returns the true values to rounding (any error in the
subtraction's turn, gain offset or index shows); from the mean's biased
estimates the passes converge to the truth; a lone coefficient is left as
estimated.
"""
import numpy as np
import pytest

import oracle
from paper_2012_08238_gb300 import configs
from test_oracle_pins import _sparse_signal


def _colliding(N, B, L, seed, K=6):
    # f0 and one partner per loop l placed in f0's bucket of loop l
    _, _, sinv = oracle.loop_params(N, L, seed)
    f0 = 1000
    freqs = [f0] + [int((f0 + sinv[l] * (3 + l)) % N) for l in range(min(K - 1, L))]
    rng = np.random.default_rng(seed)
    coefs = rng.standard_normal(len(freqs)) + 1j * rng.standard_normal(len(freqs))
    order = np.argsort(freqs)
    return np.array(freqs)[order].astype(np.int32), coefs[order]


@pytest.mark.parametrize("combine", [oracle.MEDIAN, oracle.MEAN])
def test_one_pass_from_true_values_is_exact(combine):
    N, B, L, seed = 1 << 14, 32, 6, 4
    freqs, coefs = _colliding(N, B, L, seed)
    x = _sparse_signal(N, freqs, coefs)
    w = configs.default_window(N, B)
    plan = oracle.Plan(N, len(freqs), B, w, L, seed, estimator=combine)
    sigma, tau, _ = oracle.loop_params(N, L, seed)
    _, zhat = oracle.bucketize(N, B, w, sigma, tau, plan.g, x)
    # the plain estimates are off (collisions); the refined ones exact
    plain, _ = oracle.estimate(N, B, sigma, tau, plan.Gt, zhat, freqs, combine=combine)
    assert np.max(np.abs(plain - coefs)) > 1e-3
    out = oracle.refine(plan, zhat, freqs, coefs, 1)
    np.testing.assert_allclose(out, coefs, atol=1e-9)


def test_passes_remove_the_mean_bias():
    N, B, L, seed = 1 << 14, 32, 6, 4
    freqs, coefs = _colliding(N, B, L, seed)
    x = _sparse_signal(N, freqs, coefs)
    w = configs.default_window(N, B)
    plan = oracle.Plan(N, len(freqs), B, w, L, seed, estimator=oracle.MEAN)
    sigma, tau, _ = oracle.loop_params(N, L, seed)
    _, zhat = oracle.bucketize(N, B, w, sigma, tau, plan.g, x)
    v0, _ = oracle.estimate(N, B, sigma, tau, plan.Gt, zhat, freqs, combine=oracle.MEAN)
    errs = [np.max(np.abs(v0 - coefs))]
    for p in (1, 2, 4, 8):
        errs.append(np.max(np.abs(oracle.refine(plan, zhat, freqs, v0, p) - coefs)))
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-3 * errs[0]


def test_lone_coefficient_unchanged():
    N, B, L, seed = 1 << 12, 16, 5, 2
    w = configs.default_window(N, B)
    plan = oracle.Plan(N, 1, B, w, L, seed, estimator=oracle.MEAN)
    x = _sparse_signal(N, [777], [0.5 - 0.25j])
    x = x + 1e-3 * np.random.default_rng(0).standard_normal(N)
    sigma, tau, _ = oracle.loop_params(N, L, seed)
    _, zhat = oracle.bucketize(N, B, w, sigma, tau, plan.g, x)
    v, _ = oracle.estimate(N, B, sigma, tau, plan.Gt, zhat, np.array([777]), combine=oracle.MEAN)
    np.testing.assert_allclose(oracle.refine(plan, zhat, np.array([777]), v, 3), v, atol=1e-12)


def test_refined_pipeline_noiseless_with_collisions():
    # the whole pipeline on a colliding noiseless signal of unit-magnitude
    # coefficients: the median finds the support but its values carry the
    # collisions; the refinement passes return the planted values
    N, B, L, seed = 1 << 14, 32, 6, 4
    freqs, _ = _colliding(N, B, L, seed)
    coefs = np.exp(2j * np.pi * np.random.default_rng(1).random(len(freqs)))
    x = _sparse_signal(N, freqs, coefs)
    w = configs.default_window(N, B)
    plain = oracle.sfft(oracle.Plan(N, len(freqs), B, w, L, seed), x)
    out = oracle.sfft(oracle.Plan(N, len(freqs), B, w, L, seed, refine=4), x)
    np.testing.assert_array_equal(out["idx"], freqs)
    assert np.max(np.abs(plain["val"] - coefs)) > 0.1
    np.testing.assert_allclose(out["val"], coefs, atol=1e-9)
