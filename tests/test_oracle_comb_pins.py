"""Pins of the oracle's spike-train pre-filter (sFFT2.0-style; CPU only).

Subsampling at stride N/Bc aliases the spectrum into residue classes (Eq. 10,
Eq. 16): the comb's Bc-point DFT (with 1/Bc) at shift tau holds, for class i,
the sum over f = i (mod Bc) of x^_f e^{+2 pi i tau f / N}.  The pins check
the class energies against that closed form, the kept classes against brute
force, and the filtered pipeline against the plain voting candidates.
"""
import numpy as np
import pytest

import oracle
from paper_2012_08238_gb300 import configs, signals
from test_oracle_pins import _sparse_signal


@pytest.mark.parametrize("N,Bc,K", [(1 << 12, 64, 7), (1 << 14, 256, 20)])
def test_comb_energy_closed_form(N, Bc, K):
    rng = np.random.default_rng(N + Bc)
    freqs = rng.choice(N, K, replace=False)
    coefs = rng.standard_normal(K) + 1j * rng.standard_normal(K)
    x = _sparse_signal(N, freqs, coefs)
    taus = np.array([5, 1234], np.int64)
    kept, E = oracle.comb(N, Bc, taus, 3, x)
    want = np.zeros(Bc)
    for t in taus:
        y = np.zeros(Bc, np.complex128)
        np.add.at(y, freqs % Bc, coefs * np.exp(2j * np.pi * t * freqs / N))
        want += np.abs(y) ** 2
    np.testing.assert_allclose(E, want, rtol=1e-9, atol=1e-9)


def test_comb_keeps_largest_classes_with_ties():
    N, Bc = 1 << 10, 32
    # equal energies in classes 3, 9 and 20 and a larger one in class 7: keeping 3 takes 7, then 3 and 9
    x = _sparse_signal(N, [3, 9, 20, 7], [1.0, 1.0, -1.0, 2.0])
    kept, E = oracle.comb(N, Bc, np.array([0], np.int64), 3, x)
    assert sorted(np.flatnonzero(kept).tolist()) == [3, 7, 9]
    # brute force on random energies: the nkeep largest float32 keys, ties to the lower class
    rng = np.random.default_rng(1)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    kept, E = oracle.comb(N, Bc, np.array([0, 17], np.int64), 10, x)
    key = np.sqrt(E) ** 2
    order = sorted(range(Bc), key=lambda i: (-np.float32(key[i]), i))[:10]
    assert sorted(order) == np.flatnonzero(kept).tolist()


@pytest.mark.parametrize("seed", [0, 1])
def test_filtered_candidates_are_voting_candidates_in_kept_classes(seed):
    N, K, B, L, Bc = 1 << 14, 8, 64, 8, 128
    w = configs.default_window(N, B)
    sig = signals.make_signal(N, K, seed, 20.0)
    plan = oracle.Plan(N, K, B, w, L, seed)
    full = oracle.sfft(plan, sig.x, intermediates=True)
    out = oracle.sfft2(plan, sig.x, Bc)
    filt = [f for f in full["cand"] if out["kept"][f % Bc]]
    assert out["ncand"] == len(filt)
    # the comb shifts are the tau of loops L and L + 1
    _, tau, _ = oracle.loop_params(N, L + 2, seed)
    kept, _ = oracle.comb(N, Bc, tau[L:L + 2], min(2 * K, Bc), sig.x)
    assert np.array_equal(kept, out["kept"])
    # every planted frequency's class is kept, and the answer is the planted support
    assert out["kept"][sig.freqs % Bc].all()
    assert np.array_equal(out["idx"], np.sort(sig.freqs))


@pytest.mark.parametrize("N,K,B,L,Bc", [(1 << 16, 10, 64, 8, 256), (1 << 14, 20, 128, 8, 512)])
def test_exact_recovery_noiseless(N, K, B, L, Bc):
    w = configs.default_window(N, B)
    for seed in range(3):
        sig = signals.make_signal(N, K, seed)
        out = oracle.sfft2(oracle.Plan(N, K, B, w, L, seed), sig.x, Bc)
        assert np.array_equal(out["idx"], np.sort(sig.freqs))
        assert np.max(np.abs(out["val"] - sig.xhat[out["idx"]])) < 1e-6
