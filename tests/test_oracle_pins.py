"""Pins of the FP64 oracle against facts fixed outside it (CPU only).

Each test checks one oracle step against something the paper or the
mathematics fixes: a worked example printed in the paper, a closed form, a
library routine that computes the same mathematical object another way, a
brute-force enumeration on tiny inputs, or an invariant.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2012_08238_gb300 import metrics
from paper_2012_08238_gb300 import configs, signals
from golden_io import ints, records


# ------------------------------------------------------------------ RNG
def test_philox_known_answer():
    for line in open(__file__.replace("test_oracle_pins.py", "golden/philox4x64_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        lhs, rhs = line.split("->")
        words = [int(v, 16) for v in lhs.split()]
        want = [int(v, 16) for v in rhs.split()]
        got = oracle.philox4x64_10(words[:4], words[4:])
        assert [int(v) for v in got] == want


def _numpy_block(ctr, key):
    """Philox4x64-10 block at counter ctr from numpy, which advances its
    256-bit counter before generating each block."""
    c = sum(int(v) << (64 * i) for i, v in enumerate(ctr))
    c = (c - 1) % (1 << 256)
    prev = [(c >> (64 * i)) & (2**64 - 1) for i in range(4)]
    return np.random.Philox(key=np.array(key, np.uint64),
                            counter=np.array(prev, np.uint64)).random_raw(4)


@pytest.mark.parametrize("ctr,key", [([0, 0, 0, 0], [1, 2]), ([7, 3, 0, 9], [2**63 + 5, 11]),
                                     ([0, 2**64 - 1, 5, 0], [123456789, 0])])
def test_philox_matches_numpy(ctr, key):
    assert np.array_equal(oracle.philox4x64_10(ctr, key), _numpy_block(ctr, key))


@pytest.mark.parametrize("N", [2, 16, 1 << 16, 1 << 30])
def test_loop_params_stream_and_inverse(N):
    L, seed = 12, 0xDEADBEEF
    s, t, si = oracle.loop_params(N, L, seed)
    for l in range(L):
        r = _numpy_block([l, 0, 0, 0], [seed, 0])
        assert s[l] == 2 * (int(r[0]) % (N // 2)) + 1
        assert t[l] == int(r[1]) % N
        assert s[l] % 2 == 1 and 0 < s[l] < N and 0 <= t[l] < N
        assert (int(s[l]) * int(si[l])) % N == 1 % N
        assert si[l] == pow(int(s[l]), -1, N)


def test_modinv_bijective_small():
    N = 1 << 10
    for a in range(1, N, 2):
        inv = oracle.modinv(a, N)
        assert (a * inv) % N == 1
    m = np.arange(N)
    for sigma in (1, 3, 5, 1023):
        assert len(np.unique((sigma * m + 7) % N)) == N  # odd sigma permutes Z_N


# ----------------------------------------------------------- worked examples
def test_flat_bucket_worked_example():
    rec = dict(records("worked_examples.txt"))
    r = rec["flat_buckets"]
    N, B, sigma = int(r["N"]), int(r["B"]), int(r["sigma"])
    got = [oracle.hash_(N, B, sigma, f)[0] for f in ints(r["f"])]
    assert got == ints(r["bucket"])


def test_scaling_worked_example():
    r = dict(records("worked_examples.txt"))["scaled_positions"]
    N, sigma = int(r["N"]), int(r["sigma"])
    B = 16
    for f, p in zip(ints(r["f"]), ints(r["p"])):
        h, o = oracle.hash_(N, B, sigma, f)
        assert (h * (N // B) + o) % N == p


def test_alias_remainder_example():
    r = dict(records("worked_examples.txt"))["alias_remainder"]
    B = int(r["B"])
    assert [f % B for f in ints(r["f"])] == ints(r["r"])


def test_permutation_worked_example():
    # The paper's composite reads x'_i = x_{sigma (i - tau)}; the oracle's
    # gather reads x[(sigma m + tau') mod N]; the two agree for tau' = -sigma*tau.
    r = dict(records("worked_examples.txt"))["permuted_samples"]
    sigma, tau = int(r["sigma"]), int(r["tau"])
    N = 64
    x = np.arange(N, dtype=np.float64).astype(np.complex128)
    xp = oracle.permute(N, sigma, (-sigma * tau) % N, x)
    assert [int(xp[i].real) for i in ints(r["i"])] == ints(r["src"])


def test_permutation_dft_identity():
    # Eq. 9 for b = 0 in the gather's convention: DFT(x')_{sigma f} = xhat_f e^{+2 pi i tau f / N}
    N = 64
    rng = np.random.default_rng(1)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    xhat = np.fft.fft(x) / N
    for sigma, tau in ((3, 1), (5, 17), (63, 40)):
        xph = np.fft.fft(oracle.permute(N, sigma, tau, x)) / N
        f = np.arange(N)
        np.testing.assert_allclose(xph[(sigma * f) % N], xhat * np.exp(2j * np.pi * tau * f / N),
                                   atol=1e-12)


def test_gaussian_width_example():
    r = dict(records("worked_examples.txt"))["gaussian_width"]
    N, B = int(r["N"]), int(r["B"])
    w = configs.default_window(N, B)
    g = oracle.window_taps(N, B, w)
    m = np.arange(w) - w // 2
    gauss = g / (np.sinc(m / B) / B)  # numpy's normalised sinc: sin(pi u)/(pi u)
    ok = np.abs(np.sinc(m / B)) > 1e-3
    # recover the Gaussian width from the taps: -2 log(gauss) = (m / sigma_g)^2
    sg = np.sqrt(np.median(m[ok & (m != 0)] ** 2 / (-2 * np.log(gauss[ok & (m != 0)]))))
    assert abs(sg - float(r["sigma_g"])) < 0.01
    assert abs(w - int(r["Omega"])) <= 4  # default width lands next to the example's Omega


# ------------------------------------------------------------------ taps
@pytest.mark.parametrize("N,B", [(1 << 12, 16), (1 << 16, 64), (2048, 16)])
def test_window_taps_shape(N, B):
    w = configs.default_window(N, B)
    g = oracle.window_taps(N, B, w)
    assert g[w // 2] == pytest.approx(1.0 / B, rel=1e-15)  # Eq. 12 centre value
    m = np.arange(w) - w // 2
    sg = B * np.sqrt(np.log2(N))
    np.testing.assert_allclose(g, np.sinc(m / B) / B * np.exp(-0.5 * (m / sg) ** 2), rtol=1e-12,
                               atol=1e-300)
    np.testing.assert_allclose(g[1:][::-1], g[1:], rtol=1e-12, atol=1e-300)  # even about m = 0


def _gain_by_fft(N, w, g):
    """G~(nu) for all nu in Z_N via numpy's inverse FFT of the zero-padded taps."""
    a = np.zeros(N, np.complex128)
    m = np.arange(w) - w // 2
    np.add.at(a, m % N, g)
    return np.fft.ifft(a) * N  # sum_m g(m) e^{+2 pi i m nu / N}


@pytest.mark.parametrize("N,B", [(1 << 12, 16), (1 << 14, 64), (1 << 10, 1 << 10)])
def test_filter_gain_against_fft(N, B):
    w = min(configs.default_window(N, B), N)
    w -= w % B
    g = oracle.window_taps(N, B, w)
    Gt = oracle.filter_gain(N, B, w, g)
    full = _gain_by_fft(N, w, g)
    half = (N // B) // 2
    o = np.arange(N // B) - half
    np.testing.assert_allclose(Gt, full[o % N], atol=1e-12)


def test_filter_is_flat():
    # "the flat filter has almost no spectrum leakage": ~1 inside the bucket,
    # ~1/2 at its edges, ~0 a few Gaussian widths outside
    N, B = 1 << 16, 64
    w = configs.default_window(N, B)
    full = _gain_by_fft(N, w, oracle.window_taps(N, B, w))
    nu = (np.arange(N) + N // 2) % N - N // 2
    width = N / (2 * np.pi * B * np.sqrt(np.log2(N)))  # frequency-domain Gaussian std
    inner = np.abs(nu) <= N / (2 * B) - 5 * width
    outer = np.abs(nu) >= N / (2 * B) + 5 * width
    assert np.max(np.abs(full[inner] - 1)) < 1e-5
    assert np.max(np.abs(full[outer])) < 1e-5
    edge = full[N // (2 * B)]
    assert 0.4 < abs(edge) < 0.6


# -------------------------------------------------------------- hashing
def test_hash_rounding_brute_force():
    for N, B in ((64, 8), (1024, 16), (256, 256), (128, 2)):
        NB = N // B
        for sigma in (1, 3, 7, N - 1):
            for f in range(N):
                h, o = oracle.hash_(N, B, sigma, f)
                p = (sigma * f) % N
                hh = int(Fraction(p, NB) + Fraction(1, 2)) if NB > 1 else p  # round half up
                assert h == hh % B
                assert o == p - hh * NB
                assert -(NB // 2) <= o < NB - NB // 2


# ------------------------------------------------------- bucketization
def _sparse_signal(N, freqs, coefs):
    j = np.arange(N)
    return sum(c * np.exp(2j * np.pi * j * f / N) for f, c in zip(freqs, coefs))


@pytest.mark.parametrize("N,B,L", [(1 << 10, 16, 3), (1 << 12, 64, 2), (256, 256, 1), (1 << 12, 2, 2)])
def test_bucketize_closed_form(N, B, L):
    # zhat_l[k] = sum_f xhat_f e^{2 pi i tau f / N} G~(sigma f - k N / B), exact
    w = min(configs.default_window(N, B), N)
    w -= w % B
    rng = np.random.default_rng(N + B)
    freqs = rng.choice(N, 5, replace=False)
    coefs = np.exp(2j * np.pi * rng.random(5))
    x = _sparse_signal(N, freqs, coefs)
    g = oracle.window_taps(N, B, w)
    sigma, tau, _ = oracle.loop_params(N, L, 42)
    z, zhat = oracle.bucketize(N, B, w, sigma, tau, g, x)
    full = _gain_by_fft(N, w, g)
    k = np.arange(B)
    for l in range(L):
        want = np.zeros(B, np.complex128)
        for f, c in zip(freqs, coefs):
            want += c * np.exp(2j * np.pi * tau[l] * f / N) * full[(sigma[l] * f - k * (N // B)) % N]
        np.testing.assert_allclose(zhat[l], want, atol=1e-11)
        # the fold itself, by numpy fancy indexing, and the B-point DFT by numpy's FFT
        m = np.arange(w) - w // 2
        zz = np.zeros(B, np.complex128)
        np.add.at(zz, m % B, g * x[(sigma[l] * m + tau[l]) % N])
        np.testing.assert_allclose(z[l], zz, atol=1e-12)
        np.testing.assert_allclose(zhat[l], np.fft.fft(zz), atol=1e-11)


def test_fold_identity_eq11():
    # Eq. 11: aliasing x'_i = sum_l x_{i + lB} gives xhat'_i = xhat_{iL} (up to the 1/N vs 1/B scale)
    N, B = 256, 16
    rng = np.random.default_rng(3)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    folded = x.reshape(N // B, B).sum(axis=0)
    Lr = N // B
    np.testing.assert_allclose(np.fft.fft(folded) / B, (np.fft.fft(x) / N)[::Lr] * Lr, atol=1e-12)


def test_dft_bruteforce_and_parseval():
    N = 64
    rng = np.random.default_rng(5)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    xh = oracle.dft(x)
    np.testing.assert_allclose(xh, np.fft.fft(x) / N, atol=1e-13)
    assert np.sum(np.abs(x) ** 2) == pytest.approx(N * np.sum(np.abs(xh) ** 2), rel=1e-12)


def test_signal_generator_parseval_and_snr():
    sig = signals.make_signal(1 << 14, 20, seed=3, snr_db=10.0)
    xh = np.fft.fft(sig.x.astype(np.complex128)) / sig.N
    np.testing.assert_allclose(xh, sig.xhat, atol=1e-6)
    noise = sig.xhat.copy()
    noise[sig.freqs] -= sig.coefs
    snr = 10 * np.log10(sig.K / np.sum(np.abs(noise) ** 2))
    assert abs(snr - 10.0) < 0.2
    assert np.allclose(np.abs(sig.coefs), 1.0)


# ------------------------------------------------------------- select
def test_select_brute_force_with_ties():
    rng = np.random.default_rng(9)
    B = 64
    for trial in range(20):
        mags = rng.integers(0, 6, B).astype(np.float64)  # many exact ties
        zl = np.sqrt(mags) * np.exp(2j * np.pi * rng.random(B))
        for cK in (1, 7, 20, 64, 100):
            sel = oracle.select(B, cK, zl)
            key = (np.abs(zl) ** 2).astype(np.float32)
            want = np.lexsort((np.arange(B), -key))[: min(cK, B)]
            assert np.array_equal(sel, want)


# ---------------------------------------------------------------- vote
@pytest.mark.parametrize("N,B,L,nsel,T", [(1 << 10, 16, 6, 5, 3), (1 << 9, 32, 5, 32, 5), (256, 256, 3, 10, 1)])
def test_vote_brute_force(N, B, L, nsel, T):
    rng = np.random.default_rng(N + L)
    sigma, _, sinv = oracle.loop_params(N, L, 77)
    sel = np.stack([rng.choice(B, nsel, replace=False) for _ in range(L)]).astype(np.int32)
    cand, score = oracle.vote(N, B, T, sinv, sel)
    f = np.arange(N)
    NB = N // B
    want = np.zeros(N, np.int64)
    for l in range(L):
        p = (sigma[l] * f) % N
        h = ((p + NB // 2) // NB) % B
        want += np.isin(h, sel[l])
    assert np.array_equal(score, want)
    assert np.array_equal(cand, np.nonzero(want >= T)[0])


# ------------------------------------------------------------ estimate
@pytest.mark.parametrize("N,B,L", [(1 << 12, 16, 5), (1 << 14, 64, 8)])
def test_estimate_exact_for_one_sparse(N, B, L):
    # a single tone: every per-loop estimate equals the coefficient exactly
    w = configs.default_window(N, B)
    f0, a = 1234 % N, 0.7 * np.exp(0.4j)
    x = _sparse_signal(N, [f0], [a])
    plan = oracle.Plan(N, 1, B, w, L, seed=11)
    out = oracle.sfft(plan, x, intermediates=True)
    assert list(out["idx"]) == [f0]
    assert abs(out["val"][0] - a) < 1e-11
    est, per = oracle.estimate(N, B, plan.sigma, plan.tau, plan.Gt, out["zhat"], np.array([f0]))
    np.testing.assert_allclose(per[0], np.full(L, a), atol=1e-11)


def test_median_combination():
    N, B, L = 1 << 12, 32, 6
    w = configs.default_window(N, B)
    sig = signals.make_signal(N, 8, seed=2, snr_db=5.0)
    plan = oracle.Plan(N, 8, B, w, L, seed=2)
    out = oracle.sfft(plan, sig.x, intermediates=True)
    est, per = oracle.estimate(N, B, plan.sigma, plan.tau, plan.Gt, out["zhat"], out["cand"])
    np.testing.assert_allclose(est.real, np.median(per.real, axis=1), atol=1e-15)
    np.testing.assert_allclose(est.imag, np.median(per.imag, axis=1), atol=1e-15)
    np.testing.assert_allclose(out["est"], est, atol=1e-15)


def test_topk_brute_force():
    rng = np.random.default_rng(4)
    cand = np.sort(rng.choice(5000, 400, replace=False)).astype(np.int32)
    est = rng.integers(1, 5, 400) * np.exp(2j * np.pi * rng.random(400))  # ties in |.|
    for K in (1, 10, 399, 400, 1000):
        idx, val = oracle.topk(cand, est, K)
        key = (np.abs(est) ** 2).astype(np.float32)
        order = np.lexsort((cand, -key))[: min(K, 400)]
        want = np.sort(cand[order])
        assert np.array_equal(idx, want)
        np.testing.assert_allclose(val, est[np.searchsorted(cand, want)], atol=1e-15)


# ----------------------------------------------------------- end to end
def test_exact_recovery_noiseless():
    W = configs.EXACT_N16
    for seed in range(6):
        sig = signals.make_signal(W.N, W.K, seed)
        plan = oracle.Plan(W.N, W.K, W.B, W.window, W.L, seed)
        out = oracle.sfft(plan, sig.x)
        assert np.array_equal(out["idx"], sig.freqs)
        np.testing.assert_allclose(out["val"], sig.coefs, atol=1e-5)


@pytest.mark.slow
def test_general_sparse_l2l2_guarantee():
    W = configs.GENERAL_N20
    plan = oracle.Plan(W.N, W.K, W.B, W.window, W.L, 0)
    sig = signals.make_signal(W.N, W.K, 0, W.snr_db)
    out = oracle.sfft(plan, sig.x)
    e = metrics.errors(sig.xhat, W.K, out["idx"], out["val"])
    assert e["L0"] == 0 and e["false_pos"] == 0
    assert e["L1"] < 0.05
    assert e["C"] < 1.2  # Eq. 5 with a measured approximation factor


def test_sampling_ratio_table2():
    # Table 2: expected distinct samples N (1 - (1 - w/N)^L) for random loops
    N, B, L = 1 << 14, 64, 6
    w = 1024
    vals = []
    for seed in range(40):
        s, t, _ = oracle.loop_params(N, L, seed)
        vals.append(oracle.samples_touched(N, w, s, t))
    expect = N * (1 - (1 - w / N) ** L)
    assert abs(np.mean(vals) - expect) < 3 * np.std(vals) / np.sqrt(len(vals)) + 0.002 * expect
    s, t, _ = oracle.loop_params(N, 1, 0)
    assert oracle.samples_touched(N, w, s, t) == w  # one loop touches w distinct samples
