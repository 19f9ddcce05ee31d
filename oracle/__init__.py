"""FP64 CPU oracle for the flat-window voting sparse FFT and its phase-encoding
iterative variant (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library path never does: it shares
no code with the CUDA implementation and the two never call each other.

The arithmetic lives in ``sfft_oracle.c`` (plain C99, double precision); this
module compiles it with gcc on first use and exposes numpy-friendly wrappers.
Each wrapper names the step of the method it restates; see the C header for
the paper passage behind each one.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sfft_oracle.c")
_HDR = os.path.join(_HERE, "sfft_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_int = ctypes.c_int
_p = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (gcc, -O2, no -march)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(
            ["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            _bind(lib)
            _lib = lib
    return _lib


def _bind(lib):
    """Attach argument and result types to every oracle entry point."""
    sig = {
        "oracle_philox4x64_10": (None, [_p, _p, _p]),
        "oracle_loop_params": (_int, [_i64, _int, _u64, _p, _p, _p]),
        "oracle_modinv": (_i64, [_i64, _i64]),
        "oracle_window_taps": (None, [_i64, _i64, _i64, _p]),
        "oracle_filter_gain_at": (None, [_i64, _i64, _p, _i64, _p]),
        "oracle_filter_gain": (None, [_i64, _i64, _i64, _p, _p]),
        "oracle_hash": (None, [_i64, _i64, _i64, _i64, _p, _p]),
        "oracle_permute": (None, [_i64, _i64, _i64, _p, _p]),
        "oracle_bucketize": (None, [_i64, _i64, _i64, _int, _p, _p, _p, _p, _p, _p]),
        "oracle_select": (_i64, [_i64, _i64, _p, _p]),
        "oracle_vote": (_i64, [_i64, _i64, _int, _i64, _int, _p, _p, _p, _p]),
        "oracle_estimate": (None, [_i64, _i64, _int, _p, _p, _p, _p, _i64, _p, _p, _p]),
        "oracle_estimate_ex": (None, [_i64, _i64, _int, _p, _p, _p, _p, _i64, _p, _int, _p, _p]),
        "oracle_topk": (_i64, [_i64, _p, _p, _i64, _p, _p]),
        "oracle_samples_touched": (_i64, [_i64, _i64, _int, _p, _p]),
        "oracle_dft": (None, [_i64, _p, _p]),
        "oracle_sfft": (
            _i64,
            [_i64, _i64, _i64, _i64, _int, _int, _int, _u64, _p, _p, _p, _p, _p, _p, _p,
             _p, _p, _p],
        ),
        "oracle_sfft_ex": (
            _i64,
            [_i64, _i64, _i64, _i64, _int, _int, _int, _u64, _p, _p, _p, _int, _p, _p, _p, _p,
             _p, _p, _p],
        ),
        "oracle_filter_gain_full": (None, [_i64, _i64, _p, _p]),
        "oracle_pe_subtract": (None, [_i64, _i64, _i64, _i64, _p, _i64, _p, _p, _p]),
        "oracle_pe_locate": (_i64, [_i64, _i64, _i64, _i64, _p, _p, _p, ctypes.c_double, _p, _p, _p]),
        "oracle_comb": (_i64, [_i64, _i64, _int, _p, _i64, _p, _p, _p]),
        "oracle_sfft2": (
            _i64,
            [_i64, _i64, _i64, _i64, _int, _int, _int, _i64, _int, _u64, _p, _p, _p, _p, _p, _p, _p],
        ),
        "oracle_sfft2_ex": (
            _i64,
            [_i64, _i64, _i64, _i64, _int, _int, _int, _i64, _int, _u64, _p, _p, _p, _int, _p, _p, _p, _p, _p],
        ),
        "oracle_refine": (None, [_i64, _i64, _int, _p, _p, _p, _p, _i64, _p, _int, _int, _p]),
        "oracle_bs_nshifts": (_i64, [_i64, _i64, _int]),
        "oracle_bs_shifts": (None, [_i64, _i64, _int, _p]),
        "oracle_bs_locate": (_i64, [_i64, _i64, _int, _i64, _i64, _i64, _p, _p, ctypes.c_double, ctypes.c_double,
                                    _p, _p, _p]),
        "oracle_sfft_bs": (
            _i64,
            [_i64, _i64, _i64, _i64, _int, _int, ctypes.c_double, ctypes.c_double, ctypes.c_double, _u64, _p, _p,
             _p, _p, _p, _p, _p],
        ),
        "oracle_sfft_pe": (
            _i64,
            [_i64, _i64, _i64, _i64, _int, ctypes.c_double, _u64, _p, _p, _p, _p, _p, _p, _p],
        ),
        "oracle_residual_energy": (None, [_i64, _i64, _int, _p, _p, _p, _p, _i64, _p, _p, _p, _p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args


class use_library:
    """Context manager: route every wrapper through another build of the
    oracle (used by the tests that plant a mistake in a copy of the C source)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        _load()
        self._saved = _lib
        lib = ctypes.CDLL(self.path)
        _bind(lib)
        _lib = lib
        return lib

    def __exit__(self, *exc):
        global _lib
        _lib = self._saved
        return False


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _c128(x) -> np.ndarray:
    """Complex input as contiguous complex128 (exact widening of complex64)."""
    return np.ascontiguousarray(np.asarray(x, dtype=np.complex128))


# ------------------------------------------------------------------- a0
def philox4x64_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    _load().oracle_philox4x64_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def loop_params(N: int, L: int, seed: int):
    """sigma, tau, sigma^-1 per loop (scaling method, Eq. 6-7)."""
    s = np.zeros(L, np.int64)
    t = np.zeros(L, np.int64)
    si = np.zeros(L, np.int64)
    rc = _load().oracle_loop_params(N, L, seed, _ptr(s), _ptr(t), _ptr(si))
    if rc != 0:
        raise ValueError("N must be a power of two >= 2")
    return s, t, si


def modinv(a: int, N: int) -> int:
    return int(_load().oracle_modinv(a, N))


# ------------------------------------------------------------------ a0'
def window_taps(N: int, B: int, w: int) -> np.ndarray:
    """Eq. 12 x Eq. 13 taps g[q], q in [0, w), window position m = q - w//2."""
    g = np.zeros(w, np.float64)
    _load().oracle_window_taps(N, B, w, _ptr(g))
    return g


def filter_gain(N: int, B: int, w: int, g: np.ndarray) -> np.ndarray:
    """G~(o) for o in [-N/2B, N/2B), stored at o + N/2B."""
    g = np.ascontiguousarray(g, np.float64)
    Gt = np.zeros(N // B, np.complex128)
    _load().oracle_filter_gain(N, B, w, _ptr(g), _ptr(Gt))
    return Gt


def filter_gain_at(N: int, w: int, g: np.ndarray, o: int) -> complex:
    g = np.ascontiguousarray(g, np.float64)
    out = np.zeros(1, np.complex128)
    _load().oracle_filter_gain_at(N, w, _ptr(g), o, _ptr(out))
    return complex(out[0])


# ------------------------------------------------------------------- a4
def hash_(N: int, B: int, sigma: int, f: int):
    h = np.zeros(1, np.int64)
    o = np.zeros(1, np.int64)
    _load().oracle_hash(N, B, sigma, f, _ptr(h), _ptr(o))
    return int(h[0]), int(o[0])


def permute(N: int, sigma: int, tau: int, x) -> np.ndarray:
    x = _c128(x)
    out = np.zeros(N, np.complex128)
    _load().oracle_permute(N, sigma, tau, _ptr(x), _ptr(out))
    return out


# -------------------------------------------------------------- a1 + a2
def bucketize(N, B, w, sigma, tau, g, x):
    """(z, zhat), each [L][B] complex128."""
    sigma = np.ascontiguousarray(sigma, np.int64)
    tau = np.ascontiguousarray(tau, np.int64)
    L = len(sigma)
    g = np.ascontiguousarray(g, np.float64)
    x = _c128(x)
    z = np.zeros((L, B), np.complex128)
    zhat = np.zeros((L, B), np.complex128)
    _load().oracle_bucketize(N, B, w, L, _ptr(sigma), _ptr(tau), _ptr(g), _ptr(x), _ptr(z), _ptr(zhat))
    return z, zhat


# ------------------------------------------------------------------- a3
def select(B: int, cK: int, zhat_loop) -> np.ndarray:
    zl = _c128(zhat_loop)
    sel = np.zeros(min(cK, B), np.int32)
    n = _load().oracle_select(B, cK, _ptr(zl), _ptr(sel))
    return sel[:n]


# -------------------------------------------------------------- a4 + a5
def vote(N, B, T, sigma_inv, sel):
    """(candidates in increasing f, score[N]); sel is [L][nsel]."""
    sigma_inv = np.ascontiguousarray(sigma_inv, np.int64)
    sel = np.ascontiguousarray(sel, np.int32)
    L, nsel = sel.shape
    score = np.zeros(N, np.int32)
    cand = np.zeros(N, np.int32)
    n = _load().oracle_vote(N, B, L, nsel, T, _ptr(sigma_inv), _ptr(sel), _ptr(score), _ptr(cand))
    return cand[:n].copy(), score


# ------------------------------------------------------------------- a6
MEDIAN, MEAN = 0, 1  # combinations of the per-loop estimates (a6)


def estimate(N, B, sigma, tau, Gt, zhat, cand, combine=MEDIAN):
    """(combined estimates [ncand], per-loop estimates [ncand][L]); combine is
    MEDIAN (coordinate-wise) or MEAN."""
    sigma = np.ascontiguousarray(sigma, np.int64)
    tau = np.ascontiguousarray(tau, np.int64)
    L = len(sigma)
    Gt = _c128(Gt)
    zhat = _c128(zhat)
    cand = np.ascontiguousarray(cand, np.int32)
    est = np.zeros(len(cand), np.complex128)
    per = np.zeros((len(cand), L), np.complex128)
    _load().oracle_estimate_ex(N, B, L, _ptr(sigma), _ptr(tau), _ptr(Gt), _ptr(zhat), len(cand), _ptr(cand),
                               combine, _ptr(est), _ptr(per))
    return est, per


# ------------------------------------------------------------------- a7
def topk(cand, est, K):
    cand = np.ascontiguousarray(cand, np.int32)
    est = _c128(est)
    idx = np.zeros(max(K, 1), np.int32)
    val = np.zeros(max(K, 1), np.complex128)
    n = _load().oracle_topk(len(cand), _ptr(cand), _ptr(est), K, _ptr(idx), _ptr(val))
    return idx[:n].copy(), val[:n].copy()


def samples_touched(N, w, sigma, tau) -> int:
    sigma = np.ascontiguousarray(sigma, np.int64)
    tau = np.ascontiguousarray(tau, np.int64)
    return int(_load().oracle_samples_touched(N, w, len(sigma), _ptr(sigma), _ptr(tau)))


def dft(x) -> np.ndarray:
    """Eq. 2 by the O(N^2) definition."""
    x = _c128(x)
    N = len(x)
    out = np.zeros(N, np.complex128)
    _load().oracle_dft(N, _ptr(x), _ptr(out))
    return out


# -------------------------------------------------------------- pipeline
class Plan:
    """Window taps and gains for one (N, B, w): the oracle's plan-time work."""

    def __init__(self, N, K, B, w, L, seed, c=2, T=None, estimator=MEDIAN, refine=0, residual=False):
        self.N, self.K, self.B, self.w, self.L, self.seed = N, K, B, w, L, seed
        self.c = c
        self.estimator = estimator  # MEDIAN or MEAN
        self.refine = refine        # refinement passes over the found set (0: none)
        self.residual = residual    # final residual-energy check of the output
        self.T = (L + 1) // 2 if T is None else T
        self.g = window_taps(N, B, w)
        self.Gt = filter_gain(N, B, w, self.g)
        self.sigma, self.tau, self.sigma_inv = loop_params(N, L, seed)

    @property
    def nsel(self):
        return min(self.c * self.K, self.B)


def sfft(plan: Plan, x, intermediates: bool = False):
    """Whole pipeline a0..a7.  Returns dict(idx, val, k_out[, zhat, sel, cand, est])."""
    N, K, B, L = plan.N, plan.K, plan.B, plan.L
    x = _c128(x)
    assert x.shape == (N,)
    idx = np.zeros(K, np.int32)
    val = np.zeros(K, np.complex128)
    zhat = np.zeros((L, B), np.complex128)
    sel = np.zeros((L, plan.nsel), np.int32)
    cand = np.zeros(N, np.int32) if intermediates else None
    est = np.zeros(N, np.complex128) if intermediates else None
    ncand = np.zeros(1, np.int64)
    kout = _load().oracle_sfft_ex(N, K, B, plan.w, L, plan.c, plan.T, plan.seed, _ptr(plan.g), _ptr(plan.Gt),
                                  _ptr(x), plan.estimator, _ptr(idx), _ptr(val), _ptr(zhat), _ptr(sel), _ptr(cand),
                                  _ptr(est), _ptr(ncand))
    if kout < 0:
        raise ValueError("invalid sfft parameters")
    out = {"idx": idx[:kout].copy(), "val": val[:kout].copy(), "k_out": int(kout)}
    if plan.refine:
        out["val"] = refine(plan, zhat, out["idx"], out["val"], plan.refine)
    if getattr(plan, "residual", False):
        out["residual"] = residual_energy(plan, zhat, out["idx"], out["val"])
    if intermediates:
        n = int(ncand[0])
        out.update(zhat=zhat, sel=sel, cand=cand[:n].copy(), est=est[:n].copy())
    return out


# ------------------------------------------------ sFFT3.0-style variant
def filter_gain_full(N: int, w: int, g: np.ndarray) -> np.ndarray:
    """G~(nu) for every offset nu in [0, N) (one length-N FFT of the padded window)."""
    out = np.zeros(N, np.complex128)
    _load().oracle_filter_gain_full(N, w, _ptr(np.ascontiguousarray(g, np.float64)), _ptr(out))
    return out


def pe_subtract(N, B, sigma, tau, Gfull, fidx, fval, zhat):
    """Iterative framework: remove known coefficients from one loop's bucket values (in place)."""
    fidx = np.ascontiguousarray(fidx, np.int32)
    fval = _c128(fval)
    assert zhat.dtype == np.complex128 and zhat.flags["C_CONTIGUOUS"]
    _load().oracle_pe_subtract(N, B, int(sigma), int(tau), _ptr(Gfull), len(fidx), _ptr(fidx), _ptr(fval),
                               _ptr(zhat))
    return zhat


def pe_locate(N, B, sigma, tau, Gfull, zhat0, zhat1, thr):
    """Phase-encoding location of the lone coefficients of one loop: (f, value, active buckets)."""
    f = np.zeros(B, np.int32)
    v = np.zeros(B, np.complex128)
    active = np.zeros(1, np.int64)
    n = _load().oracle_pe_locate(N, B, int(sigma), int(tau), _ptr(Gfull), _ptr(_c128(zhat0)),
                                 _ptr(_c128(zhat1)), float(thr), _ptr(f), _ptr(v), _ptr(active))
    return f[:n].copy(), v[:n].copy(), int(active[0])


class PlanPE:
    """Taps and the full gain table for one (N, B, w) of the phase-encoding variant."""

    def __init__(self, N, K, B, w, R, seed, eta=1e-6):
        self.N, self.K, self.B, self.w, self.R, self.seed, self.eta = N, K, B, w, R, seed, eta
        self.g = window_taps(N, B, w)
        self.Gfull = filter_gain_full(N, w, self.g)
        self.sigma, self.tau, self.sigma_inv = loop_params(N, R, seed)


def sfft_pe(plan: PlanPE, x):
    """Whole sFFT3.0-style pipeline.  Returns dict(idx, val, k_out, iters, nfound)."""
    x = _c128(x)
    assert x.shape == (plan.N,)
    idx = np.zeros(plan.K, np.int32)
    val = np.zeros(plan.K, np.complex128)
    iters = np.zeros(1, np.int32)
    nfound = np.zeros(1, np.int64)
    kout = _load().oracle_sfft_pe(plan.N, plan.K, plan.B, plan.w, plan.R, plan.eta, plan.seed, _ptr(plan.g),
                                  _ptr(plan.Gfull), _ptr(x), _ptr(idx), _ptr(val), _ptr(iters), _ptr(nfound))
    if kout < 0:
        raise ValueError("invalid sfft_pe parameters")
    return {"idx": idx[:kout].copy(), "val": val[:kout].copy(), "k_out": int(kout), "iters": int(iters[0]),
            "nfound": int(nfound[0])}


# ----------------------------------------------- sFFT2.0-style pre-filter
def comb(N: int, Bc: int, tau_c, nkeep: int, x):
    """Spike-train pre-filter: (kept mask [Bc] bool, energies [Bc])."""
    tau_c = np.ascontiguousarray(tau_c, np.int64)
    kept = np.zeros(Bc, np.uint8)
    E = np.zeros(Bc, np.float64)
    _load().oracle_comb(N, Bc, len(tau_c), _ptr(tau_c), nkeep, _ptr(_c128(x)), _ptr(kept), _ptr(E))
    return kept.astype(bool), E


def sfft2(plan: Plan, x, Bc: int, C: int = 2):
    """Voting pipeline behind the spike-train pre-filter.  Returns dict(idx, val, k_out, kept, ncand)."""
    x = _c128(x)
    idx = np.zeros(plan.K, np.int32)
    val = np.zeros(plan.K, np.complex128)
    kept = np.zeros(Bc, np.uint8)
    ncand = np.zeros(1, np.int64)
    zhat = np.zeros((plan.L, plan.B), np.complex128)
    kout = _load().oracle_sfft2_ex(plan.N, plan.K, plan.B, plan.w, plan.L, plan.c, plan.T, Bc, C, plan.seed,
                                   _ptr(plan.g), _ptr(plan.Gt), _ptr(x), plan.estimator, _ptr(idx), _ptr(val),
                                   _ptr(kept), _ptr(ncand), _ptr(zhat))
    if kout < 0:
        raise ValueError("invalid sfft2 parameters")
    out = {"idx": idx[:kout].copy(), "val": val[:kout].copy(), "k_out": int(kout), "kept": kept.astype(bool),
           "ncand": int(ncand[0])}
    if plan.refine:
        out["val"] = refine(plan, zhat, out["idx"], out["val"], plan.refine)
    if getattr(plan, "residual", False):
        out["residual"] = residual_energy(plan, zhat, out["idx"], out["val"])
    return out


# ------------------------------------ iterative-framework refinement
def refine(plan: Plan, zhat, idx, val, passes: int = 1):
    """Refined values of the found coefficients idx (start: val) after
    `passes` rounds of subtracting the other found coefficients from each
    loop's bucket and re-estimating (combined by plan.estimator)."""
    sigma, tau, _ = loop_params(plan.N, plan.L, plan.seed)
    Gfull = filter_gain_full(plan.N, plan.w, plan.g)
    idx = np.ascontiguousarray(idx, np.int32)
    out = _c128(np.array(val, np.complex128))
    _load().oracle_refine(plan.N, plan.B, plan.L, _ptr(sigma), _ptr(tau), _ptr(_c128(Gfull)), _ptr(_c128(zhat)),
                          len(idx), _ptr(idx), plan.estimator, passes, _ptr(out))
    return out


# ---------------------------------------- final residual-energy check
def residual_energy(plan, zhat, idx, val):
    """(e_res, e_tot): energy of the plan's L loops of bucket values zhat
    after subtracting the coefficients (idx, val) from every bucket by the
    exact bucket identity, and their energy before (Eq. 5's error left after
    recovery, seen through the buckets)."""
    sigma, tau, _ = loop_params(plan.N, plan.L, plan.seed)
    Gfull = filter_gain_full(plan.N, plan.w, plan.g)
    idx = np.ascontiguousarray(idx, np.int32)
    v = _c128(np.asarray(val, np.complex128))
    er = np.zeros(1, np.float64)
    et = np.zeros(1, np.float64)
    _load().oracle_residual_energy(plan.N, plan.B, plan.L, _ptr(sigma), _ptr(tau), _ptr(_c128(Gfull)),
                                   _ptr(_c128(zhat)), len(idx), _ptr(idx), _ptr(v), _ptr(er), _ptr(et))
    return float(er[0]), float(et[0])


# ------------------------------- sFFT4.0 / MPFFT-style search location
def bs_shifts(N: int, B: int, b: int) -> np.ndarray:
    """Shifts of the search's bucketizations: 0, then N / 2^min((j+1) b, log2(N/B))."""
    n = int(_load().oracle_bs_nshifts(N, B, b))
    s = np.zeros(n, np.int64)
    _load().oracle_bs_shifts(N, B, b, _ptr(s))
    return s


def bs_locate(N, B, b, sigma, sigma_inv, tau, Gfull, zhat, thr, rho=0.25):
    """Located (f [n], values [n], active) from the nshifts bucketizations zhat [nshifts][B]."""
    zhat = _c128(zhat)
    f = np.zeros(B, np.int32)
    v = np.zeros(B, np.complex128)
    act = np.zeros(1, np.int64)
    n = _load().oracle_bs_locate(N, B, b, int(sigma), int(sigma_inv), int(tau), _ptr(_c128(Gfull)), _ptr(zhat),
                                 float(thr), float(rho), _ptr(f), _ptr(v), _ptr(act))
    return f[:n].copy(), v[:n].copy(), int(act[0])


class PlanBS:
    """Search-location variant: R iterations at most, digits of b bits
    (1: binary search, 2: multi-scale search with l = 4)."""

    def __init__(self, N, K, B, w, R, seed, b=1, eta=1e-6, kappa=20.0, rho=0.25):
        self.N, self.K, self.B, self.w, self.R, self.seed = N, K, B, w, R, seed
        self.b, self.eta, self.kappa, self.rho = b, eta, kappa, rho
        self.g = window_taps(N, B, w)
        self.Gfull = filter_gain_full(N, w, self.g)


def sfft_bs(plan: PlanBS, x):
    """Whole search-location pipeline.  Returns dict(idx, val, k_out, iters, nfound)."""
    x = _c128(x)
    idx = np.zeros(max(plan.K, 1), np.int32)
    val = np.zeros(max(plan.K, 1), np.complex128)
    iters = np.zeros(1, np.int32)
    nfound = np.zeros(1, np.int64)
    kout = _load().oracle_sfft_bs(plan.N, plan.K, plan.B, plan.w, plan.R, plan.b, plan.eta, plan.kappa, plan.rho,
                                  plan.seed,
                                  _ptr(plan.g), _ptr(plan.Gfull), _ptr(x), _ptr(idx), _ptr(val), _ptr(iters),
                                  _ptr(nfound))
    if kout < 0:
        raise ValueError("invalid sfft_bs parameters")
    return {"idx": idx[:kout].copy(), "val": val[:kout].copy(), "k_out": int(kout), "iters": int(iters[0]),
            "nfound": int(nfound[0])}
