"""L0 / L1 / L2 error of a recovered sparse spectrum against the exact one.

The paper's platform reports L0, L1 and L2 errors of each result against the
best result but never defines them (Experimental Setup).  The reading used
here, in FP64, against the best K-term approximation y of the exact spectrum
xhat (the y of Eq. 5):

* L0 = number of locations of supp(y) missing from the recovered support;
  false positives are reported separately;
* L1 = (1/K) * sum over f in supp(y) U supp(x') of |x'_f - xhat_f|;
* L2 = || x' - xhat ||_2 restricted to the same union, and L2 / ||y||_2;
* C  = || xhat - x' ||_2 / || xhat - y ||_2 over all N bins: the constant of
  the l2/l2 guarantee of Eq. 5 (infinite for an exactly sparse xhat).
"""
from __future__ import annotations

import numpy as np


def best_k_support(xhat: np.ndarray, K: int) -> np.ndarray:
    """Indices of the K largest |xhat| (ties to the lower index), sorted."""
    mag = np.abs(xhat)
    order = np.lexsort((np.arange(len(xhat)), -mag))
    return np.sort(order[:K])


def errors(xhat: np.ndarray, K: int, idx: np.ndarray, val: np.ndarray) -> dict:
    xhat = np.asarray(xhat, np.complex128)
    idx = np.asarray(idx, np.int64)
    val = np.asarray(val, np.complex128)
    supp = best_k_support(xhat, K)
    y_norm = float(np.linalg.norm(xhat[supp]))
    union = np.union1d(supp, idx)
    rec = np.zeros(len(union), np.complex128)
    pos = np.searchsorted(union, idx)
    rec[pos] = val
    diff = rec - xhat[union]
    l0 = int(len(np.setdiff1d(supp, idx)))
    fp = int(len(np.setdiff1d(idx, supp)))
    l1 = float(np.sum(np.abs(diff)) / K)
    l2 = float(np.linalg.norm(diff))
    # Eq. 5 over all bins: ||xhat - x'||^2 = ||diff on union||^2 + ||xhat off union||^2
    off = np.ones(len(xhat), bool)
    off[union] = False
    err_full = float(np.sqrt(l2 * l2 + np.sum(np.abs(xhat[off]) ** 2)))
    tail = np.ones(len(xhat), bool)
    tail[supp] = False
    best = float(np.linalg.norm(xhat[tail]))
    return {
        "L0": l0,
        "false_pos": fp,
        "L1": l1,
        "L2": l2,
        "L2_rel": l2 / y_norm if y_norm > 0 else float("nan"),
        "C": err_full / best if best > 0 else float("inf"),
    }


def errors_sparse(K: int, supp: np.ndarray, xhat_supp: np.ndarray, idx: np.ndarray, val: np.ndarray,
                  xhat_idx: np.ndarray) -> dict:
    """L0, false positives, L1, L2 and L2_rel of errors() from the exact
    spectrum's values on the two supports only: supp = the best K-term
    support with values xhat_supp, and xhat_idx = the exact values at the
    recovered frequencies idx.  For spectra too large to hold on the host
    (C, which needs every bin, is not computed)."""
    supp = np.asarray(supp, np.int64)
    idx = np.asarray(idx, np.int64)
    union = np.union1d(supp, idx)
    exact = np.zeros(len(union), np.complex128)
    exact[np.searchsorted(union, idx)] = np.asarray(xhat_idx, np.complex128)
    exact[np.searchsorted(union, supp)] = np.asarray(xhat_supp, np.complex128)
    rec = np.zeros(len(union), np.complex128)
    rec[np.searchsorted(union, idx)] = np.asarray(val, np.complex128)
    diff = rec - exact
    y_norm = float(np.linalg.norm(np.asarray(xhat_supp, np.complex128)))
    l2 = float(np.linalg.norm(diff))
    return {
        "L0": int(len(np.setdiff1d(supp, idx))),
        "false_pos": int(len(np.setdiff1d(idx, supp))),
        "L1": float(np.sum(np.abs(diff)) / K),
        "L2": l2,
        "L2_rel": l2 / y_norm if y_norm > 0 else float("nan"),
    }

