"""L0 / L1 / L2 / C error definitions pinned to a hand-computed case (CPU only).

The paper's platform reports L0, L1 and L2 errors but never defines them
(Experimental Setup); the reading is in paper_2012_08238_gb300/metrics.py and
the Eq. 5 constant C is the l2/l2 guarantee's (Problem Statement of sFFT).
The case below is small enough that every figure is written out by hand:

    N = 16, K = 3, exact spectrum xhat:
        xhat[2] = 3, xhat[5] = -2i, xhat[9] = 1 + 1i      (best 3-term support)
        xhat[11] = 0.5, xhat[14] = 0.25i                  (tail)
    recovered: idx = [2, 9, 11], val = [2.9, 1 + 0.5i, 0.4]

    supp(y) = {2, 5, 9};  ||y||_2 = sqrt(9 + 4 + 2) = sqrt(15)
    L0 = |{5}| = 1 (f = 5 missed), false positives = |{11}| = 1
    union = {2, 5, 9, 11}; |x' - xhat| there = 0.1, 2, 0.5, 0.1
    L1 = (0.1 + 2 + 0.5 + 0.1) / 3 = 0.9
    L2 = sqrt(0.01 + 4 + 0.25 + 0.01) = sqrt(4.27);  L2_rel = sqrt(4.27 / 15)
    C  = sqrt(4.27 + 0.25^2) / sqrt(0.5^2 + 0.25^2) = sqrt(4.3325 / 0.3125)

Planted mistakes in a copy of the module (L1 over supp(y) only, L1 without
1/K, false positives counted into L0, C over the union instead of all N
bins, the best K-term tail taken over the union) must each break the pin.
"""
import importlib.util
import math
import os

import numpy as np
import pytest

from paper_2012_08238_gb300 import metrics

SRC = metrics.__file__


def _case():
    xhat = np.zeros(16, np.complex128)
    xhat[2], xhat[5], xhat[9], xhat[11], xhat[14] = 3.0, -2.0j, 1 + 1j, 0.5, 0.25j
    idx = np.array([2, 9, 11])
    val = np.array([2.9, 1 + 0.5j, 0.4], np.complex64)
    return xhat, idx, val


EXPECTED = {
    "L0": 1,
    "false_pos": 1,
    "L1": 0.9,
    "L2": math.sqrt(4.27),
    "L2_rel": math.sqrt(4.27 / 15.0),
    "C": math.sqrt(4.3325 / 0.3125),
}


def _check(mod):
    xhat, idx, val = _case()
    e = mod.errors(xhat, 3, idx, val)
    for k, v in EXPECTED.items():
        # complex64 inputs: 2.9, 0.4 and 0.5 carry float32 rounding (~1e-8)
        assert e[k] == pytest.approx(v, rel=1e-6, abs=1e-7), (k, e[k], v)


def test_errors_hand_computed_case():
    _check(metrics)


def test_exact_recovery_has_zero_error():
    xhat, _, _ = _case()
    supp = np.array([2, 5, 9])
    e = metrics.errors(xhat, 3, supp, xhat[supp])
    assert e["L0"] == 0 and e["false_pos"] == 0 and e["L1"] == 0.0 and e["L2"] == 0.0
    assert e["C"] == pytest.approx(1.0)  # x' = y exactly: the error is the tail itself


def test_best_support_ties_to_lower_index():
    xhat = np.array([1, 2, 2, 0, 2], np.complex128)
    assert list(metrics.best_k_support(xhat, 2)) == [1, 2]


MUTANTS = [
    ("L1 over supp(y) only", "l1 = float(np.sum(np.abs(diff)) / K)",
     "l1 = float(np.sum(np.abs(diff[np.isin(union, supp)])) / K)"),
    ("L1 without 1/K", "l1 = float(np.sum(np.abs(diff)) / K)", "l1 = float(np.sum(np.abs(diff)))"),
    ("false positives in L0", "l0 = int(len(np.setdiff1d(supp, idx)))",
     "l0 = int(len(np.setdiff1d(supp, idx))) + int(len(np.setdiff1d(idx, supp)))"),
    ("C over the union", "err_full = float(np.sqrt(l2 * l2 + np.sum(np.abs(xhat[off]) ** 2)))", "err_full = l2"),
    ("tail over the union", "tail[supp] = False", "tail[union] = False"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pin_catches_planted_mistake(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name!r} not unique"
    path = tmp_path / "metrics_mutant.py"
    path.write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location("metrics_mutant", str(path))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    with pytest.raises(AssertionError):
        _check(mod)
    assert os.path.exists(SRC)


def test_sparse_form_equals_the_full_definition():
    # the hand case, then random spectra with misses and false positives
    xhat, idx, val = _case()
    supp = metrics.best_k_support(xhat, 3)
    e = metrics.errors_sparse(3, supp, xhat[supp], idx, val, xhat[idx])
    for k in ("L0", "false_pos", "L1", "L2", "L2_rel"):
        assert e[k] == pytest.approx(EXPECTED[k], rel=1e-6, abs=1e-7), k
    rng = np.random.default_rng(7)
    for _ in range(20):
        N, K = 256, int(rng.integers(1, 20))
        xh = (rng.standard_normal(N) + 1j * rng.standard_normal(N)) * 0.01
        xh[rng.choice(N, K, replace=False)] += np.exp(2j * np.pi * rng.uniform(size=K))
        idx = np.sort(rng.choice(N, int(rng.integers(0, K + 1)), replace=False))
        val = xh[idx] + 0.05 * (rng.standard_normal(len(idx)) + 1j * rng.standard_normal(len(idx)))
        full = metrics.errors(xh, K, idx, val)
        supp = metrics.best_k_support(xh, K)
        sp = metrics.errors_sparse(K, supp, xh[supp], idx, val, xh[idx])
        for k in sp:
            assert sp[k] == pytest.approx(full[k], rel=1e-12, abs=1e-15), k

