"""The C-ABI library builds, loads and exports every declared symbol (CPU only).

Also checks the host-only parts of the library: the loop parameters it
derives from a seed (against the oracle and numpy's Philox) and the size
validation that runs before any device call.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_2012_08238_gb300 import build, sfft

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(sfft_[a-z_]+)\s*\(", text)
    return sorted(set(names))


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    assert os.path.exists(path)
    so = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(so, name), f"{name} declared in include/ but not exported"
    assert set(names) == set(sfft.EXPORTED), "binding and header disagree"


@pytest.mark.parametrize("N,L,seed", [(1 << 16, 8, 0), (1 << 20, 12, 12345), (2, 3, 7), (1 << 30, 32, 2**63 + 1)])
def test_loop_params_match_oracle(N, L, seed):
    s, t, si = sfft.sfft_loop_params(N, L, seed)
    os_, ot, osi = oracle.loop_params(N, L, seed)
    assert list(os_) == s and list(ot) == t and list(osi) == si


@pytest.mark.parametrize("args", [
    (1000, 10, 64, 2368, 8),        # N not a power of two
    (1 << 16, 10, 48, 2400, 8),     # B not a power of two
    (1 << 16, 10, 64, 2370, 8),     # w not a multiple of B
    (1 << 16, 10, 64, 32, 8),       # w < B
    (1 << 16, 10, 64, 2368, 0),     # L = 0
    (1 << 16, 10, 64, 2368, 33),    # L > 32
    (1 << 16, 0, 64, 2368, 8),      # K = 0
    (1 << 16, 20000, 64, 2368, 8),  # K > 16384
    (1 << 31, 10, 64, 2368, 8),     # N > 2^30
    (1 << 16, 10, 1 << 15, 1 << 15, 8),  # B > 16384
])
def test_invalid_sizes_rejected_before_any_device_call(args):
    with pytest.raises(sfft.SfftError) as ei:
        sfft.sfft_plan_create(*args, seed=0)
    assert ei.value.status == sfft.SFFT_EINVAL


def test_invalid_options_rejected():
    with pytest.raises(sfft.SfftError) as ei:
        sfft.sfft_plan_create_ex(1 << 16, 10, 64, 2368, 8, 0, c=1, T=9)
    assert ei.value.status == sfft.SFFT_EINVAL
    for bad in (dict(precision=2), dict(precision=1, B=32), dict(precision=1, method=sfft.SFFT_METHOD_SEARCH)):
        kw = dict(bad)
        B = kw.pop("B", 64)
        with pytest.raises(sfft.SfftError) as ei:  # refused before any device call
            sfft.sfft_plan_create_ex(1 << 16, 10, B, B * 37, 8, 0, **kw)
        assert ei.value.status == sfft.SFFT_EINVAL


def test_status_strings():
    assert sfft.status_string(sfft.SFFT_OK) == "ok"
    assert sfft.status_string(sfft.SFFT_EPENDING) == "pending"


def _c_layout(tmp_path, structs):
    """sizeof and offsetof of the header's structs, from gcc."""
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "sfft.h"', "int main(void) {"]
    for name, fields in structs.items():
        lines.append(f'    printf("{name} size %zu\\n", sizeof({name}));')
        for f in fields:
            lines.append(f'    printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess

    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    out = {}
    for line in subprocess.check_output([str(exe)]).decode().splitlines():
        key, val = line.rsplit(" ", 1)
        out[key] = int(val)
    return out


def test_binding_structs_match_the_header(tmp_path):
    # the ctypes mirrors must have the header's sizes and field offsets
    classes = [sfft.sfft_opts, sfft.sfft_plan_info, sfft.sfft_exec_stats, sfft.sfft_request, sfft.sfft_result]
    structs = {c.__name__: [f[0] for f in c._fields_] for c in classes}
    c = _c_layout(tmp_path, structs)
    for cls in classes:
        name = cls.__name__
        assert ctypes.sizeof(cls) == c[f"{name} size"], name
        for f in structs[name]:
            assert getattr(cls, f).offset == c[f"{name}.{f}"], f"{name}.{f}"


@pytest.mark.parametrize("kw", [
    dict(method=4),                                    # no such method
    dict(estimator=2),                                 # no such estimator
    dict(refine=9),                                    # at most 8 passes
    dict(refine=-1),
    dict(method=sfft.SFFT_METHOD_PHASE, refine=1),     # refinement is for voting / comb
    dict(method=sfft.SFFT_METHOD_PHASE, estimator=sfft.SFFT_ESTIMATOR_MEAN),
    dict(method=sfft.SFFT_METHOD_SEARCH, estimator=sfft.SFFT_ESTIMATOR_MEAN),
    dict(search_bits=1),                               # search_bits is for the search method
    dict(method=sfft.SFFT_METHOD_SEARCH, search_bits=5),
    dict(comb=256),                                    # comb is for the comb method
    dict(method=sfft.SFFT_METHOD_COMB, comb=1000),     # not a power of two
])
def test_invalid_variant_options_rejected(kw):
    with pytest.raises(sfft.SfftError) as ei:
        sfft.sfft_plan_create_ex(1 << 16, 10, 64, 2368, 8, 0, **kw)
    assert ei.value.status == sfft.SFFT_EINVAL


def test_refinement_and_search_size_limits_rejected():
    with pytest.raises(sfft.SfftError):  # refinement keeps the found set in shared memory: K <= 4096
        sfft.sfft_plan_create_ex(1 << 20, 5000, 8192, 8192 * 41, 8, 0, refine=1)
    with pytest.raises(sfft.SfftError):  # the search's bucket buffers must fit one CTA
        sfft.sfft_plan_create_ex(1 << 24, 8, 8192, 8192 * 45, 8, 0, method=sfft.SFFT_METHOD_SEARCH)


@pytest.mark.parametrize("N,K,snr,want", [
    (1 << 16, 10, None, (64, 64 * 37, 8)),          # the exactly sparse workload
    (1 << 20, 100, 20.0, (512, 512 * 41, 12)),      # the general workload
    (1 << 24, 1000, 20.0, (4096, 4096 * 45, 12)),   # the precision sweep
    (1 << 14, 100, 0.0, (256, 256 * 35, 12)),       # capped at N/64 (still >= 2K)
    (1 << 22, 5000, 10.0, (16384, 16384 * 43, 12)),  # capped at 16384
    (1 << 20, 4096, 10.0, (16384, 16384 * 41, 12)),  # the largest serving K
    (1 << 10, 3, None, (16, 16 * 31, 8)),           # small N: N/64
    (1 << 11, 16, None, (32, 32 * 32, 8)),          # N/64 = 2K exactly
    (32, 1, None, (2, 32, 8)),                      # tiny N: at least 2, window within N
])
def test_suggested_params_follow_the_size_class_rule(N, K, snr, want):
    B, w, L = sfft.sfft_suggest_params(N, K, snr)
    assert (B, w, L) == want
    assert w % B == 0 and w <= N


def test_suggested_params_agree_with_the_mixed_batch_rule():
    # the mixed-size batch test's rule is this entry point's
    import test_gpu_configs as tc

    for N, K, B, L, seed, snr in tc._mixed_specs(96):
        assert sfft.sfft_suggest_params(N, K, snr)[:1] == (B,)
    with pytest.raises(sfft.SfftError):
        sfft.sfft_suggest_params(1000, 10, 20.0)


@pytest.mark.parametrize("N,K", [(1 << 14, 1000), (1 << 12, 4096), (1 << 12, 33), (1 << 26, 8193)])
def test_suggested_params_refuse_K_beyond_the_rule(N, K):
    # the capped B would be below 2K (K > N/128 or K > 8192)
    with pytest.raises(sfft.SfftError) as ei:
        sfft.sfft_suggest_params(N, K, 20.0)
    assert ei.value.status == sfft.SFFT_EINVAL and "K too large" in str(ei.value)


def test_tuning_cache_overrides_the_rule_for_its_classes(tmp_path):
    import json

    path = tmp_path / "tune.json"
    path.write_text(json.dumps({"version": 1, "device": "test", "classes": [
        {"logN": 20, "K_lo": 50, "K_hi": 200, "snr_lo": 10.0, "snr_hi": 30.0, "B_per_K": 16, "w_extra": 15, "L": 8,
         "spectra_per_s": 1.0},
        {"logN": 16, "K_lo": 1, "K_hi": 20, "snr_lo": None, "snr_hi": None, "B_per_K": 32, "w_extra": 21, "L": 12}]}))
    try:
        sfft.sfft_tuning_load(path)
        assert sfft.sfft_tuning_classes() == 2
        assert sfft.sfft_suggest_params(1 << 20, 100, 20.0) == (2048, 2048 * 35, 8)  # 16 K -> 2048
        assert sfft.sfft_suggest_params(1 << 20, 100, 5.0) == (512, 512 * 41, 12)    # SNR outside: the rule
        assert sfft.sfft_suggest_params(1 << 16, 10, None) == (512, 512 * 37, 12)    # the noiseless class
        assert sfft.sfft_suggest_params(1 << 16, 10, 20.0) == (64, 64 * 37, 12)      # noisy: the rule
        assert sfft.sfft_suggest_params(1 << 20, 1000, 20.0)[0] == 4096              # K outside the class
    finally:
        sfft.sfft_tuning_clear()
    assert sfft.sfft_tuning_classes() == 0
    assert sfft.sfft_suggest_params(1 << 20, 100, 20.0) == (512, 512 * 41, 12)


@pytest.mark.parametrize("text", ['{"version": 2, "classes": []}', '{"classes": [', '[1, 2]',
                                  '{"version": 1, "classes": [{"logN": 20}]}',
                                  '{"version": 1, "classes": [{"logN": 20, "K_lo": 5, "K_hi": 1, "B_per_K": 4, '
                                  '"w_extra": 21, "L": 12}]}'])
def test_tuning_cache_rejects_malformed_files(tmp_path, text):
    path = tmp_path / "bad.json"
    path.write_text(text)
    with pytest.raises(sfft.SfftError) as ei:
        sfft.sfft_tuning_load(path)
    assert ei.value.status == sfft.SFFT_EINVAL and "tuning cache" in str(ei.value)
    with pytest.raises(sfft.SfftError):
        sfft.sfft_tuning_load(tmp_path / "missing.json")
