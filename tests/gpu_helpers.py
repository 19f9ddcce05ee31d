"""Helpers for the GPU tests: run the CUDA path through the C ABI on torch buffers."""
import numpy as np

from paper_2012_08238_gb300 import sfft

torch = None


def _torch():
    global torch
    if torch is None:
        import torch as t

        torch = t
    return torch


def dev(a, dtype=None):
    t = _torch()
    arr = np.ascontiguousarray(a)
    out = t.from_numpy(arr).cuda()
    return out if dtype is None else out.to(dtype)


def run_execute(plan, x):
    """Whole pipeline on one signal; returns (idx, val, k_out) as numpy."""
    t = _torch()
    K = plan.info.K
    xd = dev(np.asarray(x, np.complex64))
    idx = t.full((K,), -1, dtype=t.int32, device="cuda")
    val = t.zeros((K,), dtype=t.complex64, device="cuda")
    kout = t.zeros((1,), dtype=t.int32, device="cuda")
    sfft.sfft_execute(plan, xd, idx, val, kout)
    t.cuda.synchronize()
    k = int(kout.item())
    return idx.cpu().numpy()[:k], val.cpu().numpy()[:k], k


def run_bucketize(plan, x):
    t = _torch()
    info = plan.info
    xd = dev(np.asarray(x, np.complex64))
    zhat = t.zeros((info.L, info.B), dtype=t.complex64, device="cuda")
    sfft.sfft_bucketize(plan, xd, zhat)
    t.cuda.synchronize()
    return zhat.cpu().numpy()


def run_select(plan, zhat):
    t = _torch()
    info = plan.info
    zd = dev(np.asarray(zhat, np.complex64))
    sel = t.zeros((info.L, info.nsel), dtype=t.int32, device="cuda")
    sfft.sfft_select(plan, zd, sel)
    t.cuda.synchronize()
    return sel.cpu().numpy()


def run_vote(plan, sel):
    t = _torch()
    cap = plan.info.candidate_capacity
    sd = dev(np.asarray(sel, np.int32))
    cand = t.zeros((max(cap, 1),), dtype=t.int32, device="cuda")
    n = t.zeros((1,), dtype=t.int32, device="cuda")
    sfft.sfft_vote(plan, sd, cand, n, cap)
    t.cuda.synchronize()
    k = int(n.item())
    return np.sort(cand.cpu().numpy()[:k])


def run_estimate(plan, zhat, cand):
    t = _torch()
    zd = dev(np.asarray(zhat, np.complex64))
    cd = dev(np.asarray(cand, np.int32))
    est = t.zeros((max(len(cand), 1),), dtype=t.complex64, device="cuda")
    sfft.sfft_estimate(plan, zd, cd, len(cand), est)
    t.cuda.synchronize()
    return est.cpu().numpy()[: len(cand)]


def rel_l2(a, b):
    a = np.asarray(a, np.complex128)
    b = np.asarray(b, np.complex128)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))
