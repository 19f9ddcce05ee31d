"""Measuring autotuner of the plan sizes (B, w, L) per size class.

The paper tunes its parameters "to balance time efficiency and robustness"
(Experimental Setup) and gives no values.  This tuner measures them on the
device it runs on.  For every size class (N = 2^n, a band of K, a band of SNR)
it synthesises a set of signals of that class (the platform's recipe,
signals.make_signal_device), and for every candidate (B/K ratio, window
width, L) it times sfft_execute_batch_timed over them and computes their L1
error and support recall against the exact spectra (metrics.errors_sparse).
The fixed rule of sfft_suggest_params (B = 4K, w = B (log2 N + 21), L = 12)
is the reference: the class takes the fastest candidate whose L1 error is at
most the rule's (plus 2 %) and whose recall is at least the rule's (minus
0.002), i.e. spectra/s at a fixed L1 error.  The result is a JSON cache that
the library reads with sfft_tuning_load (sfft_suggest_params then uses it).

    python -m paper_2012_08238_gb300.tune --out paper_2012_08238_gb300/tuning/gb300.json
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

from . import configs, metrics, sfft, signals

# candidates: (B_per_K, w_extra, L); the rule is (4, 21, 12)
RULE = (4, 21, 12)
CANDIDATES = [(r, 21, L) for r in (4, 8, 16, 32) for L in (8, 12, 16)]
K_BANDS = [(1, 4), (5, 32), (33, 128), (129, 512), (513, 4096)]
SNR_BANDS = [(-10.0, 10.0), (10.0, 25.0), (25.0, None)]  # None: no upper bound
L1_SLACK, RECALL_SLACK = 1.02, 0.002


def plan_sizes(N: int, K: int, cand) -> tuple[int, int, int] | None:
    """(B, w, L) of a candidate within the size rule's bounds, or None."""
    r, wex, L = cand
    b = 64
    while b < r * K:
        b <<= 1
    b = max(2, min(b, 16384, N // 64))
    if b < 2 * K:
        return None
    w = b * (N.bit_length() - 1 + wex)
    if w > N:
        w = N // b * b
    return b, w, L


class ClassSet:
    """The signals of one size class on the device, with what their error figures need."""

    def __init__(self, torch, dev, n: int, kb, sb, count: int, seed: int):
        N = 1 << n
        rng = np.random.default_rng(seed)
        kmax = min(kb[1], configs.max_K(N))
        hi = 40.0 if sb[1] is None else sb[1]
        self.N, self.items = N, []
        for i in range(count):
            K = int(rng.integers(kb[0], kmax + 1))
            snr = float(rng.uniform(sb[0], hi))
            sd = seed * 1000 + i
            x, _, _, xhat = signals.make_signal_device(N, K, sd, snr, dev, with_xhat=True)
            supp = torch.sort(torch.topk(xhat.abs(), K).indices).values
            self.items.append((K, snr, sd, x, xhat, supp.cpu().numpy(), xhat[supp].cpu().numpy()))


def measure(torch, dev, stream, cs: ClassSet, cand, steps: int):
    """(spectra/s, mean L1 error, support recall) of one candidate on a class's signals."""
    plans, xs, idxs, vals = [], [], [], []
    for K, snr, sd, x, xhat, supp, xs_supp in cs.items:
        sz = plan_sizes(cs.N, K, cand)
        if sz is None:
            return None
        B, w, L = sz
        plans.append(sfft.sfft_plan_create(cs.N, K, B, w, L, sd))
        xs.append(x)
        idxs.append(torch.zeros(K, dtype=torch.int32, device=dev))
        vals.append(torch.zeros(K, dtype=torch.complex64, device=dev))
    kout = torch.zeros(len(plans), dtype=torch.int32, device=dev)
    for _ in range(2):
        sfft.sfft_execute_batch(plans, xs, idxs, vals, kout, stream)
    torch.cuda.synchronize(dev)
    total_ms, _ = sfft.sfft_execute_batch_timed(plans, xs, idxs, vals, kout, steps, stream)
    k = kout.cpu().numpy()
    l1, miss, kk = [], 0, 0
    for i, (K, snr, sd, x, xhat, supp, xs_supp) in enumerate(cs.items):
        idx = idxs[i][: k[i]].to(torch.int64)
        e = metrics.errors_sparse(K, supp, xs_supp, idx.cpu().numpy(), vals[i][: k[i]].cpu().numpy(),
                                  xhat[idx].cpu().numpy())
        l1.append(e["L1"])
        miss += e["L0"]
        kk += K
    del plans
    return len(cs.items) * steps / (total_ms / 1e3), float(np.mean(l1)), 1.0 - miss / kk


def choose(results: dict):
    """The fastest candidate at the rule's accuracy (the rule itself if none is)."""
    base = results.get(RULE)
    if base is None:
        return None
    best = RULE
    for cand, (rate, l1, rec) in results.items():
        if l1 <= base[1] * L1_SLACK + 1e-9 and rec >= base[2] - RECALL_SLACK and rate > results[best][0]:
            best = cand
    return best


def tune(logNs, out_path: str, steps: int = 3, log=print, signals_max: int = 256):
    import torch

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    classes = []
    if os.path.exists(out_path):  # merge: classes of other logN stay
        with open(out_path) as fh:
            classes = [c for c in json.load(fh)["classes"] if c["logN"] not in logNs]
    t0 = time.perf_counter()
    for n in logNs:
        N = 1 << n
        for kb in K_BANDS:
            if kb[0] > configs.max_K(N):
                continue
            for sb in SNR_BANDS:
                # enough signals for a throughput-bound batch (2^27 samples), 4..signals_max
                count = int(min(signals_max, max(4, (1 << 27) // N)))
                cs = ClassSet(torch, dev, n, kb, sb, count, seed=7919 * n + 131 * kb[0] + int(sb[0] + 20))
                results = {}
                for cand in CANDIDATES:
                    r = measure(torch, dev, stream, cs, cand, steps)
                    if r is not None:
                        results[cand] = r
                best = choose(results)
                del cs
                torch.cuda.empty_cache()
                if best is None:
                    continue
                rate, l1, rec = results[best]
                base = results[RULE]
                classes.append({"logN": n, "K_lo": kb[0], "K_hi": kb[1], "snr_lo": sb[0], "snr_hi": sb[1],
                                "B_per_K": best[0], "w_extra": best[1], "L": best[2],
                                "spectra_per_s": rate, "l1_error": l1, "support_recall": rec,
                                "rule_spectra_per_s": base[0], "rule_l1_error": base[1],
                                "rule_support_recall": base[2], "signals": count})
                log(f"2^{n} K {kb} SNR {sb}: {best} {rate:.0f}/s (rule {base[0]:.0f}/s) "
                    f"L1 {l1:.4f} (rule {base[1]:.4f}) recall {rec:.4f} [{time.perf_counter() - t0:.0f} s]")
    classes.sort(key=lambda c: (c["logN"], c["K_lo"], c["snr_lo"]))
    doc = {"version": 1, "device": torch.cuda.get_device_name(dev),
           "what": "per size class the fastest (B_per_K, w_extra, L) whose L1 error and support recall match the "
                   "fixed rule's (4, 21, 12); measured by paper_2012_08238_gb300/tune.py",
           "l1_slack": L1_SLACK, "recall_slack": RECALL_SLACK, "classes": classes}
    os.makedirs(os.path.dirname(os.path.abspath(out_path)), exist_ok=True)
    with open(out_path, "w") as fh:
        json.dump(doc, fh, indent=1)
    return doc


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning", "gb300.json"))
    ap.add_argument("--logN", default="12-26", help="range of log2 N to tune, e.g. 14-22")
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--signals-max", type=int, default=256,
                    help="most signals per class (fewer: a class measured nearer its share of a mixed batch)")
    a = ap.parse_args(argv)
    lo, hi = (int(v) for v in a.logN.split("-"))
    tune(list(range(lo, hi + 1)), a.out, a.steps, log=lambda m: print(m, flush=True), signals_max=a.signals_max)


if __name__ == "__main__":
    main(sys.argv[1:])
