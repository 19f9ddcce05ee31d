"""Throughput benchmark of the flat-window voting sparse FFT on GB300.

One step = the whole hot path (gather-window-fold, B-point FFT, top-cK select,
vote, estimate, top-K) over one batch of seeded synthetic signals of the
general-sparse workload (N = 2^20 complex64, K = 100 frequencies of magnitude
1, SNR 20 dB; B = 512 buckets, L = 12 loops, w = 20992, c*K = 200 kept
buckets, vote threshold T = 6).  Inputs are resident in HBM when the timed
region starts; the batch's inputs (signals_per_step x 8 MiB) exceed the 129 MB
L2, and so do the sectors one step touches, so no L2 flush is needed.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
instead, on the host cores, over a bounded sample of the same workload.
Multi-GPU (torchrun): every rank runs its own shard of signals (replicas, no
collective in the data path); the elapsed time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2012_08238_gb300 import configs, replicas, signals  # noqa: E402

METRIC = "spectra/s batched+served vs plain at fixed L1 error; p50/p99 ms; HBM GB/s"

# kernels of one batched step: gather, FFT/select, vote scan, estimate (whose
# last CTA per job takes the top K) and the fallback pass (whose CTAs return
# at once unless a job's pruned records could not certify its top K)
LAUNCHES_PER_STEP = 5

# DRAM bytes per spectrum of the gather kernel (dram__bytes_read.sum +
# dram__bytes_write.sum of one ncu capture of the 64-signal launch, divided by
# 64); the capture's summary is under profiles/.  None when the kernel changed
# after the capture.
NCU_GATHER_TRAFFIC_PER_SPECTRUM = (531_569_408 + 22_112_512) / 64
UNIT = "spectra/s"

# plan options of the variants a --profile run may take (the headline is
# "voting"); strings name the binding's constants
PROFILE_VARIANTS = {
    "voting": {},
    "comb": {"method": "SFFT_METHOD_COMB", "comb": 4096},
    "median_refine": {"refine": 2},
    "mean_refine": {"estimator": "SFFT_ESTIMATOR_MEAN", "refine": 2},
    "search": {"method": "SFFT_METHOD_SEARCH", "L": 8},
    "split_bf16": {"precision": 1},
    "stream": {"mode": "SFFT_GATHER_STREAM"},
}
WORKLOAD = configs.GENERAL_N20


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), float(p.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------ CPU oracle
_ORACLE_STATE = {}


def _oracle_init(W):
    import oracle

    g = oracle.window_taps(W.N, W.B, W.window)
    _ORACLE_STATE.update(W=W, g=g, Gt=oracle.filter_gain(W.N, W.B, W.window, g))


def _oracle_run(seed):
    """One signal through the oracle as it stands (plan tables precomputed);
    returns (worker pid, compute seconds, k_out)."""
    import oracle

    W = _ORACLE_STATE["W"]
    plan = oracle.Plan.__new__(oracle.Plan)
    plan.N, plan.K, plan.B, plan.w, plan.L, plan.seed = W.N, W.K, W.B, W.window, W.L, seed
    plan.c, plan.T = W.c, W.threshold
    plan.estimator, plan.refine = oracle.MEDIAN, 0  # the bench line's estimator, no refinement
    plan.g, plan.Gt = _ORACLE_STATE["g"], _ORACLE_STATE["Gt"]
    plan.sigma, plan.tau, plan.sigma_inv = oracle.loop_params(W.N, W.L, seed)
    x = signals.make_signal(W.N, W.K, seed, W.snr_db, keep_xhat=False).x
    t0 = time.perf_counter()
    out = oracle.sfft(plan, x)
    return os.getpid(), time.perf_counter() - t0, out["k_out"]


def _oracle_signal_job(job):
    """The oracle on one signal it synthesises itself (N, K, B, w, L, plan seed,
    signal seed, SNR): returns (idx, val, seconds)."""
    import oracle

    N, K, B, w, L, pseed, sseed, snr = job
    x = signals.make_signal(N, K, sseed, snr, keep_xhat=False).x
    t0 = time.perf_counter()
    out = oracle.sfft(oracle.Plan(N, K, B, w, L, pseed), x)
    return out["idx"], out["val"], time.perf_counter() - t0


def oracle_pool(cores: int):
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    return ctx.Pool(cores, initializer=_oracle_init, initargs=(WORKLOAD,))


def time_oracle(pool, seeds):
    """Seconds the oracle needs for `seeds` on the pool's workers running in
    parallel: the largest per-worker sum of compute time (signal synthesis
    and inter-process transfer excluded); and the median seconds of one
    signal on one core."""
    per, each = {}, []
    for pid, dt, _ in pool.map(_oracle_run, seeds, chunksize=1):
        per[pid] = per.get(pid, 0.0) + dt
        each.append(dt)
    return max(per.values()), float(np.median(each))


def _slices(torch, dev, Ks):
    """One int32 and one complex64 device buffer holding every job's K outputs."""
    off = np.concatenate([[0], np.cumsum(Ks)]).astype(np.int64)
    idx_all = torch.zeros(int(off[-1]), dtype=torch.int32, device=dev)
    val_all = torch.zeros(int(off[-1]), dtype=torch.complex64, device=dev)
    return ([idx_all[off[i]:off[i + 1]] for i in range(len(Ks))],
            [val_all[off[i]:off[i + 1]] for i in range(len(Ks))])


def _device_errors(torch, dev, N, K, seed, snr, idx, val):
    """errors_sparse of one output against its regenerated exact spectrum (on the device)."""
    from paper_2012_08238_gb300 import metrics as _m

    _, _, _, xhat = signals.make_signal_device(N, K, seed, snr, dev, with_xhat=True)
    supp = torch.sort(torch.topk(xhat.abs(), K).indices).values
    idx_t = idx.to(torch.int64)
    return _m.errors_sparse(K, supp.cpu().numpy(), xhat[supp].cpu().numpy(), idx_t.cpu().numpy(),
                            val.cpu().numpy(), xhat[idx_t].cpu().numpy())


def measure_batched_c3(sfft, torch, dev, stream, args):
    """The batched workload: 4096 signals of uneven N (2^14..2^22), K and SNR
    in one sfft_execute_batch (one launch per stage over every signal), plans
    sized by sfft_suggest_params; spectra/s timed by the library, by graph
    replay and through the plain per-signal path, with L1 error and support
    recall per size class."""
    specs = configs.batched_mix(args.c3_signals)
    plans, xs, Ks = [], [], []
    for N, K, snr, seed in specs:
        B, w, L = sfft.sfft_suggest_params(N, K, snr)
        plans.append(sfft.sfft_plan_create(N, K, B, w, L, 50_000 + seed))
        xs.append(signals.make_signal_device(N, K, 50_000 + seed, snr, dev)[0])
        Ks.append(K)
    idxs, vals = _slices(torch, dev, Ks)
    kout = torch.zeros(len(specs), dtype=torch.int32, device=dev)
    in_bytes = sum(8 * N for N, _, _, _ in specs)
    for _ in range(max(3, args.warmup)):
        sfft.sfft_execute_batch(plans, xs, idxs, vals, kout, stream)
    torch.cuda.synchronize(dev)
    steps = max(3, args.steps // 4)
    total_ms, stage_ms = sfft.sfft_execute_batch_timed(plans, xs, idxs, vals, kout, steps, stream)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        sfft.sfft_execute_batch(plans, xs, idxs, vals, kout, stream)  # cached graph
    e1.record(stream)
    torch.cuda.synchronize(dev)
    graph_ms = e0.elapsed_time(e1) / steps
    ks = torch.zeros(1, dtype=torch.int32, device=dev)
    e0.record(stream)
    for i in range(len(specs)):
        sfft.sfft_execute(plans[i], xs[i], idxs[i], vals[i], ks, stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    plain_ms = e0.elapsed_time(e1)
    sfft.sfft_execute_batch(plans, xs, idxs, vals, kout, stream)
    torch.cuda.synchronize(dev)
    k = kout.cpu().numpy()
    classes = {}
    for i, (N, K, snr, seed) in enumerate(specs):
        if i % args.c3_error_stride:
            continue
        e = _device_errors(torch, dev, N, K, 50_000 + seed, snr, idxs[i][: k[i]], vals[i][: k[i]])
        c = classes.setdefault(N.bit_length() - 1, {"signals": 0, "l1": [], "miss": 0, "K": 0})
        c["signals"] += 1
        c["l1"].append(e["L1"])
        c["miss"] += e["L0"]
        c["K"] += K
    per_class = {f"2^{n}": {"signals_checked": c["signals"], "l1_error": float(np.mean(c["l1"])),
                            "support_recall": 1.0 - c["miss"] / c["K"]} for n, c in sorted(classes.items())}
    S = len(specs)
    out = {"value": S * steps / (total_ms / 1e3), "unit": UNIT, "ms_per_step": total_ms / steps,
           "graph_value": S / (graph_ms / 1e3), "plain_value": S / (plain_ms / 1e3),
           "signals": S, "input_bytes": in_bytes,
           "l1_error": float(np.mean([x for c in classes.values() for x in c["l1"]])),
           "support_recall": 1.0 - sum(c["miss"] for c in classes.values()) / sum(c["K"] for c in classes.values()),
           "per_size_class": per_class,
           "stage_ms_per_step": {kk: v / steps for kk, v in stage_ms.items()},
           "what": "4096 signals, N = 2^n with n uniform on 14..22, K uniform on [10, 1000] (<= N/128), SNR "
                   "uniform on [0, 40] dB, one batch (one launch per stage); B, w, L per signal by "
                   "sfft_suggest_params; errors over every "
                   f"{args.c3_error_stride}th signal"}
    # the same batch with the split-BF16 tensor-core DFT where B allows it (64 <= B <= 4096)
    k32 = kout.cpu().numpy().copy()
    ref = [idxs[i][: k32[i]].cpu().numpy() for i in range(len(specs))]
    sizes = [(p.info.B, p.info.w, p.info.L) for p in plans]
    del plans
    torch.cuda.empty_cache()
    plans16, n16 = [], 0
    for (N, K, snr, seed), (B, w, L) in zip(specs, sizes):
        prec = 1 if 64 <= B <= 4096 else 0
        n16 += prec
        plans16.append(sfft.sfft_plan_create_ex(N, K, B, w, L, 50_000 + seed, precision=prec))
    for _ in range(max(3, args.warmup)):
        sfft.sfft_execute_batch(plans16, xs, idxs, vals, kout, stream)
    torch.cuda.synchronize(dev)
    t16, st16 = sfft.sfft_execute_batch_timed(plans16, xs, idxs, vals, kout, steps, stream)
    k16 = kout.cpu().numpy()
    common = sum(len(np.intersect1d(idxs[i][: k16[i]].cpu().numpy(), ref[i])) for i in range(len(specs)))
    out["split_bf16"] = {"value": S * steps / (t16 / 1e3), "unit": UNIT, "ms_per_step": t16 / steps,
                         "signals_on_tensor_cores": n16,
                         "support_agreement_with_fp32": common / max(1, int(np.sum(k32))),
                         "stage_ms_per_step": {kk: v / steps for kk, v in st16.items()},
                         "what": "the same batch with precision 1 (split-BF16 B-point DFT) for every plan with "
                                 "64 <= B <= 4096, the rest FP32"}
    del plans16, xs
    torch.cuda.empty_cache()
    return out


def _serve_stream(sfft, torch, dev, reqs, pool, slots, budget, count=None):
    """Replays the request stream (arrival s, N, K, snr) through a server with
    `slots` slots: submits each request at its arrival time, waits for all;
    returns (latencies ms, wall seconds from the first submission to the last
    completion, lag of the submitter behind the arrivals in ms, outputs)."""
    n = len(reqs) if count is None else min(count, len(reqs))
    Ks = [reqs[i][2] for i in range(n)]
    idxs, vals = _slices(torch, dev, Ks)
    srv = sfft.sfft_server_create(budget, slots)
    # one request of every shape first, so plans and tables exist (not timed)
    seen, warm = set(), []
    for i in range(n):
        t, N, K, snr = reqs[i]
        B, w, L = sfft.sfft_suggest_params(N, K, snr)
        if (N, B, K) not in seen:
            seen.add((N, B, K))
            x = pool[(N, K)][0][0]
            warm.append(sfft.sfft_submit(srv, N, K, B, w, L, 1, x, idxs[i], vals[i], count_samples=0))
    for tk in warm:
        sfft.sfft_wait(srv, tk, 600000)
    tickets, lag = [], 0.0
    t0 = time.perf_counter()
    for i in range(n):
        t, N, K, snr = reqs[i]
        while time.perf_counter() - t0 < t:
            pass
        lag = max(lag, time.perf_counter() - t0 - t)
        B, w, L = sfft.sfft_suggest_params(N, K, snr)
        sigs = pool[(N, K)]
        x = sigs[i % len(sigs)][0]
        tickets.append(sfft.sfft_submit(srv, N, K, B, w, L, 70_000 + i, x, idxs[i], vals[i], count_samples=0))
    res = [sfft.sfft_wait(srv, tk, 600000) for tk in tickets]
    wall = time.perf_counter() - t0
    srv.destroy()
    lat = np.asarray([r.latency_ns for r in res]) / 1e6
    return lat, wall, 1e3 * lag, idxs, vals, res


def measure_served_c5(sfft, torch, dev, args):
    """The serving workload: a Poisson request stream (2000 requests/s, N
    2^12..2^26, K log-uniform, SNR -10..40 dB, a distinct seed per request)
    through the continuous-batching server, and the same stream through a
    one-slot server (the plain per-signal path); p50/p99 latency and
    spectra/s of both, and the error figures of a sample of requests."""
    reqs = configs.serving_stream(args.c5_rate, args.c5_seconds)
    # a pool of device signals per (N, K): requests of one shape cycle through it
    pool = {}
    for _, N, K, _ in reqs:
        if (N, K) not in pool:
            P = max(2, min(8, (1 << 30) // (8 * N)))
            snrs = np.random.default_rng(31 * N + K).uniform(-10.0, 40.0, P)  # the stream's SNR range
            seeds = [90_000 + 97 * j + 13 * N.bit_length() + K for j in range(P)]
            pool[(N, K)] = [signals.make_signal_device(N, K, sd, float(sn), dev) + (sd, float(sn))
                            for sd, sn in zip(seeds, snrs)]
    pool_bytes = sum(8 * N * len(v) for (N, K), v in pool.items())
    budget = int(args.c5_budget_gb * (1 << 30))
    lat, wall, lag, idxs, vals, res = _serve_stream(sfft, torch, dev, reqs, pool, 64, budget)
    n = len(reqs)
    ok = sum(r.status == sfft.SFFT_OK for r in res)
    # errors of a sample (every 97th request): its output against its pooled signal's spectrum
    e1, miss, kk = [], 0, 0
    for i in range(0, n, 97):
        t, N, K, snr = reqs[i]
        sigs = pool[(N, K)]
        _, _, _, seed, s_snr = sigs[i % len(sigs)]
        k = res[i].k_out
        e = _device_errors(torch, dev, N, K, seed, s_snr, idxs[i][:k], vals[i][:k])
        e1.append(e["L1"])
        miss += e["L0"]
        kk += K
    out = {"value": ok / wall, "unit": UNIT, "requests": n, "ok": ok, "offered_per_s": args.c5_rate,
           "seconds": args.c5_seconds, "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
           "submit_lag_max_ms": lag, "pool_signals": sum(len(v) for v in pool.values()), "pool_bytes": pool_bytes,
           "mean_input_bytes": float(np.mean([8 * N for _, N, _, _ in reqs])),
           "l1_error_sample": float(np.mean(e1)), "support_recall_sample": 1.0 - miss / max(kk, 1),
           "what": "Poisson arrivals; N = 2^n, n uniform on 12..26; K log-uniform on the powers of two 1..4096 "
                   "(<= N/128); SNR uniform on [-10, 40] dB; a distinct seed per request; signals from a device "
                   "pool per (N, K); 64 slots, plans cached by shape and rebound per request"}
    del idxs, vals
    # the plain per-signal path: the same stream through a one-slot server
    lat1, wall1, lag1, idxs, vals, res1 = _serve_stream(sfft, torch, dev, reqs, pool, 1, budget,
                                                        count=args.c5_plain_requests)
    n1 = len(res1)
    out["plain"] = {"value": sum(r.status == sfft.SFFT_OK for r in res1) / wall1, "unit": UNIT, "requests": n1,
                    "p50_ms": float(np.percentile(lat1, 50)), "p99_ms": float(np.percentile(lat1, 99)),
                    "submit_lag_max_ms": lag1,
                    "what": "the first requests of the same stream, one at a time (one-slot server)"}
    del idxs, vals, pool
    torch.cuda.empty_cache()
    return out


def measure_split_bf16(sfft, torch, dev, stream, args, W, sigs, xs, idx32, val32, k32):
    """The headline's signals with the split-BF16 tensor-core DFT (precision
    1): spectra/s timed by the library, per-stage times, the error figures,
    and the agreement of its output with the FP32 path's."""
    from paper_2012_08238_gb300 import metrics as _m

    S = len(xs)
    plans = [sfft.sfft_plan_create_ex(W.N, W.K, W.B, W.window, W.L, s, precision=1) for s in range(S)]
    idxs = [torch.zeros(W.K, dtype=torch.int32, device=dev) for _ in range(S)]
    vals = [torch.zeros(W.K, dtype=torch.complex64, device=dev) for _ in range(S)]
    kout = torch.zeros(S, dtype=torch.int32, device=dev)
    for _ in range(max(3, args.warmup)):
        sfft.sfft_execute_batch(plans, xs, idxs, vals, kout, stream)
    torch.cuda.synchronize(dev)
    total_ms, stage_ms = sfft.sfft_execute_batch_timed(plans, xs, idxs, vals, kout, args.steps, stream)
    k = kout.cpu().numpy()
    errs, common, d2, n2 = [], 0, 0.0, 0.0
    for i, sg in enumerate(sigs):
        ii, vv = idxs[i].cpu().numpy()[: k[i]], vals[i].cpu().numpy()[: k[i]]
        errs.append(_m.errors(sg.xhat, W.K, ii, vv))
        c, gi, oi = np.intersect1d(ii, idx32[i][: k32[i]], return_indices=True)
        common += len(c)
        d2 += float(np.sum(np.abs(vv[gi].astype(np.complex128) - val32[i][: k32[i]][oi]) ** 2))
        n2 += float(np.sum(np.abs(val32[i][: k32[i]][oi].astype(np.complex128)) ** 2))
    st = [sfft.sfft_plan_last_stats(p).device_error for p in plans]
    del plans
    return {"value": S * args.steps / (total_ms / 1e3), "unit": UNIT, "ms_per_step": total_ms / args.steps,
            "stage_ms_per_step": {kk: v / args.steps for kk, v in stage_ms.items()},
            "l1_error": float(np.mean([e["L1"] for e in errs])),
            "support_recall": 1.0 - float(np.sum([e["L0"] for e in errs])) / (W.K * S),
            "support_agreement_with_fp32": common / max(1, int(np.sum(k32))),
            "value_rel_l2_vs_fp32": float(np.sqrt(d2 / max(n2, 1e-30))), "device_errors": int(np.count_nonzero(st)),
            "what": "same signals as the headline; the B-point DFT as a tcgen05 GEMM with hi/lo BF16 splits "
                    "(3 products, FP32 accumulation in tensor memory)"}


def _gather_modes_at(sfft, torch, dev, stream, N, K, count, snr, steps):
    """Permuted vs stream gather on `count` signals of one shape (the fixed
    size rule's B, w, L): the gather stage's device time, the whole step's
    spectra/s, and the agreement of the stream plans' supports with the
    permuted ones'."""
    B = 64
    while B < 4 * K:
        B <<= 1
    B = min(B, 4096, N // 64)
    w = min(configs.default_window(N, B), N // B * B)
    L = 12
    xs = [signals.make_signal_device(N, K, 900 + i, snr, dev)[0] for i in range(count)]
    out = {"N": N, "K": K, "B": B, "w": w, "L": L, "signals": count, "snr_db": snr}
    sup = {}
    for name, mode in (("permuted", sfft.SFFT_GATHER_PERMUTED), ("stream", sfft.SFFT_GATHER_STREAM)):
        plans = [sfft.sfft_plan_create_ex(N, K, B, w, L, 900 + i, mode=mode) for i in range(count)]
        idxs = [torch.zeros(K, dtype=torch.int32, device=dev) for _ in range(count)]
        vals = [torch.zeros(K, dtype=torch.complex64, device=dev) for _ in range(count)]
        kout = torch.zeros(count, dtype=torch.int32, device=dev)
        for _ in range(3):
            sfft.sfft_execute_batch(plans, xs, idxs, vals, kout, stream)
        torch.cuda.synchronize(dev)
        total_ms, stage_ms = sfft.sfft_execute_batch_timed(plans, xs, idxs, vals, kout, steps, stream)
        k = kout.cpu().numpy()
        sup[name] = [np.sort(idxs[i].cpu().numpy()[: k[i]]) for i in range(count)]
        out[name] = {"gather_ms": stage_ms["gather_fold"] / steps, "ms_per_step": total_ms / steps,
                     "value": count * steps / (total_ms / 1e3),
                     "gather_read_gbs": count * N * 8 / (stage_ms["gather_fold"] / steps / 1e3) / 1e9}
        del plans
    common = sum(len(np.intersect1d(a, b)) for a, b in zip(sup["permuted"], sup["stream"]))
    out["support_agreement"] = common / max(1, sum(len(a) for a in sup["permuted"]))
    out["stream_speedup_gather"] = out["permuted"]["gather_ms"] / out["stream"]["gather_ms"]
    del xs
    torch.cuda.empty_cache()
    return out


def measure_gather_modes(sfft, torch, dev, stream, args, W, xs):
    """Step a1's two readers (sfft_opts.mode): the headline's signals through
    stream-gather plans (graph-replay spectra/s and stage times, as the
    headline), and permuted vs stream at N = 2^14 .. 2^26."""
    S = len(xs)
    plans = [sfft.sfft_plan_create_ex(W.N, W.K, W.B, W.window, W.L, s, mode=sfft.SFFT_GATHER_STREAM)
             for s in range(S)]
    idxs = [torch.zeros(W.K, dtype=torch.int32, device=dev) for _ in range(S)]
    vals = [torch.zeros(W.K, dtype=torch.complex64, device=dev) for _ in range(S)]
    kout = torch.zeros(S, dtype=torch.int32, device=dev)
    for _ in range(max(3, args.warmup)):
        sfft.sfft_execute_batch(plans, xs, idxs, vals, kout, stream)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        sfft.sfft_execute_batch(plans, xs, idxs, vals, kout, stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    replay_ms = e0.elapsed_time(e1)
    total_ms, stage_ms = sfft.sfft_execute_batch_timed(plans, xs, idxs, vals, kout, args.steps, stream)
    del plans
    g_ms = stage_ms["gather_fold"] / args.steps
    head = {"value": S * args.steps / (replay_ms / 1e3), "unit": UNIT,
            "stage_timed_value": S * args.steps / (total_ms / 1e3),
            "stage_ms_per_step": {k: v / args.steps for k, v in stage_ms.items()},
            "gather_read_gbs": S * W.N * 8 / (g_ms / 1e3) / 1e9}
    shapes = [(1 << 14, 100, 256), (1 << 16, 100, 128), (1 << 18, 300, 64), (1 << 20, 100, 64),
              (1 << 22, 100, 16), (1 << 24, 1000, 4), (1 << 26, 1000, 2)]
    sweep = [_gather_modes_at(sfft, torch, dev, stream, N, K, n, 20.0, args.steps) for N, K, n in shapes]
    return {"headline_stream": head, "sweep": sweep,
            "what": "stream gather: the signal read once in order (8 N bytes, coalesced) and each loop's reads "
                    "visited by the three-gap return map; permuted: one sector per window tap"}


def measure_precision_sweep(sfft, torch, dev, stream, args, pool):
    """The precision sweep: N = 2^24, K = 1000, B = 4096, L = 12 at SNR -10,
    0, 10, 20, 40 dB, args.c4_seeds signals each, through the FP32 and the
    split-BF16 paths: L1 / L2 error and support recall against the planted
    spectra, agreement between the two paths; and, on args.c4_oracle_seeds
    signals per SNR, agreement of both with the FP64 oracle (run on the host
    cores meanwhile)."""
    W = configs.SWEEP_N24
    snrs = (-10.0, 0.0, 10.0, 20.0, 40.0)
    no = args.c4_oracle_seeds
    jobs = [(W.N, W.K, W.B, W.window, W.L, j, 30_000 + 100 * i + j, snr) for i, snr in enumerate(snrs)
            for j in range(no)]
    pending = pool.map_async(_oracle_signal_job, jobs, chunksize=1) if pool is not None and no > 0 else None
    S = args.c4_seeds
    plans = {prec: [sfft.sfft_plan_create_ex(W.N, W.K, W.B, W.window, W.L, s, precision=prec) for s in range(S)]
             for prec in (0, 1)}
    idxs = [torch.zeros(W.K, dtype=torch.int32, device=dev) for _ in range(S)]
    vals = [torch.zeros(W.K, dtype=torch.complex64, device=dev) for _ in range(S)]
    kout = torch.zeros(S, dtype=torch.int32, device=dev)
    rows = []
    for i, snr in enumerate(snrs):
        row = {"snr_db": snr}
        gen = [signals.make_signal_device(W.N, W.K, 40_000 + 100 * i + s, snr, dev, with_xhat=True) for s in range(S)]
        xs = [g[0] for g in gen]
        outs = {}
        for prec in (0, 1):
            sfft.sfft_execute_batch(plans[prec], xs, idxs, vals, kout, stream)
            torch.cuda.synchronize(dev)
            k = kout.cpu().numpy()
            outs[prec] = [(idxs[s][: k[s]].to(torch.int64), vals[s][: k[s]].clone()) for s in range(S)]
        for prec, name in ((0, "fp32"), (1, "split_bf16")):
            l1, l2, miss = [], [], 0
            for s in range(S):
                x, _, _, xhat = gen[s]
                supp = torch.sort(torch.topk(xhat.abs(), W.K).indices).values
                ii, vv = outs[prec][s]
                from paper_2012_08238_gb300 import metrics as _m

                e = _m.errors_sparse(W.K, supp.cpu().numpy(), xhat[supp].cpu().numpy(), ii.cpu().numpy(),
                                     vv.cpu().numpy(), xhat[ii].cpu().numpy())
                l1.append(e["L1"])
                l2.append(e["L2_rel"])
                miss += e["L0"]
            row[name] = {"l1_error": float(np.mean(l1)), "l2_rel_error": float(np.mean(l2)),
                         "support_recall": 1.0 - miss / (W.K * S)}
        agree, d2, n2, tot = 0, 0.0, 0.0, 0
        for s in range(S):
            a, va = outs[0][s]
            b, vb = outs[1][s]
            c, ia, ib = np.intersect1d(a.cpu().numpy(), b.cpu().numpy(), return_indices=True)
            agree += len(c)
            tot += len(a)
            va_, vb_ = va.cpu().numpy()[ia].astype(np.complex128), vb.cpu().numpy()[ib].astype(np.complex128)
            d2 += float(np.sum(np.abs(vb_ - va_) ** 2))
            n2 += float(np.sum(np.abs(va_) ** 2))
        row["support_agreement_bf16_vs_fp32"] = agree / max(tot, 1)
        row["value_rel_l2_bf16_vs_fp32"] = float(np.sqrt(d2 / max(n2, 1e-30)))
        rows.append(row)
        del gen, xs, outs
        torch.cuda.empty_cache()
    out = {"workload": f"N=2^24, K={W.K}, B={W.B}, L={W.L}, w={W.window}; {S} signals per SNR", "rows": rows}
    if pending is not None:
        res = pending.get()
        for i, snr in enumerate(snrs):
            agg = {0: [0, 0, 0.0, 0.0], 1: [0, 0, 0.0, 0.0]}
            for j in range(no):
                oidx, oval, _ = res[i * no + j]
                sig = signals.make_signal(W.N, W.K, 30_000 + 100 * i + j, snr, keep_xhat=False)
                xd = torch.from_numpy(sig.x).to(dev)
                for prec in (0, 1):
                    ii = torch.zeros(W.K, dtype=torch.int32, device=dev)
                    vv = torch.zeros(W.K, dtype=torch.complex64, device=dev)
                    ko = torch.zeros(1, dtype=torch.int32, device=dev)
                    sfft.sfft_execute(plans[prec][j], xd, ii, vv, ko, stream)
                    torch.cuda.synchronize(dev)
                    kk = int(ko.item())
                    gi_, gv_ = ii.cpu().numpy()[:kk], vv.cpu().numpy()[:kk]
                    c, a, b = np.intersect1d(gi_, oidx, return_indices=True)
                    g = agg[prec]
                    g[0] += len(c)
                    g[1] += len(oidx)
                    g[2] += float(np.sum(np.abs(gv_[a].astype(np.complex128) - oval[b]) ** 2))
                    g[3] += float(np.sum(np.abs(oval[b]) ** 2))
                del xd
            for prec, name in ((0, "fp32"), (1, "split_bf16")):
                g = agg[prec]
                rows[i][name]["support_agreement_vs_oracle"] = g[0] / max(g[1], 1)
                rows[i][name]["value_rel_l2_vs_oracle"] = float(np.sqrt(g[2] / max(g[3], 1e-30)))
        out["oracle"] = {"signals_per_snr": no, "seconds_per_signal": float(np.mean([r[2] for r in res])),
                         "what": "FP64 oracle on the host cores (its own signals of the same recipe)"}
    del plans
    torch.cuda.empty_cache()
    return out


def measure_comb(sfft, torch, dev, stream, args, W, sigs, xs, Bc=4096):
    """The bench workload's signals through voting behind the spike-train
    pre-filter (Bc residue classes, top 2K kept): spectra/s timed by the
    library, and the error figures against the planted spectra."""
    from paper_2012_08238_gb300 import metrics as _m

    S = len(xs)
    plans = [sfft.sfft_plan_create_ex(W.N, W.K, W.B, W.window, W.L, s, method=sfft.SFFT_METHOD_COMB, comb=Bc)
             for s in range(S)]
    idxs = [torch.zeros(W.K, dtype=torch.int32, device=dev) for _ in range(S)]
    vals = [torch.zeros(W.K, dtype=torch.complex64, device=dev) for _ in range(S)]
    kout = torch.zeros(S, dtype=torch.int32, device=dev)
    for _ in range(max(3, args.warmup)):
        sfft.sfft_execute_batch(plans, xs, idxs, vals, kout, stream)
    torch.cuda.synchronize(dev)
    total_ms, stage_ms = sfft.sfft_execute_batch_timed(plans, xs, idxs, vals, kout, args.steps, stream)
    k = kout.cpu().numpy()
    errs = [_m.errors(sg.xhat, W.K, idxs[i].cpu().numpy()[: k[i]], vals[i].cpu().numpy()[: k[i]])
            for i, sg in enumerate(sigs)]
    st = sfft.sfft_plan_last_stats(plans[0])
    return {"value": S * args.steps / (total_ms / 1e3), "unit": UNIT, "ms_per_step": total_ms / args.steps,
            "classes": Bc, "kept_classes": min(2 * W.K, Bc),
            "l1_error": float(np.mean([e["L1"] for e in errs])),
            "support_recall": 1.0 - float(np.sum([e["L0"] for e in errs])) / (W.K * S),
            "survivors_first_signal": int(st.estimated),
            "stage_ms_per_step": {kk: v / args.steps for kk, v in stage_ms.items()},
            "what": "same signals as the headline; voting restricted to the kept residue classes"}


def measure_mean(sfft, torch, dev, stream, args, W, sigs, xs, snrs=(0.0, 10.0, 20.0, 40.0), per_snr=8):
    """The bench workload's signals with the averaging estimator (the mean of
    the L per-loop estimates; every candidate is estimated): spectra/s timed
    by the library and the error figures, also with two refinement passes;
    then the L1 error of both estimators, plain and refined, over an SNR
    sweep (per_snr signals per SNR, context)."""
    from paper_2012_08238_gb300 import metrics as _m

    S = len(xs)

    def run(plans, xs_, K):
        idxs = [torch.zeros(K, dtype=torch.int32, device=dev) for _ in plans]
        vals = [torch.zeros(K, dtype=torch.complex64, device=dev) for _ in plans]
        kout = torch.zeros(len(plans), dtype=torch.int32, device=dev)
        return idxs, vals, kout

    plans = [sfft.sfft_plan_create_ex(W.N, W.K, W.B, W.window, W.L, s, estimator=sfft.SFFT_ESTIMATOR_MEAN)
             for s in range(S)]
    idxs, vals, kout = run(plans, xs, W.K)
    for _ in range(max(3, args.warmup)):
        sfft.sfft_execute_batch(plans, xs, idxs, vals, kout, stream)
    torch.cuda.synchronize(dev)
    total_ms, stage_ms = sfft.sfft_execute_batch_timed(plans, xs, idxs, vals, kout, args.steps, stream)
    k = kout.cpu().numpy()
    errs = [_m.errors(sg.xhat, W.K, idxs[i].cpu().numpy()[: k[i]], vals[i].cpu().numpy()[: k[i]])
            for i, sg in enumerate(sigs)]
    st = sfft.sfft_plan_last_stats(plans[0])
    out = {"value": S * args.steps / (total_ms / 1e3), "unit": UNIT, "ms_per_step": total_ms / args.steps,
           "l1_error": float(np.mean([e["L1"] for e in errs])),
           "support_recall": 1.0 - float(np.sum([e["L0"] for e in errs])) / (W.K * S),
           "estimated_first_signal": int(st.estimated),
           "stage_ms_per_step": {kk: v / args.steps for kk, v in stage_ms.items()},
           "what": "same signals as the headline; a6 by the mean of the L per-loop estimates"}
    del plans
    # both estimators with two refinement passes (the iterative framework's subtraction)
    for key, est in (("refined", sfft.SFFT_ESTIMATOR_MEAN), ("median_refined", sfft.SFFT_ESTIMATOR_MEDIAN)):
        plans = [sfft.sfft_plan_create_ex(W.N, W.K, W.B, W.window, W.L, s, estimator=est, refine=2)
                 for s in range(S)]
        for _ in range(max(3, args.warmup)):
            sfft.sfft_execute_batch(plans, xs, idxs, vals, kout, stream)
        torch.cuda.synchronize(dev)
        total_ms, stage_ms = sfft.sfft_execute_batch_timed(plans, xs, idxs, vals, kout, args.steps, stream)
        k = kout.cpu().numpy()
        errs = [_m.errors(sg.xhat, W.K, idxs[i].cpu().numpy()[: k[i]], vals[i].cpu().numpy()[: k[i]])
                for i, sg in enumerate(sigs)]
        out[key] = {"value": S * args.steps / (total_ms / 1e3), "unit": UNIT, "ms_per_step": total_ms / args.steps,
                    "estimator": "mean" if est == sfft.SFFT_ESTIMATOR_MEAN else "median", "passes": 2,
                    "l1_error": float(np.mean([e["L1"] for e in errs])),
                    "support_recall": 1.0 - float(np.sum([e["L0"] for e in errs])) / (W.K * S),
                    "refine_ms_per_step": stage_ms["refine"] / args.steps}
        del plans
    sweep = []
    for snr in snrs:
        sg = [signals.make_signal(W.N, W.K, 20_000 + s, snr) for s in range(per_snr)]
        xd = [torch.from_numpy(g.x).to(dev) for g in sg]
        row = {"snr_db": snr}
        for name, est, passes in (("median", sfft.SFFT_ESTIMATOR_MEDIAN, 0), ("mean", sfft.SFFT_ESTIMATOR_MEAN, 0),
                                  ("median_refined", sfft.SFFT_ESTIMATOR_MEDIAN, 2),
                                  ("mean_refined", sfft.SFFT_ESTIMATOR_MEAN, 2)):
            pl = [sfft.sfft_plan_create_ex(W.N, W.K, W.B, W.window, W.L, 20_000 + s, estimator=est, refine=passes)
                  for s in range(per_snr)]
            ii, vv, ko = run(pl, xd, W.K)
            sfft.sfft_execute_batch(pl, xd, ii, vv, ko, stream)
            torch.cuda.synchronize(dev)
            kk = ko.cpu().numpy()
            e = [_m.errors(g.xhat, W.K, ii[i].cpu().numpy()[: kk[i]], vv[i].cpu().numpy()[: kk[i]])
                 for i, g in enumerate(sg)]
            row[name + "_l1"] = float(np.mean([x["L1"] for x in e]))
            row[name + "_recall"] = 1.0 - float(np.sum([x["L0"] for x in e])) / (W.K * per_snr)
        sweep.append(row)
    out["snr_sweep"] = sweep
    return out


def measure_search(sfft, torch, dev, stream, args, W, sigs, xs, R=8):
    """The bench workload's (noisy) signals located by binary search in the
    iterative framework (R iterations; phase encoding finds nothing at this
    noise level): spectra/s timed by the library, the error figures, and the
    same for phase encoding (context)."""
    from paper_2012_08238_gb300 import metrics as _m

    S = len(xs)
    out = {"what": "same signals as the headline (20 dB); iterative framework, R = 8 iterations at most"}
    for name, method, sb in (("binary_search", sfft.SFFT_METHOD_SEARCH, 1),
                             ("phase_encoding", sfft.SFFT_METHOD_PHASE, 0)):
        plans = [sfft.sfft_plan_create_ex(W.N, W.K, W.B, W.window, R, s, method=method, search_bits=sb)
                 for s in range(S)]
        idxs = [torch.zeros(W.K, dtype=torch.int32, device=dev) for _ in range(S)]
        vals = [torch.zeros(W.K, dtype=torch.complex64, device=dev) for _ in range(S)]
        kout = torch.zeros(S, dtype=torch.int32, device=dev)
        for _ in range(max(3, args.warmup)):
            sfft.sfft_execute_batch(plans, xs, idxs, vals, kout, stream)
        torch.cuda.synchronize(dev)
        total_ms, _ = sfft.sfft_execute_batch_timed(plans, xs, idxs, vals, kout, args.steps, stream)
        k = kout.cpu().numpy()
        errs = [_m.errors(sg.xhat, W.K, idxs[i].cpu().numpy()[: k[i]], vals[i].cpu().numpy()[: k[i]])
                for i, sg in enumerate(sigs)]
        out[name] = {"value": S * args.steps / (total_ms / 1e3), "unit": UNIT, "ms_per_step": total_ms / args.steps,
                     "l1_error": float(np.mean([e["L1"] for e in errs])),
                     "support_recall": 1.0 - float(np.sum([e["L0"] for e in errs])) / (W.K * S),
                     "samples_per_spectrum": plans[0].info.samples_touched,
                     "iterations_first_signal": sfft.sfft_plan_last_stats(plans[0]).iterations}
        del plans
    return out


def measure_batch_sizes(sfft, torch, dev, stream, args, W, sizes=(8, 16, 32, 128, 256)):
    """The headline's signal shape at other batch sizes (context for the
    headline's 64): spectra/s through sfft_execute_batch (graph replay),
    device-generated signals of the same recipe."""
    out = []
    for S in sizes:
        plans = [sfft.sfft_plan_create(W.N, W.K, W.B, W.window, W.L, 7000 + s) for s in range(S)]
        xs = [signals.make_signal_device(W.N, W.K, 7000 + s, W.snr_db, dev)[0] for s in range(S)]
        idxs = [torch.zeros(W.K, dtype=torch.int32, device=dev) for _ in range(S)]
        vals = [torch.zeros(W.K, dtype=torch.complex64, device=dev) for _ in range(S)]
        kout = torch.zeros(S, dtype=torch.int32, device=dev)
        for _ in range(max(3, args.warmup)):
            sfft.sfft_execute_batch(plans, xs, idxs, vals, kout, stream)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            sfft.sfft_execute_batch(plans, xs, idxs, vals, kout, stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / args.steps
        out.append({"signals_per_step": S, "value": S / (ms / 1e3), "unit": UNIT, "ms_per_step": ms})
        del plans, xs
    torch.cuda.empty_cache()
    return out


def measure_exact(sfft, torch, dev, stream, args, S=256, R=8):
    """The exactly sparse workload (N = 2^16, K = 10, noiseless, B = 64) through
    sfft_execute_batch with the phase-encoding method and the binary and
    multi-scale (l = 4) search (R iterations at most), and with voting
    (L = 8): spectra/s on the device, support recall, mean iterations, and the
    phase-encoding oracle on one host core (context)."""
    from paper_2012_08238_gb300 import metrics as _m

    W = configs.EXACT_N16
    w = configs.default_window(W.N, W.B)
    sigs = [signals.make_signal(W.N, W.K, 10_000 + s) for s in range(S)]
    xs = [torch.from_numpy(sg.x).to(dev) for sg in sigs]
    out = {"workload": f"exact_N2^16_K10_B64 (noiseless), {S} signals per step, inputs "
                       f"{S * W.N * 8 / 2**20:.0f} MiB (> L2)"}
    for name, method, L, sb in (("phase_encoding", sfft.SFFT_METHOD_PHASE, R, 0),
                                ("binary_search", sfft.SFFT_METHOD_SEARCH, R, 1),
                                ("multiscale_search_l4", sfft.SFFT_METHOD_SEARCH, R, 2),
                                ("voting", sfft.SFFT_METHOD_VOTING, W.L, 0)):
        plans = [sfft.sfft_plan_create_ex(W.N, W.K, W.B, w, L, 10_000 + s, method=method, search_bits=sb)
                 for s in range(S)]
        idxs = [torch.zeros(W.K, dtype=torch.int32, device=dev) for _ in range(S)]
        vals = [torch.zeros(W.K, dtype=torch.complex64, device=dev) for _ in range(S)]
        kout = torch.zeros(S, dtype=torch.int32, device=dev)
        for _ in range(max(3, args.warmup)):
            sfft.sfft_execute_batch(plans, xs, idxs, vals, kout, stream)
        torch.cuda.synchronize(dev)
        # device time of `steps` batches enqueued by the library itself
        total_ms, _ = sfft.sfft_execute_batch_timed(plans, xs, idxs, vals, kout, args.steps, stream)
        ms = total_ms / args.steps
        # and the rate of the Python-level call (ctypes marshalling of S signals per call)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            sfft.sfft_execute_batch(plans, xs, idxs, vals, kout, stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        call_ms = e0.elapsed_time(e1) / args.steps
        k = kout.cpu().numpy()
        miss = sum(_m.errors(sg.xhat, W.K, idxs[i].cpu().numpy()[: k[i]], vals[i].cpu().numpy()[: k[i]])["L0"]
                   for i, sg in enumerate(sigs))
        entry = {"value": S / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "python_call_value": S / (call_ms / 1e3),
                 "support_recall": 1.0 - miss / (W.K * S),
                 "samples_per_spectrum": plans[0].info.samples_touched, "max_iterations": L}
        if method in (sfft.SFFT_METHOD_PHASE, sfft.SFFT_METHOD_SEARCH):
            its = [sfft.sfft_plan_last_stats(p).iterations for p in plans[:16]]
            entry["iterations_mean_first16"] = float(np.mean(its))
        out[name] = entry
        del plans
    if not args.no_cpu:
        import oracle as _oracle

        n = 4
        t0 = time.perf_counter()
        for s in range(n):
            _oracle.sfft_pe(_oracle.PlanPE(W.N, W.K, W.B, w, R, 10_000 + s), sigs[s].x)
        out["oracle_phase_cpu"] = {"value": n / (time.perf_counter() - t0), "unit": UNIT, "cores": 1,
                                   "sample": f"{n} signals, FP64 oracle incl. its plan tables, one process"}
    return out


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ------------------------------------------------------------ GPU run
def run_ours(args):
    import torch

    from paper_2012_08238_gb300 import sfft

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist_

        dist_.init_process_group("nccl")
        dist = dist_

    # the oracle pool starts before any GPU work (spawned workers)
    cores = host_cores()
    want_cpu = rank == 0 and world == 1 and not args.no_cpu and not args.profile
    pool = oracle_pool(min(cores, args.cpu_signals)) if want_cpu else None
    # measured plan sizes per size class (the batched and serving legs size their plans by them)
    tuning = None
    if args.tuning and os.path.exists(args.tuning):
        sfft.sfft_tuning_load(args.tuning)
        tuning = {"file": os.path.relpath(args.tuning, ROOT), "classes": sfft.sfft_tuning_classes()}

    W = WORKLOAD
    S = args.signals
    seeds = replicas.shard(rank, world, S)
    sigs = [signals.make_signal(W.N, W.K, s, W.snr_db) for s in seeds]
    # (profiler runs may take a variant's plans; the bench line is always the voting path)
    vopts = {k: getattr(sfft, v) if isinstance(v, str) else v for k, v in PROFILE_VARIANTS[args.variant].items()}
    L = vopts.pop("L", W.L)
    plans = [sfft.sfft_plan_create_ex(W.N, W.K, W.B, W.window, L, s, **vopts) for s in seeds]
    info = plans[0].info
    dev = torch.device("cuda", local)
    xs = [torch.from_numpy(sg.x).to(dev) for sg in sigs]
    idxs = [torch.zeros(W.K, dtype=torch.int32, device=dev) for _ in seeds]
    vals = [torch.zeros(W.K, dtype=torch.complex64, device=dev) for _ in seeds]
    kout = torch.zeros(S, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    # warm-up (also fills the graph cache for the same job list)
    for _ in range(args.warmup):
        sfft.sfft_execute_batch(plans, xs, idxs, vals, kout, stream)
    torch.cuda.synchronize(dev)

    # accuracy at this configuration (the platform's L1 error, paper_2012_08238_gb300.metrics)
    from paper_2012_08238_gb300 import metrics as _m

    errs = [_m.errors(sg.xhat, W.K, idxs[i].cpu().numpy()[: int(kout[i])], vals[i].cpu().numpy()[: int(kout[i])])
            for i, sg in enumerate(sigs)]
    l1 = float(np.mean([e["L1"] for e in errs]))
    recall = 1.0 - float(np.sum([e["L0"] for e in errs])) / (W.K * S)

    # ---- per-stage device times of K steps (CUDA events around each stage on
    # the launching stream): the stage shares and the gather's roofline
    total_ms_st, stage_ms = sfft.sfft_execute_batch_timed(plans, xs, idxs, vals, kout, args.steps, stream)
    if args.profile:
        if pool is not None:
            pool.close()
        if rank == 0:
            print(json.dumps({"profile_run": True, "value": S * args.steps / (total_ms_st / 1e3),
                              "stage_ms": stage_ms}), flush=True)
        return

    # ---- timed region: K back-to-back steps through the production call
    # (sfft_execute_batch: a seen job list replays its cached CUDA graph),
    # events on the launching stream, barrier + synchronize on both sides
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local).start() if rank == 0 else None
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    t_wall = time.perf_counter()
    e0.record(stream)
    for _ in range(args.steps):
        sfft.sfft_execute_batch(plans, xs, idxs, vals, kout, stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    t_wall = time.perf_counter() - t_wall
    if dist:
        dist.barrier()
    clk = clocks.stop() if clocks else None
    total_ms = e0.elapsed_time(e1)
    elapsed = replicas.max_over_ranks(total_ms / 1e3, dist, dev)
    value = replicas.throughput(world * S * args.steps, elapsed)

    # ---- plain per-signal path (context)
    ks = torch.zeros(1, dtype=torch.int32, device=dev)
    for i in range(S):
        sfft.sfft_execute(plans[i], xs[i], idxs[i], vals[i], ks, stream)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    reps = max(1, args.steps // 2)
    for _ in range(reps):
        for i in range(S):
            sfft.sfft_execute(plans[i], xs[i], idxs[i], vals[i], ks, stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    plain_value = S * reps / (e0.elapsed_time(e1) / 1e3)


    # ---- end to end through the host-buffer batch call (pinned host memory)
    xh = [torch.from_numpy(sg.x).pin_memory() for sg in sigs]
    ih = [torch.zeros(W.K, dtype=torch.int32).pin_memory() for _ in seeds]
    vh = [torch.zeros(W.K, dtype=torch.complex64).pin_memory() for _ in seeds]
    kh = torch.zeros(S, dtype=torch.int32).pin_memory()
    sfft.sfft_execute_batch_host(plans, xh, ih, vh, kh, stream)
    e2e_steps = max(1, args.steps // 2)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        sfft.sfft_execute_batch_host(plans, xh, ih, vh, kh, stream)
    e2e_s = time.perf_counter() - t0
    e2e_value = S * e2e_steps / e2e_s
    h2d = S * W.N * 8
    d2h = S * (W.K * 12 + 4)

    # ---- roofline of the dominant kernel (the gather: HBM-bound)
    hbm_peak, sm_max_mhz, peak_kind = _peaks()
    per_launch = {k: v / args.steps for k, v in stage_ms.items()}
    distinct = S * 8 * info.samples_touched  # algorithmic bytes: distinct samples read
    bucket_ms = per_launch["gather_fold"]
    gather_gbs = distinct / (bucket_ms / 1e3) / 1e9
    sector_bytes = S * W.L * W.window * 32
    traffic = None if NCU_GATHER_TRAFFIC_PER_SPECTRUM is None else S * NCU_GATHER_TRAFFIC_PER_SPECTRUM
    roofline = {"kernel": "k_gather", "bound": "hbm", "achieved": gather_gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": gather_gbs / hbm_peak, "traffic": traffic,
                "per_unit": f"8 B x {info.samples_touched} distinct samples per spectrum",
                "peak_source": peak_kind,
                "sector_gbs": sector_bytes / (bucket_ms / 1e3) / 1e9,
                "sector_efficiency": distinct / sector_bytes}
    if traffic is not None:
        # physical DRAM bytes of the launch over its event-timed duration
        roofline["dram_gbs"] = traffic / (bucket_ms / 1e3) / 1e9
        roofline["dram_frac"] = roofline["dram_gbs"] / hbm_peak
    # vote scan: N x L table lookups per spectrum (integer ALU work)
    roofline_scan = {"kernel": "k_scan_bits", "bound": "alu",
                     "lookups_per_s": S * W.N * W.L / (per_launch["vote_scan"] / 1e3),
                     "per_unit": f"N x L = {W.N * W.L} bucket lookups per spectrum"}

    # ---- context: a dense FFT of the same batch (cuFFT through torch.fft)
    xb = torch.stack(xs)
    torch.fft.fft(xb)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(args.steps):
        torch.fft.fft(xb)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    dense_ms = e0.elapsed_time(e1) / args.steps
    dense = {"value": S / (dense_ms / 1e3), "unit": UNIT, "ms_per_step": dense_ms,
             "what": f"dense complex64 FFT of the same {S} signals (cuFFT via torch.fft), context only"}
    del xb

    # ---- exactly sparse workload: phase encoding (iterative) vs voting (context)
    batch_sizes = measure_batch_sizes(sfft, torch, dev, stream, args, W) if rank == 0 else None
    exact = measure_exact(sfft, torch, dev, stream, args) if rank == 0 else None
    comb = measure_comb(sfft, torch, dev, stream, args, W, sigs, xs) if rank == 0 else None
    mean = measure_mean(sfft, torch, dev, stream, args, W, sigs, xs) if rank == 0 else None
    search = measure_search(sfft, torch, dev, stream, args, W, sigs, xs) if rank == 0 else None
    k32 = kout.cpu().numpy()
    idx32 = [t.cpu().numpy() for t in idxs]
    val32 = [t.cpu().numpy().astype(np.complex128) for t in vals]
    split = measure_split_bf16(sfft, torch, dev, stream, args, W, sigs, xs, idx32, val32, k32) if rank == 0 else None
    gmodes = measure_gather_modes(sfft, torch, dev, stream, args, W, xs) if rank == 0 and not args.no_modes else None
    batched = measure_batched_c3(sfft, torch, dev, stream, args) if rank == 0 and not args.no_c3 else None
    if batched is not None:
        batched["plan_sizes"] = tuning or "fixed size-class rule"
    served = measure_served_c5(sfft, torch, dev, args) if rank == 0 and not args.no_c5 else None
    if served is not None:
        served["plan_sizes"] = tuning or "fixed size-class rule"
    sweep = (measure_precision_sweep(sfft, torch, dev, stream, args, pool)
             if rank == 0 and not args.no_c4 else None)

    # ---- CPU baseline: the oracle on a bounded sample, host cores
    cpu = None
    if pool is not None:
        n = args.cpu_signals
        cs = seeds[:n]
        wall, one = time_oracle(pool, cs)
        pool.close()
        cpu = {"value": n / wall, "unit": UNIT, "cores": min(cores, n), "kind": "oracle",
               "single_thread_s_per_signal": one, "host_nproc": os.cpu_count(),
               "sample": f"{n} signals of the same workload (seeds {cs[0]}..{cs[-1]}), one per worker process, "
                         f"plan tables precomputed per worker"}
    elif pool is not None:
        pool.close()

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": W.name, "N": W.N, "K": W.K, "B": W.B, "w": W.window, "L": W.L, "c": W.c,
                   "T": W.threshold, "snr_db": W.snr_db, "signals_per_step": S, "parallelism": f"replicas{world}",
                   "l2": f"no flush: inputs {S * W.N * 8 / 2**20:.0f} MiB and touched sectors "
                         f"{sector_bytes / 2**20:.0f} MiB per step exceed the 129 MB L2"},
        "what": "value: inputs resident in HBM, K steps of sfft_execute_batch (cached CUDA graph) timed with "
                "CUDA events; stage_timed_value: the same steps with events around every stage (the stage "
                "shares and the roofline); e2e: the same metric through sfft_execute_batch_host from pinned "
                "host buffers, bound by the host link (8 MiB copied per spectrum)",
        "l1_error": l1, "support_recall": recall,
        "plain_value": plain_value, "stage_timed_value": S * args.steps / (total_ms_st / 1e3),
        "batched_c3": batched, "served_c5": served,
        "stage_ms_per_step": per_launch, "stage_share": {k: v / sum(per_launch.values()) for k, v in per_launch.items()},
        "samples_touched": info.samples_touched, "sampling_ratio": info.samples_touched / W.N,
        "roofline": roofline, "roofline_scan": roofline_scan, "dense_fft_context": dense,
        "exactly_sparse": exact, "comb_prefilter": comb, "averaging_estimator": mean, "search_location": search,
        "split_bf16_dft": split, "precision_sweep": sweep, "gather_modes": gmodes, "batch_sizes": batch_sizes,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": LAUNCHES_PER_STEP * args.steps,
        "clocks": clk,
        "wall_s_timed": t_wall,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_reference(args):
    """The oracle as it stands on the host cores, same workload and metric."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    W = WORKLOAD
    cores = host_cores()
    per_step = max(1, min(cores, args.cpu_signals))
    pool = oracle_pool(per_step)
    seed = 0
    for _ in range(args.warmup):
        time_oracle(pool, list(range(seed, seed + per_step)))
        seed += per_step
    t = 0.0
    for _ in range(args.steps):
        t += time_oracle(pool, list(range(seed, seed + per_step)))[0]
        seed += per_step
    pool.close()
    value = per_step * args.steps / t
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": W.name, "N": W.N, "K": W.K, "B": W.B, "w": W.window, "L": W.L,
                   "snr_db": W.snr_db, "signals_per_step": per_step},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": per_step, "kind": "oracle",
                         "sample": f"{per_step} signals per step, one per worker process"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--signals", type=int, default=64, help="signals per step (per GPU)")
    ap.add_argument("--cpu-signals", type=int, default=32, help="oracle sample size for cpu_baseline")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--c3-signals", type=int, default=4096, help="signals of the batched workload")
    ap.add_argument("--c3-error-stride", type=int, default=8, help="error figures of every n-th batched signal")
    ap.add_argument("--no-c3", action="store_true", help="skip the batched workload")
    ap.add_argument("--c5-rate", type=float, default=2000.0, help="serving: Poisson arrival rate (requests/s)")
    ap.add_argument("--c5-seconds", type=float, default=20.0, help="serving: length of the request stream (s)")
    ap.add_argument("--c5-budget-gb", type=float, default=96.0, help="serving: device memory budget of the plans")
    ap.add_argument("--c5-plain-requests", type=int, default=4000, help="serving: requests of the one-slot run")
    ap.add_argument("--no-c5", action="store_true", help="skip the serving workload")
    ap.add_argument("--c4-seeds", type=int, default=64, help="precision sweep: signals per SNR")
    ap.add_argument("--c4-oracle-seeds", type=int, default=2, help="precision sweep: signals per SNR checked by "
                                                                       "the oracle")
    ap.add_argument("--no-c4", action="store_true", help="skip the precision sweep")
    ap.add_argument("--no-modes", action="store_true", help="skip the permuted-vs-stream gather comparison")
    ap.add_argument("--tuning", default=os.path.join(ROOT, "paper_2012_08238_gb300", "tuning", "gb300.json"),
                    help="autotuner cache for the batched and serving legs ('' for the fixed rule)")
    ap.add_argument("--variant", default="voting", choices=sorted(PROFILE_VARIANTS),
                    help="plans of this variant (--profile runs only; the bench line is the voting path)")
    ap.add_argument("--profile", action="store_true",
                    help="profiler runs: only the warm-up and timed steps (no context runs, no CPU baseline)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.variant != "voting" and not args.profile:
        ap.error("--variant is for --profile runs; the bench line measures the voting path")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
