"""bench.py's CPU-baseline leg runs the oracle as it stands (CPU only).

The workers build the oracle's plan from precomputed tables; this runs one
signal of the bench workload through that path and checks it against the
oracle's own plan, so a plan field added to the oracle cannot leave the
baseline (and the reference arm) broken until a GPU run.
"""
import os
import sys

import oracle

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402
from paper_2012_08238_gb300 import signals  # noqa: E402


def test_oracle_worker_matches_plain_plan():
    W = bench.WORKLOAD
    bench._oracle_init(W)
    pid, dt, kout = bench._oracle_run(3)
    assert kout == W.K and dt > 0
    x = signals.make_signal(W.N, W.K, 3, W.snr_db, keep_xhat=False).x
    ref = oracle.sfft(oracle.Plan(W.N, W.K, W.B, W.window, W.L, 3, c=W.c, T=W.threshold), x)
    assert ref["k_out"] == kout
