"""Named workloads: sizes and parameters of the paper-shaped synthetic runs.

Each workload is a signal shape (N, K, SNR) plus the flat-window plan that
processes it (B buckets, window width w, L loops, c*K selected buckets,
vote threshold T).  The shapes follow the paper's experiments (general sparse
case at SNR 20 dB, exactly sparse case without noise); the plan sizes are
this library's.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def default_window(N: int, B: int) -> int:
    """Window width w = B (log2 N + 21): 512 at the worked example's N=2048, B=16."""
    return B * (N.bit_length() - 1 + 21)


@dataclass(frozen=True)
class Workload:
    name: str
    N: int
    K: int
    B: int
    L: int
    snr_db: float | None
    c: int = 2
    T: int | None = None
    w: int | None = None

    @property
    def window(self) -> int:
        return self.w if self.w is not None else default_window(self.N, self.B)

    @property
    def threshold(self) -> int:
        return self.T if self.T is not None else (self.L + 1) // 2


# exactly sparse single signal: N=2^16, K=10, B=64, L=8 (w = 2368)
EXACT_N16 = Workload("exact_N2^16_K10_B64_L8", 1 << 16, 10, 64, 8, None)
# general sparse single signal: N=2^20, K=100, SNR 20 dB, B=512, L=12 (w = 20992)
GENERAL_N20 = Workload("general_N2^20_K100_snr20_B512_L12", 1 << 20, 100, 512, 12, 20.0)
# precision sweep shape: N=2^24, K=1000, B=4096, L=12 (w = 184320)
SWEEP_N24 = Workload("sweep_N2^24_K1000_B4096_L12", 1 << 24, 1000, 4096, 12, 20.0)


def max_K(N: int) -> int:
    """Largest K the flat window serves at length N: 2K kept buckets need
    B >= 2K, and the window needs N/B >= 64, so K <= N/128 (and <= 8192)."""
    return max(1, min(8192, N // 128))


def batched_mix(n_signals: int = 4096, seed: int = 0):
    """The batched workload: (N, K, snr_db, signal seed) per signal, N = 2^n
    with n uniform on {14..22}, K uniform on [10, 1000] (at most N/128),
    SNR uniform on [0, 40] dB; signal seeds 0..n_signals-1."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_signals):
        N = 1 << int(rng.integers(14, 23))
        K = int(rng.integers(10, 1001))
        out.append((N, min(K, max_K(N)), float(rng.uniform(0.0, 40.0)), i))
    return out


def serving_stream(rate: float = 2000.0, seconds: float = 60.0, seed: int = 0):
    """The serving workload: Poisson arrivals at `rate` per second for
    `seconds`; per request (arrival s, N, K, snr_db) with N = 2^n, n uniform
    on {12..26}, K log-uniform on the powers of two 1..4096 (at most N/128),
    SNR uniform on [-10, 40] dB."""
    rng = np.random.default_rng(seed)
    n_req = int(rng.poisson(rate * seconds))
    t = np.sort(rng.uniform(0.0, seconds, n_req))
    out = []
    for i in range(n_req):
        N = 1 << int(rng.integers(12, 27))
        K = 1 << int(rng.integers(0, 13))
        out.append((float(t[i]), N, min(K, 1 << (max_K(N).bit_length() - 1)), float(rng.uniform(-10.0, 40.0))))
    return out

