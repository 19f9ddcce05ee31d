"""Seeded synthetic test signals (inputs only; none of the method's arithmetic).

Both the CUDA path and the FP64 oracle consume the signals made here; this
module holds no step of the sparse-FFT method.  The recipe follows the
paper's experimental platform: K frequencies drawn uniformly without
replacement from [0, N), each with magnitude 1 and a phase uniform in
[0, 2 pi); the remaining bins are zero (exactly sparse) or complex white
Gaussian noise (general sparse) scaled to the requested SNR.

Normalisation follows Eq. 2 (1/N on the forward DFT), so the time signal is
x_j = sum_f xhat_f exp(+2 pi i j f / N) and every planted coefficient has
|xhat_f| = 1.  SNR_dB = 10 log10(sum |planted|^2 / E sum |noise|^2), so each
noise bin has variance K * 10^(-SNR/10) / N (split evenly between re and im).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

_FREQ, _PHASE, _NOISE = 1, 2, 3


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[seed & (2**64 - 1), stream]))


@dataclass
class Signal:
    x: np.ndarray        # complex64 [N], the time-domain input
    freqs: np.ndarray    # int64 [K], planted frequencies, sorted
    coefs: np.ndarray    # complex128 [K], planted coefficients (|.| = 1)
    xhat: np.ndarray     # complex128 [N], exact spectrum that x was built from
    N: int
    K: int
    snr_db: float | None


def make_signal(N: int, K: int, seed: int, snr_db: float | None = None,
                keep_xhat: bool = True) -> Signal:
    """One seeded signal of length N with K planted frequencies."""
    if N < 2 or N & (N - 1):
        raise ValueError("N must be a power of two")
    if not 1 <= K <= N:
        raise ValueError("K must lie in [1, N]")
    freqs = np.sort(_rng(seed, _FREQ).choice(N, size=K, replace=False).astype(np.int64))
    phase = _rng(seed, _PHASE).uniform(0.0, 2.0 * np.pi, size=K)
    coefs = np.exp(1j * phase)
    xhat = np.zeros(N, np.complex128)
    if snr_db is not None:
        var = K * 10.0 ** (-snr_db / 10.0) / N
        r = _rng(seed, _NOISE)
        xhat += np.sqrt(var / 2.0) * (r.standard_normal(N) + 1j * r.standard_normal(N))
    xhat[freqs] += coefs
    x = (np.fft.ifft(xhat) * N).astype(np.complex64)
    return Signal(x=x, freqs=freqs, coefs=coefs, xhat=xhat if keep_xhat else None,
                  N=N, K=K, snr_db=snr_db)


def make_signal_device(N: int, K: int, seed: int, snr_db: float | None, device, with_xhat: bool = False):
    """The same recipe generated on a CUDA device with torch, for workloads
    too large to synthesise on the host (thousands of signals, N up to 2^26).

    Frequencies and phases come from the same numpy streams as make_signal;
    the noise bins come from torch's own counter-based generator on the
    device, seeded by `seed`, so the spectrum is reproducible but its noise
    differs from make_signal's.  Returns (x, freqs, coefs[, xhat]) with x and
    xhat complex64 device tensors.
    """
    import torch

    if N < 2 or N & (N - 1):
        raise ValueError("N must be a power of two")
    if not 1 <= K <= N:
        raise ValueError("K must lie in [1, N]")
    freqs = np.sort(_rng(seed, _FREQ).choice(N, size=K, replace=False).astype(np.int64))
    coefs = np.exp(1j * _rng(seed, _PHASE).uniform(0.0, 2.0 * np.pi, size=K))
    if snr_db is not None:
        g = torch.Generator(device=device)
        g.manual_seed((seed * 2654435761 + _NOISE) & (2**63 - 1))
        var = K * 10.0 ** (-snr_db / 10.0) / N
        xhat = torch.randn(N, dtype=torch.complex64, device=device, generator=g) * float(np.sqrt(var))
    else:
        xhat = torch.zeros(N, dtype=torch.complex64, device=device)
    fi = torch.from_numpy(freqs).to(device)
    xhat[fi] += torch.from_numpy(coefs.astype(np.complex64)).to(device)
    x = torch.fft.ifft(xhat) * N
    return (x, freqs, coefs, xhat) if with_xhat else (x, freqs, coefs)

