"""GB300-native flat-window voting sparse FFT (sFFT1.0-style hot path).

The compute path is the CUDA library built from ``csrc/`` (C ABI declared in
``include/sfft.h``); ``sfft`` is its thin ctypes binding.  ``signals`` and
``configs`` describe seeded synthetic workloads.
"""
