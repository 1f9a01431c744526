"""GB300 (sm_103a) discrete Gabor transform on a nonseparable lattice.

The compute path is libdgt.so (hand-written CUDA behind the C ABI in include/dgt.h);
this package holds its sources (csrc/), the in-tree build (build.py), the ctypes
binding (_capi.py), the PyTorch-facing API (api.py) and the serving loop (serve.py).
"""
from .api import DGTFunction, LogMagLoss, Plan, Plan2, debug_status, dgt, fft_selftest, log_magnitude_loss  # noqa: F401
from ._capi import DGTError  # noqa: F401
