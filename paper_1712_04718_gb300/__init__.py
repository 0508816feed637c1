"""Spectral Ewald (SE) k-space on GB300: a C-ABI CUDA library (libse, see
include/se.h) with a thin PyTorch-facing binding.

Method: arXiv:1712.04718, Sec. 3 (spread, FFT, scale, inverse FFT, gather).
Importing this package loads nothing native; the library is loaded by the
first Plan and a missing build raises there.
"""
__version__ = "0.1.0"


def __getattr__(name):
    # lazy submodules: importing the package must not require CUDA
    if name in ("Plan",):
        from .se import Plan
        return Plan
    raise AttributeError(name)
