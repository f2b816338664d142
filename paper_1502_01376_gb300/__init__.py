"""GB300 (sm_103a) hybrid Yee-FFT Maxwell field advance (arXiv:1502.01376).

The work runs in libhyb.so (hand-written CUDA, C ABI in include/hyb.h);
``hyb`` is a thin ctypes binding with the same names.  ``workloads`` holds the
seeded synthetic inputs.
"""
from . import workloads  # noqa: F401

__all__ = ["hyb", "workloads"]
