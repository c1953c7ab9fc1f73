"""GB300-native work-efficient SpMSpV (Azad & Buluc, arXiv 1610.07902).

The computation lives in hand-written CUDA kernels for sm_103a, compiled
into libspmspv.so and reached through the C ABI of include/spmspv.h; the
Python module ``spmspv`` is a thin ctypes binding of that ABI.
"""
from .builder import build  # noqa: F401

__all__ = ["build", "spmspv"]
