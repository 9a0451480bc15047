"""GB300-native space-variant elliptical filtering with radially-uniform box splines.

The compute path is the CUDA library ``libbsf.so`` (C ABI in include/bsf.h),
reached through ``paper_1003_2022_gb300.api`` (torch tensors) or
``paper_1003_2022_gb300._lib`` (same names as the C ABI).
"""
from . import _lib  # noqa: F401

__all__ = ["api", "_lib", "synth", "build"]
