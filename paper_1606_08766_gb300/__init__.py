"""Robust multi-level sample sort on one GB300 (sm_103a).

A from-scratch GPU implementation of the robust sample-sort partition step of
Axtmann & Sanders, "Robust Massively Parallel Sorting" (arXiv 1606.08766), and
of the sorts built on it.  All work runs in the CUDA kernels of ``librsort.so``
behind the C ABI declared in ``include/rsort.h``; this package only marshals
arguments (PyTorch supplies device memory and streams).
"""
from .binding import (ALGO_NAMES, KEY_F64, KEY_U64, Context, RsortError, Stats,
                      library_path, load_library, partition_noalloc)

__all__ = ["Context", "RsortError", "Stats", "KEY_U64", "KEY_F64", "ALGO_NAMES",
           "load_library", "library_path", "partition_noalloc"]
