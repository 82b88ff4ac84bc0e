"""CPU oracle for robust sample sort -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference leg
of ``bench.py`` may import this package.  The product library never loads it,
and it shares no code with the CUDA path (see ``oracle.c`` for what each
function computes and which passage of Axtmann & Sanders, "Robust Massively
Parallel Sorting" (arXiv 1606.08766) it follows).

The C source is compiled with the host ``gcc`` into ``oracle/_build/`` on first
use (or by ``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

KEY_U64 = 0
KEY_F64 = 1


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (plain -O2, portable flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", _SRC, "-o", tmp],
                   check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64p = ctypes.POINTER(ctypes.c_uint64)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            lib.oracle_sort.argtypes = [u64p, ctypes.c_uint64, ctypes.c_int, u64p, u32p]
            lib.oracle_sort.restype = ctypes.c_int
            lib.oracle_sort_parallel.argtypes = [u64p, ctypes.c_uint64, ctypes.c_int,
                                                 ctypes.c_int, u64p, u32p]
            lib.oracle_sort_parallel.restype = ctypes.c_int
            lib.oracle_segmented.argtypes = [u64p, u64p, ctypes.c_uint32, ctypes.c_int,
                                             u64p, u32p]
            lib.oracle_segmented.restype = ctypes.c_int
            lib.oracle_splitmix64_at.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.oracle_splitmix64_at.restype = ctypes.c_uint64
            lib.oracle_sample_count.argtypes = [ctypes.c_uint64, ctypes.c_uint32]
            lib.oracle_sample_count.restype = ctypes.c_uint64
            lib.oracle_partition.argtypes = [u64p, ctypes.c_uint64, ctypes.c_int,
                                             ctypes.c_uint32, ctypes.c_uint64, u64p, u64p,
                                             u32p, u32p, u64p, u32p, u64p]
            lib.oracle_partition.restype = ctypes.c_int
            lib.oracle_partition_ex.argtypes = [u64p, ctypes.c_uint64, ctypes.c_int,
                                                ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int,
                                                ctypes.c_uint32, u64p, u32p, u64p, u32p, u64p]
            lib.oracle_partition_ex.restype = ctypes.c_int
            lib.oracle_tree_median.argtypes = [u64p, ctypes.c_uint64, ctypes.c_int,
                                               ctypes.c_uint32, ctypes.c_uint64]
            lib.oracle_tree_median.restype = ctypes.c_int64
            _lib = lib
    return _lib


def _p64(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)) if a is not None else None


def _p32(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)) if a is not None else None


def _as_bits(keys) -> np.ndarray:
    a = np.ascontiguousarray(keys)
    if a.dtype == np.float64:
        a = a.view(np.uint64)
    if a.dtype != np.uint64:
        raise TypeError(f"keys must be uint64 or float64, got {a.dtype}")
    return a


def sort(keys, key_type: int = KEY_U64):
    """Sorted keys (raw bits, uint64) and the stable permutation (uint32)."""
    k = _as_bits(keys)
    n = k.shape[0]
    ko = np.empty(n, np.uint64)
    po = np.empty(n, np.uint32)
    rc = _load().oracle_sort(_p64(k), n, key_type, _p64(ko), _p32(po))
    if rc:
        raise ValueError("oracle_sort rejected its arguments")
    return ko, po


def sort_parallel(keys, key_type: int = KEY_U64, threads: int | None = None):
    """sort() on `threads` host threads (default: every core): equal chunks
    merge-sorted at once, then pairwise merges."""
    k = _as_bits(keys)
    n = k.shape[0]
    t = threads or os.cpu_count() or 1
    ko = np.empty(n, np.uint64)
    po = np.empty(n, np.uint32)
    rc = _load().oracle_sort_parallel(_p64(k), n, key_type, int(t), _p64(ko), _p32(po))
    if rc:
        raise ValueError("oracle_sort_parallel rejected its arguments")
    return ko, po


def segmented(keys, offsets, key_type: int = KEY_U64):
    """Per-segment sort; offsets has num_segments + 1 entries."""
    k = _as_bits(keys)
    off = np.ascontiguousarray(offsets, dtype=np.uint64)
    ko = np.empty(k.shape[0], np.uint64)
    po = np.empty(k.shape[0], np.uint32)
    rc = _load().oracle_segmented(_p64(k), _p64(off), off.shape[0] - 1, key_type,
                                  _p64(ko), _p32(po))
    if rc:
        raise ValueError("oracle_segmented rejected its arguments")
    return ko, po


def splitmix64_at(state: int, counter: int) -> int:
    return int(_load().oracle_splitmix64_at(state & (2**64 - 1), counter & (2**64 - 1)))


def sample_count(n: int, k: int) -> int:
    return int(_load().oracle_sample_count(n, k))


def partition(keys, k: int, seed: int, key_type: int = KEY_U64):
    """One level of the robust sample-sort partition step.

    Returns a dict with sample_pos, spl_key (phi-mapped), spl_pos, bucket,
    keys_out (raw bits), pos_out and offsets."""
    kb = _as_bits(keys)
    n = kb.shape[0]
    S = sample_count(n, k)
    out = {
        "sample_pos": np.empty(max(S, 1), np.uint64),
        "spl_key": np.empty(max(k - 1, 1), np.uint64),
        "spl_pos": np.empty(max(k - 1, 1), np.uint32),
        "bucket": np.empty(max(n, 1), np.uint32),
        "keys_out": np.empty(max(n, 1), np.uint64),
        "pos_out": np.empty(max(n, 1), np.uint32),
        "offsets": np.empty(k + 1, np.uint64),
    }
    rc = _load().oracle_partition(_p64(kb), n, key_type, k, seed & (2**64 - 1),
                                  _p64(out["sample_pos"]), _p64(out["spl_key"]),
                                  _p32(out["spl_pos"]), _p32(out["bucket"]),
                                  _p64(out["keys_out"]), _p32(out["pos_out"]),
                                  _p64(out["offsets"]))
    if rc:
        raise ValueError("oracle_partition rejected its arguments")
    out["sample_pos"] = out["sample_pos"][:S]
    out["spl_key"] = out["spl_key"][:max(k - 1, 0)]
    out["spl_pos"] = out["spl_pos"][:max(k - 1, 0)]
    for name in ("bucket", "keys_out", "pos_out"):
        out[name] = out[name][:n]
    return out


def partition_ex(keys, k: int, seed: int, key_type: int = KEY_U64, tie_break: bool = True,
                 over: int = 1):
    """The partition step with the NTB switch (tie_break=False: classify by key
    only) and AMS overpartitioning (over = b > 1: b*k fine partitions grouped
    greedily into k outputs).

    Returns a dict with fine_sizes [b*k], group_first [k+1], keys_out, pos_out
    and offsets [k+1]."""
    kb = _as_bits(keys)
    n = kb.shape[0]
    K = k * over
    out = {
        "fine_sizes": np.empty(max(K, 1), np.uint64),
        "group_first": np.empty(k + 1, np.uint32),
        "keys_out": np.empty(max(n, 1), np.uint64),
        "pos_out": np.empty(max(n, 1), np.uint32),
        "offsets": np.empty(k + 1, np.uint64),
    }
    rc = _load().oracle_partition_ex(_p64(kb), n, key_type, k, seed & (2**64 - 1),
                                     1 if tie_break else 0, over, _p64(out["fine_sizes"]),
                                     _p32(out["group_first"]), _p64(out["keys_out"]),
                                     _p32(out["pos_out"]), _p64(out["offsets"]))
    if rc:
        raise ValueError("oracle_partition_ex rejected its arguments")
    out["fine_sizes"] = out["fine_sizes"][:K]
    for name in ("keys_out", "pos_out"):
        out[name] = out[name][:n]
    return out


def tree_median(keys, k: int, seed: int, key_type: int = KEY_U64) -> int:
    """Binary-tree median approximation: the position of the chosen element."""
    kb = _as_bits(keys)
    r = _load().oracle_tree_median(_p64(kb), kb.shape[0], key_type, k, seed & (2**64 - 1))
    if r < 0:
        raise ValueError("oracle_tree_median rejected its arguments")
    return int(r)
