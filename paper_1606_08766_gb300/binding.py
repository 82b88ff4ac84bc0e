"""ctypes binding of librsort (the C ABI in include/rsort.h).

Argument marshalling only: tensors are passed as raw device pointers with the
current PyTorch CUDA stream; every step of the sort runs in librsort's kernels.
There is no CPU fallback: if the library is missing or cannot load, calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

from . import build as _build

KEY_U64 = 0
KEY_F64 = 1

# rsort_stats.algo_elems: elements finished by each in-SM algorithm
ALGO_NAMES = ("rank", "bins", "bitonic", "quicksort", "merge", "in_order")

_STATUS = {0: "ok", 1: "pending", -1: "invalid argument", -2: "out of memory",
           -3: "CUDA error", -4: "timed out", -5: "cancelled", -6: "unsupported",
           -7: "device-side error"}

_lib = None


class RsortError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {_STATUS.get(status, status)} (status {status})")
        self.status = status


class _Stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("p", ctypes.c_uint32), ("levels", ctypes.c_uint32),
                ("path", ctypes.c_uint32), ("max_bucket", ctypes.c_uint32),
                ("max_over_mean", ctypes.c_double), ("final_buckets", ctypes.c_uint64),
                ("bytes_moved", ctypes.c_uint64), ("level_elems", ctypes.c_uint64 * 4),
                ("class_elems", ctypes.c_uint64 * 5), ("algo_elems", ctypes.c_uint64 * 6)]


class _PartOpts(ctypes.Structure):
    _fields_ = [("tie_break", ctypes.c_uint32), ("overpartition", ctypes.c_uint32)]


class _Request(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("d_keys_in", ctypes.c_void_p),
                ("d_keys_out", ctypes.c_void_p), ("d_perm_out", ctypes.c_void_p),
                ("n", ctypes.c_uint64), ("p_virtual", ctypes.c_uint32), ("seed", ctypes.c_uint64)]


class _ServeStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("cancelled", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("queued", ctypes.c_uint64), ("inflight_batches", ctypes.c_uint32),
                ("batches", ctypes.c_uint64), ("keys_completed", ctypes.c_uint64),
                ("mean_batch_requests", ctypes.c_double), ("p50_us", ctypes.c_double),
                ("p99_us", ctypes.c_double), ("max_us", ctypes.c_double),
                ("elapsed_s", ctypes.c_double)]


@dataclass
class Stats:
    n: int
    p: int
    levels: int
    path: int
    max_bucket: int
    max_over_mean: float
    final_buckets: int
    bytes_moved: int
    level_elems: list
    class_elems: list
    algo_elems: list


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Loads librsort.so (building it first if it is absent and nvcc exists)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path) or not _build.up_to_date():
        if not build_if_missing:
            raise RuntimeError(f"librsort is not built ({path}); run __graft_entry__.build()")
        _build.build()
    lib = ctypes.CDLL(path)
    vp, u64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32
    sig = {
        "rsort_create": (i32, [ctypes.POINTER(vp), ctypes.c_int, u64, ctypes.c_char_p]),
        "rsort_destroy": (i32, [vp]),
        "rsort_strerror": (ctypes.c_char_p, [i32]),
        "rsort_check": (i32, [vp]),
        "rsort_partition": (i32, [vp, i32, vp, u64, u32, u64, vp, vp, vp, vp]),
        "rsort_partition_ex": (i32, [vp, i32, vp, u64, u32, u64, ctypes.POINTER(_PartOpts),
                                     vp, vp, vp, vp, vp, vp]),
        "rsort_approx_median": (i32, [vp, i32, vp, u64, u32, u64, vp, vp]),
        "rsort_sort": (i32, [vp, i32, vp, vp, vp, u64, u32, u64, vp, ctypes.POINTER(_Stats)]),
        "rsort_segmented": (i32, [vp, i32, vp, vp, vp, u64, vp, u32, u64, vp]),
        "rsort_partition_noalloc": (i32, [i32, vp, u64, u32, u64, vp, vp, vp, vp]),
        "rsort_set_profiling": (i32, [vp, ctypes.c_int]),
        "rsort_phase_times": (i32, [vp, ctypes.POINTER(ctypes.c_char_p),
                                    ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_uint64), ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_int)]),
        "rsort_launch_count": (i32, [vp, ctypes.POINTER(u64)]),
        "rsort_set_tunable": (i32, [vp, ctypes.c_char_p, ctypes.c_int64]),
        "rsort_submit": (i32, [vp, ctypes.POINTER(_Request), ctypes.POINTER(u64)]),
        "rsort_poll": (i32, [vp, u64, ctypes.POINTER(u64)]),
        "rsort_wait": (i32, [vp, u64, u64]),
        "rsort_cancel": (i32, [vp, u64]),
        "rsort_get_serve_stats": (i32, [vp, ctypes.POINTER(_ServeStats)]),
        "rsort_reset_serve_stats": (i32, [vp]),
        "rsort_get_tunable": (i32, [vp, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int64)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int, what: str):
    if status != 0:
        raise RsortError(status, what)


def _ptr(t: torch.Tensor | None):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream_handle(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _key_type(t: torch.Tensor, key_type):
    if key_type is not None:
        return key_type
    return KEY_F64 if t.dtype == torch.float64 else KEY_U64


def _check_keys(t: torch.Tensor):
    if not t.is_cuda:
        raise ValueError("keys must be a CUDA tensor")
    if t.element_size() != 8 or not t.is_contiguous() or t.dim() != 1:
        raise ValueError("keys must be a contiguous 1-D tensor of 8-byte elements")


def partition_noalloc(keys: torch.Tensor, k: int, seed: int, keys_out: torch.Tensor,
                      pos_out: torch.Tensor, offsets_out: torch.Tensor, key_type=None, stream=None):
    """Allocation-free partition step on the current device.

    For callers that cannot allocate device memory when they partition; the
    outputs must be supplied (keys_out like keys, pos_out int32[n],
    offsets_out int64[k + 1]) and the scratch is librsort's fixed static
    array.  Calls that overlap on the GPU race on that array."""
    lib = load_library()
    _check_keys(keys)
    n = keys.numel()
    dev = torch.cuda.current_device()
    for name, t in (("keys", keys), ("keys_out", keys_out), ("pos_out", pos_out),
                    ("offsets_out", offsets_out)):
        if not t.is_cuda or t.device.index != dev:
            raise ValueError(f"{name} must be on the current CUDA device (cuda:{dev})")
        if t.dim() != 1 or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous 1-D tensor")
    if keys_out.dtype != keys.dtype:
        raise ValueError("keys_out must have the dtype of keys")
    if pos_out.dtype != torch.int32:
        raise ValueError("pos_out must be int32 (it holds uint32 positions)")
    if offsets_out.dtype != torch.int64:
        raise ValueError("offsets_out must be int64")
    if keys_out.numel() != n or pos_out.numel() != n or offsets_out.numel() != k + 1:
        raise ValueError("output sizes do not match n and k")
    rc = lib.rsort_partition_noalloc(_key_type(keys, key_type), _ptr(keys), n, k,
                                     seed & (2**64 - 1), _ptr(keys_out), _ptr(pos_out),
                                     _ptr(offsets_out), _stream_handle(stream))
    _check(rc, "rsort_partition_noalloc")


class Context:
    """Owns one rsort_ctx (scratch pool + plan state) on one CUDA device."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, tune_table: str | None = None):
        self._lib = load_library()
        self._ctx = ctypes.c_void_p()
        self.device = device
        tt = tune_table.encode() if tune_table else None
        _check(self._lib.rsort_create(ctypes.byref(self._ctx), device, hbm_budget_bytes, tt),
               "rsort_create")

    def close(self):
        if self._ctx:
            self._lib.rsort_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- calls ------------------------------------------------------------
    def sort(self, keys: torch.Tensor, p: int = 1, seed: int = 1, keys_out=None, perm_out=None,
             key_type=None, stream=None, stats: bool = False):
        """Sorted keys (same dtype/bits as ``keys``) and the stable permutation
        (int32 tensor holding uint32 values)."""
        _check_keys(keys)
        n = keys.numel()
        if keys_out is None:
            keys_out = torch.empty_like(keys)
        if perm_out is None:
            perm_out = torch.empty(n, dtype=torch.int32, device=keys.device)
        st = _Stats()
        rc = self._lib.rsort_sort(self._ctx, _key_type(keys, key_type), _ptr(keys), _ptr(keys_out),
                                  _ptr(perm_out), n, p, seed & (2**64 - 1),
                                  _stream_handle(stream), ctypes.byref(st) if stats else None)
        _check(rc, "rsort_sort")
        if stats:
            return keys_out, perm_out, Stats(st.n, st.p, st.levels, st.path, st.max_bucket,
                                             st.max_over_mean, st.final_buckets, st.bytes_moved,
                                             list(st.level_elems), list(st.class_elems),
                                             list(st.algo_elems))
        return keys_out, perm_out

    def sort_raw(self, key_type: int, d_in: int, d_out: int, d_perm: int, n: int, p: int,
                 seed: int, stream_handle: int):
        """Pointer-level call (no tensors): used by timing loops."""
        _check(self._lib.rsort_sort(self._ctx, key_type, ctypes.c_void_p(d_in),
                                    ctypes.c_void_p(d_out), ctypes.c_void_p(d_perm), n, p,
                                    seed & (2**64 - 1), ctypes.c_void_p(stream_handle), None),
               "rsort_sort")

    def segmented(self, keys: torch.Tensor, offsets: torch.Tensor, seed: int = 1, keys_out=None,
                  perm_out=None, key_type=None, stream=None):
        """Sorts every segment [offsets[s], offsets[s+1]) on its own; the
        permutation holds segment-local positions."""
        _check_keys(keys)
        if not offsets.is_cuda or offsets.element_size() != 8 or not offsets.is_contiguous():
            raise ValueError("offsets must be a contiguous CUDA tensor of 8-byte integers")
        n = keys.numel()
        if keys_out is None:
            keys_out = torch.empty_like(keys)
        if perm_out is None:
            perm_out = torch.empty(n, dtype=torch.int32, device=keys.device)
        nseg = max(offsets.numel() - 1, 0)
        rc = self._lib.rsort_segmented(self._ctx, _key_type(keys, key_type), _ptr(keys),
                                       _ptr(keys_out), _ptr(perm_out), n, _ptr(offsets), nseg,
                                       seed & (2**64 - 1), _stream_handle(stream))
        _check(rc, "rsort_segmented")
        return keys_out, perm_out

    def partition(self, keys: torch.Tensor, k: int, seed: int = 1, key_type=None, stream=None):
        """One robust partition step: (keys_out, positions, offsets[k+1])."""
        _check_keys(keys)
        n = keys.numel()
        keys_out = torch.empty_like(keys)
        pos_out = torch.empty(n, dtype=torch.int32, device=keys.device)
        offsets = torch.empty(k + 1, dtype=torch.int64, device=keys.device)
        rc = self._lib.rsort_partition(self._ctx, _key_type(keys, key_type), _ptr(keys), n, k,
                                       seed & (2**64 - 1), _ptr(keys_out), _ptr(pos_out),
                                       _ptr(offsets), _stream_handle(stream))
        _check(rc, "rsort_partition")
        return keys_out, pos_out, offsets

    def partition_ex(self, keys: torch.Tensor, k: int, seed: int = 1, tie_break: bool = True,
                     overpartition: int = 1, key_type=None, stream=None):
        """Partition step with the NTB switch and AMS overpartitioning:
        (keys_out, positions, offsets[k+1], fine_sizes[b*k], group_first[k+1])."""
        _check_keys(keys)
        n = keys.numel()
        dev = keys.device
        keys_out = torch.empty_like(keys)
        pos_out = torch.empty(n, dtype=torch.int32, device=dev)
        offsets = torch.empty(k + 1, dtype=torch.int64, device=dev)
        fine = torch.empty(max(k * overpartition, 1), dtype=torch.int64, device=dev)
        first = torch.empty(k + 1, dtype=torch.int32, device=dev)
        opts = _PartOpts(1 if tie_break else 0, overpartition)
        rc = self._lib.rsort_partition_ex(self._ctx, _key_type(keys, key_type), _ptr(keys), n, k,
                                          seed & (2**64 - 1), ctypes.byref(opts), _ptr(keys_out),
                                          _ptr(pos_out), _ptr(offsets), _ptr(fine), _ptr(first),
                                          _stream_handle(stream))
        _check(rc, "rsort_partition_ex")
        return keys_out, pos_out, offsets, fine[:k * overpartition], first

    def approx_median(self, keys: torch.Tensor, k: int = 16, seed: int = 1, key_type=None,
                      stream=None) -> torch.Tensor:
        """Binary-tree median approximation: a device int64 tensor holding the
        position of the chosen element."""
        _check_keys(keys)
        out = torch.empty(1, dtype=torch.int64, device=keys.device)
        rc = self._lib.rsort_approx_median(self._ctx, _key_type(keys, key_type), _ptr(keys),
                                           keys.numel(), k, seed & (2**64 - 1), _ptr(out),
                                           _stream_handle(stream))
        _check(rc, "rsort_approx_median")
        return out

    def check(self):
        _check(self._lib.rsort_check(self._ctx), "rsort_check")

    def set_profiling(self, on: bool):
        _check(self._lib.rsort_set_profiling(self._ctx, 1 if on else 0), "rsort_set_profiling")

    def phase_times(self):
        """{kernel name: (milliseconds, launches)} accumulated since the last read."""
        cap = 64
        names = (ctypes.c_char_p * cap)()
        ms = (ctypes.c_double * cap)()
        cnt = (ctypes.c_uint64 * cap)()
        count = ctypes.c_int()
        _check(self._lib.rsort_phase_times(self._ctx, names, ms, cnt, cap, ctypes.byref(count)),
               "rsort_phase_times")
        return {names[i].decode(): (ms[i], int(cnt[i])) for i in range(min(cap, count.value))}

    def set_tunable(self, name: str, value: int):
        _check(self._lib.rsort_set_tunable(self._ctx, name.encode(), value), "rsort_set_tunable")

    def get_tunable(self, name: str) -> int:
        v = ctypes.c_int64()
        _check(self._lib.rsort_get_tunable(self._ctx, name.encode(), ctypes.byref(v)),
               "rsort_get_tunable")
        return v.value

    # -- serving ----------------------------------------------------------
    def submit(self, keys: torch.Tensor, keys_out: torch.Tensor, perm_out: torch.Tensor,
               p: int = 0, seed: int = 1, key_type=None) -> int:
        """Queues a sort request; the tensors must stay alive and untouched
        until the ticket reports a final status."""
        _check_keys(keys)
        req = _Request(_key_type(keys, key_type), keys.data_ptr(), keys_out.data_ptr(),
                       perm_out.data_ptr(), keys.numel(), p, seed & (2**64 - 1))
        t = ctypes.c_uint64()
        _check(self._lib.rsort_submit(self._ctx, ctypes.byref(req), ctypes.byref(t)),
               "rsort_submit")
        return t.value

    def poll(self, ticket: int):
        """(status, latency_ns); status 1 = pending, 0 = done."""
        lat = ctypes.c_uint64(0)
        st = self._lib.rsort_poll(self._ctx, ticket, ctypes.byref(lat))
        return st, lat.value

    def wait(self, ticket: int, timeout_s: float = 60.0) -> int:
        return self._lib.rsort_wait(self._ctx, ticket, int(timeout_s * 1e9))

    def cancel(self, ticket: int) -> int:
        return self._lib.rsort_cancel(self._ctx, ticket)

    def serve_stats(self) -> dict:
        s = _ServeStats()
        _check(self._lib.rsort_get_serve_stats(self._ctx, ctypes.byref(s)), "rsort_get_serve_stats")
        return {name: getattr(s, name) for name, _ in _ServeStats._fields_}

    def reset_serve_stats(self):
        _check(self._lib.rsort_reset_serve_stats(self._ctx), "rsort_reset_serve_stats")

    def launch_count(self) -> int:
        v = ctypes.c_uint64()
        _check(self._lib.rsort_launch_count(self._ctx, ctypes.byref(v)), "rsort_launch_count")
        return v.value
