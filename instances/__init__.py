"""Seeded synthetic input instances for robust sample sort.

This module only draws inputs; it holds none of the sorting method's
arithmetic.  Both sides of every parity check (the CPU oracle and the CUDA
library) consume the same arrays produced here.

All random numbers come from the splitmix64 counter generator (Steele, Lea &
Flood 2014): output c of the stream with state s is
``mix(s + (c + 1) * 0x9e3779b97f4a7c15)``.  Each instance uses its own stream
state ``splitmix64(seed, instance_id)``.

The instance names follow the Helman et al. inputs that the paper runs
(Section 6 and Appendix "Experimental Results"); where the paper's wording is
incomplete the readings below are used:

* partition ``i`` of ``p`` holds positions ``[floor(i*n/p), floor((i+1)*n/p))``
  (element ``e`` is in partition ``floor(e*p/n)``);
* "slice ``s``" of the key range is ``[s*w, (s+1)*w)`` with
  ``w = floor((2**64 - 1) / p)``.
"""
from __future__ import annotations

import math

import numpy as np

U64 = np.uint64
_GAMMA = U64(0x9E3779B97F4A7C15)
_M1 = U64(0xBF58476D1CE4E5B9)
_M2 = U64(0x94D049BB133111EB)
_MASK = (1 << 64) - 1
_CHUNK = 1 << 22

NAMES = ("uniform", "gaussian", "reverse", "bucket_sorted", "staggered", "g_group",
         "mirrored", "all_to_one", "zero", "rand_dupl", "deter_dupl")
_IDS = {name: i + 1 for i, name in enumerate(NAMES)}
_IDS["segmented_f64"] = 101


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> U64(30))) * _M1
        z = (z ^ (z >> U64(27))) * _M2
    return z ^ (z >> U64(31))


def splitmix64(state: int, counters: np.ndarray) -> np.ndarray:
    """Vectorised splitmix64: output ``counters[i]`` of the stream at ``state``."""
    c = np.asarray(counters, dtype=U64)
    with np.errstate(over="ignore"):
        z = U64(state & _MASK) + (c + U64(1)) * _GAMMA
    return _mix(z)


def splitmix64_scalar(state: int, counter: int) -> int:
    z = (state + (counter + 1) * 0x9E3779B97F4A7C15) & _MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def _stream(seed: int, name: str) -> int:
    return splitmix64_scalar(seed & _MASK, _IDS[name])


def _rand(state: int, lo: int, hi: int) -> np.ndarray:
    return splitmix64(state, np.arange(lo, hi, dtype=U64))


def _slice_width(p: int) -> int:
    return _MASK // p


def _partition_of(e: np.ndarray, n: int, p: int) -> np.ndarray:
    # floor(e * p / n) without overflow for n < 2**32 and p < 2**31
    return (e.astype(U64) * U64(p)) // U64(n)


def _partition_start(i: np.ndarray, n: int, p: int) -> np.ndarray:
    # first position e with floor(e*p/n) == i is ceil(i*n/p)
    i = i.astype(U64)
    return (i * U64(n) + U64(p - 1)) // U64(p)


def _fill(n: int, fn) -> np.ndarray:
    out = np.empty(n, dtype=U64)
    for lo in range(0, n, _CHUNK):
        hi = min(n, lo + _CHUNK)
        out[lo:hi] = fn(lo, hi)
    return out


def generate(name: str, n: int, p: int = 1024, seed: int = 1, g: int = 32) -> np.ndarray:
    """Keys (uint64) of instance ``name`` with ``n`` elements over ``p`` partitions."""
    if name not in _IDS:
        raise ValueError(f"unknown instance {name!r}; known: {NAMES}")
    if n < 0 or n > 0xFFFFFFFF:
        raise ValueError("n must be in [0, 2**32 - 1]")
    if n == 0:
        return np.empty(0, dtype=U64)
    st = _stream(seed, name)
    w = _slice_width(p)

    if name == "uniform":
        return _fill(n, lambda lo, hi: _rand(st, lo, hi))

    if name == "gaussian":
        # round(2**63 + 2**60 * z), z ~ N(0, 1) by Box-Muller, clamped to [0, 2**64 - 1]
        def gauss(lo, hi):
            r1 = splitmix64(st, 2 * np.arange(lo, hi, dtype=U64))
            r2 = splitmix64(st, 2 * np.arange(lo, hi, dtype=U64) + U64(1))
            u1 = ((r1 >> U64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
            u2 = (r2 >> U64(11)).astype(np.float64) * 2.0 ** -53
            z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)
            v = np.rint(2.0 ** 63 + 2.0 ** 60 * z)
            out = np.empty(hi - lo, dtype=U64)
            big = v >= 2.0 ** 64
            neg = v <= 0.0
            mid = ~(big | neg)
            out[mid] = v[mid].astype(U64)
            out[big] = U64(_MASK)
            out[neg] = U64(0)
            return out
        return _fill(n, gauss)

    if name == "reverse":
        # strictly descending: slot n-1-i of width floor((2**64-1)/n), random inside
        ws = _MASK // n

        def rev(lo, hi):
            e = np.arange(lo, hi, dtype=U64)
            r = _rand(st, lo, hi) % U64(ws)
            with np.errstate(over="ignore"):
                return (U64(n - 1) - e) * U64(ws) + r
        return _fill(n, rev)

    if name in ("bucket_sorted", "staggered", "all_to_one"):
        def sliced(lo, hi):
            e = np.arange(lo, hi, dtype=U64)
            part = _partition_of(e, n, p)
            if name == "bucket_sorted":
                sl = part
            elif name == "staggered":
                half = U64(p // 2)
                sl = np.where(part < half, U64(2) * part + U64(1), U64(2) * (part - half))
            else:
                sl = np.zeros_like(part)
            with np.errstate(over="ignore"):
                return sl * U64(w) + _rand(st, lo, hi) % U64(w)
        return _fill(n, sliced)

    if name == "g_group":
        def grouped(lo, hi):
            e = np.arange(lo, hi, dtype=U64)
            part = _partition_of(e, n, p)
            local = e - _partition_start(part, n, p)
            grp = part // U64(g)
            sl = (grp * U64(g) + U64(p // 2) + local % U64(g)) % U64(p)
            with np.errstate(over="ignore"):
                return sl * U64(w) + _rand(st, lo, hi) % U64(w)
        return _fill(n, grouped)

    if name == "mirrored":
        # first ceil(n/2) uniform, a[n-1-j] = a[j]
        out = np.empty(n, dtype=U64)
        first = n - n // 2
        out[:first] = _fill(first, lambda lo, hi: _rand(st, lo, hi))
        if n // 2:
            out[first:] = out[: n // 2][::-1]
        return out

    if name == "zero":
        return np.zeros(n, dtype=U64)

    if name == "rand_dupl":
        # runs of length uniform in [1, 4096], each run one value uniform in {0..15}
        lengths = []
        values = []
        total = 0
        r = 0
        while total < n:
            batch = max(16, (n - total) // 2048 + 16)
            rl = splitmix64(st, 2 * np.arange(r, r + batch, dtype=U64))
            rv = splitmix64(st, 2 * np.arange(r, r + batch, dtype=U64) + U64(1))
            lengths.append((rl % U64(4096) + U64(1)).astype(np.int64))
            values.append(rv % U64(16))
            total += int(lengths[-1].sum())
            r += batch
        return np.repeat(np.concatenate(values), np.concatenate(lengths))[:n].astype(U64)

    if name == "deter_dupl":
        def dd(lo, hi):
            v = _partition_of(np.arange(lo, hi, dtype=U64), n, p) + U64(1)
            lg = np.zeros(hi - lo, dtype=U64)
            for b in range(1, 64):
                lg += (v >> U64(b)) > 0
            return lg
        return _fill(n, dd)

    raise AssertionError(name)


def segmented_f64(num_segments: int, max_log2: int, seed: int = 1, dup_frac: float = 0.1,
                  total_cap: int | None = None):
    """Batched segmented instance: float64 N(0, 1) keys (as raw uint64 bits).

    Segment sizes are floor(exp(U * ln(2**max_log2))) with U uniform in [0, 1),
    i.e. log-uniform in [1, 2**max_log2).  Roughly ``dup_frac`` of the positions
    of every segment are overwritten by a copy of another key of the same
    segment (exact duplicates).  ``total_cap`` stops drawing segments once the
    total would pass it.  Returns ``(keys_bits, offsets)``.
    """
    st = _stream(seed, "segmented_f64")
    ru = splitmix64(st, np.arange(num_segments, dtype=U64))
    u = (ru >> U64(11)).astype(np.float64) * 2.0 ** -53
    sizes = np.floor(np.exp(u * (max_log2 * math.log(2.0)))).astype(np.int64)
    sizes = np.clip(sizes, 1, (1 << max_log2))
    if total_cap is not None:
        cum = np.cumsum(sizes)
        sizes = sizes[cum <= total_cap]
    offsets = np.zeros(sizes.shape[0] + 1, dtype=U64)
    offsets[1:] = np.cumsum(sizes).astype(U64)
    n = int(offsets[-1])
    base = U64(num_segments) * U64(4)
    keys = np.empty(n, dtype=np.float64)
    for lo in range(0, n, _CHUNK):
        hi = min(n, lo + _CHUNK)
        e = np.arange(lo, hi, dtype=U64)
        r1 = splitmix64(st, base + U64(4) * e)
        r2 = splitmix64(st, base + U64(4) * e + U64(1))
        u1 = ((r1 >> U64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
        u2 = (r2 >> U64(11)).astype(np.float64) * 2.0 ** -53
        keys[lo:hi] = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)
    if dup_frac > 0 and n:
        seg_of = np.repeat(np.arange(sizes.shape[0]), sizes)
        starts = offsets[:-1].astype(np.int64)
        e = np.arange(n, dtype=U64)
        rsel = splitmix64(st, base + U64(4) * e + U64(2))
        rsrc = splitmix64(st, base + U64(4) * e + U64(3))
        pick = (rsel >> U64(11)).astype(np.float64) * 2.0 ** -53 < dup_frac
        src = starts[seg_of] + (rsrc % sizes[seg_of].astype(U64)).astype(np.int64)
        idx = np.nonzero(pick)[0]
        keys[idx] = keys[src[idx]]
    return keys.view(U64), offsets


# ---------------------------------------------------------------------------
# The same instances drawn with torch on any device (the GPU for full-size
# inputs).  Integer instances give the same bytes as generate(); the Gaussian
# one may differ in the last bits where the device's log / sqrt / cos round
# differently from numpy's.  Keys are returned as int64 tensors holding the
# uint64 bit patterns.  uint64 arithmetic is done on int64: additions and
# products wrap modulo 2**64 alike, right shifts are masked to be logical,
# and remainders are corrected for patterns above 2**63.
# ---------------------------------------------------------------------------

def _s64(v: int) -> int:
    v &= _MASK
    return v - (1 << 64) if v >= (1 << 63) else v


def _t_shr(x, s: int):
    import torch
    return torch.bitwise_and(torch.bitwise_right_shift(x, s), (1 << (64 - s)) - 1)


def t_splitmix64(state: int, counters):
    """splitmix64 outputs for an int64 tensor of counters (wrapping uint64)."""
    z = counters + 1
    z = z * _s64(0x9E3779B97F4A7C15) + _s64(state)
    z = torch_xor(z, _t_shr(z, 30)) * _s64(0xBF58476D1CE4E5B9)
    z = torch_xor(z, _t_shr(z, 27)) * _s64(0x94D049BB133111EB)
    return torch_xor(z, _t_shr(z, 31))


def torch_xor(a, b):
    import torch
    return torch.bitwise_xor(a, b)


def _t_umod(r, m: int):
    """r (int64 holding uint64 patterns) modulo m, 0 < m < 2**64."""
    import torch
    if not 0 < m <= _MASK:
        raise ValueError("modulus out of range")
    if m >= (1 << 63):
        # r < 2**64 < 2m: subtract m once when r >= m (unsigned compare by
        # flipping the sign bits)
        ms = _s64(m)
        sign = _s64(1 << 63)
        below = torch.bitwise_xor(r, sign) < (ms ^ sign)
        return torch.where(below, r, r - ms)
    a = torch.remainder(r, m)                 # r mod m for r read as signed
    c = (1 << 64) % m                         # patterns below zero are r + 2**64
    neg = r < 0
    up = torch.where(a >= m - c, a - (m - c), a + c)
    return torch.where(neg, up, a)


def _t_partition_of(e, n: int, p: int):
    return (e * p) // n


def generate_torch(name: str, n: int, p: int = 1024, seed: int = 1, g: int = 32,
                   device="cpu"):
    """Keys of instance ``name`` as an int64 tensor on ``device`` (bit patterns
    of the uint64 keys that generate() returns)."""
    import torch
    if name not in _IDS:
        raise ValueError(f"unknown instance {name!r}; known: {NAMES}")
    if n < 0 or n > 0xFFFFFFFF:
        raise ValueError("n must be in [0, 2**32 - 1]")
    dev = torch.device(device)
    if n == 0:
        return torch.empty(0, dtype=torch.int64, device=dev)
    st = _stream(seed, name)
    w = _slice_width(p)
    e = torch.arange(n, dtype=torch.int64, device=dev)

    if name == "uniform":
        return t_splitmix64(st, e)

    if name == "gaussian":
        r1 = t_splitmix64(st, 2 * e)
        r2 = t_splitmix64(st, 2 * e + 1)
        u1 = (_t_shr(r1, 11).to(torch.float64) + 1.0) * 2.0 ** -53
        u2 = _t_shr(r2, 11).to(torch.float64) * 2.0 ** -53
        del r1, r2
        z = torch.sqrt(-2.0 * torch.log(u1)) * torch.cos(2.0 * math.pi * u2)
        v = torch.round(2.0 ** 63 + 2.0 ** 60 * z)
        hi = v >= 2.0 ** 63
        # values at or above 2**63: subtract it (exact) and set the top bit
        lo_part = torch.where(hi, v - 2.0 ** 63, v).clamp(min=0.0)
        lo_part = torch.where(lo_part >= 2.0 ** 63, torch.full_like(lo_part, 2.0 ** 63 - 1024),
                              lo_part)
        out = lo_part.to(torch.int64)
        out = torch.where(hi, torch.bitwise_xor(out, _s64(1 << 63)), out)
        out = torch.where(v >= 2.0 ** 64, torch.full_like(out, -1), out)
        out = torch.where(v <= 0.0, torch.zeros_like(out), out)
        return out

    if name == "reverse":
        ws = _MASK // n
        return (n - 1 - e) * _s64(ws) + _t_umod(t_splitmix64(st, e), ws)

    if name in ("bucket_sorted", "staggered", "all_to_one", "g_group"):
        part = _t_partition_of(e, n, p)
        if name == "bucket_sorted":
            sl = part
        elif name == "staggered":
            half = p // 2
            sl = torch.where(part < half, 2 * part + 1, 2 * (part - half))
        elif name == "all_to_one":
            sl = torch.zeros_like(part)
        else:
            local = e - (part * n + (p - 1)) // p
            sl = torch.remainder((part // g) * g + p // 2 + torch.remainder(local, g), p)
        return sl * _s64(w) + _t_umod(t_splitmix64(st, e), w)

    if name == "mirrored":
        first = n - n // 2
        out = torch.empty(n, dtype=torch.int64, device=dev)
        out[:first] = t_splitmix64(st, e[:first])
        if n // 2:
            out[first:] = torch.flip(out[: n // 2], dims=(0,))
        return out

    if name == "zero":
        return torch.zeros(n, dtype=torch.int64, device=dev)

    if name == "rand_dupl":
        lengths, values = [], []
        total = 0
        r = 0
        while total < n:
            batch = max(16, (n - total) // 2048 + 16)
            c = torch.arange(r, r + batch, dtype=torch.int64, device=dev)
            rl = t_splitmix64(st, 2 * c)
            rv = t_splitmix64(st, 2 * c + 1)
            lengths.append(torch.bitwise_and(rl, 4095) + 1)
            values.append(torch.bitwise_and(rv, 15))
            total += int(lengths[-1].sum().item())
            r += batch
        return torch.repeat_interleave(torch.cat(values), torch.cat(lengths))[:n].contiguous()

    if name == "deter_dupl":
        # floor(log2(partition + 1)), one value per partition
        table = torch.tensor([(i + 1).bit_length() - 1 for i in range(p)], dtype=torch.int64,
                             device=dev)
        return table[_t_partition_of(e, n, p)]

    raise AssertionError(name)


def _t_umod_t(r, m):
    """r (int64 holding uint64 patterns) modulo the int64 tensor m (0 < m < 2**62)."""
    import torch
    a = torch.remainder(r, m)
    c63 = torch.remainder(torch.remainder(torch.full_like(m, (1 << 63) - 1), m) + 1, m)
    c64 = torch.remainder(2 * c63, m)           # 2**64 mod m
    return torch.where(r < 0, torch.remainder(a + c64, m), a)


def segmented_f64_torch(num_segments: int, max_log2: int, seed: int = 1, dup_frac: float = 0.1,
                        total_cap: int | None = None, device="cpu"):
    """segmented_f64 drawn with torch on ``device``: the same segment sizes and
    duplicate choices, keys equal to the numpy ones up to the last bits of the
    device's log / sqrt / cos.  Returns (keys as float64 tensor, int64
    offsets tensor)."""
    import torch
    st = _stream(seed, "segmented_f64")
    ru = splitmix64(st, np.arange(num_segments, dtype=U64))
    u = (ru >> U64(11)).astype(np.float64) * 2.0 ** -53
    sizes = np.floor(np.exp(u * (max_log2 * math.log(2.0)))).astype(np.int64)
    sizes = np.clip(sizes, 1, (1 << max_log2))
    if total_cap is not None:
        cum = np.cumsum(sizes)
        sizes = sizes[cum <= total_cap]
    offsets = np.zeros(sizes.shape[0] + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    n = int(offsets[-1])
    dev = torch.device(device)
    base = num_segments * 4
    keys = torch.empty(n, dtype=torch.float64, device=dev)
    chunk = 1 << 24
    for lo in range(0, n, chunk):
        hi = min(n, lo + chunk)
        e = torch.arange(lo, hi, dtype=torch.int64, device=dev)
        r1 = t_splitmix64(st, base + 4 * e)
        r2 = t_splitmix64(st, base + 4 * e + 1)
        u1 = (_t_shr(r1, 11).to(torch.float64) + 1.0) * 2.0 ** -53
        u2 = _t_shr(r2, 11).to(torch.float64) * 2.0 ** -53
        keys[lo:hi] = torch.sqrt(-2.0 * torch.log(u1)) * torch.cos(2.0 * math.pi * u2)
    offs = torch.from_numpy(offsets).to(dev)
    if dup_frac > 0 and n:
        sz = torch.from_numpy(sizes).to(dev)
        picked, sources = [], []
        for lo in range(0, n, chunk):
            hi = min(n, lo + chunk)
            e = torch.arange(lo, hi, dtype=torch.int64, device=dev)
            seg = torch.searchsorted(offs, e, right=True) - 1
            rsel = t_splitmix64(st, base + 4 * e + 2)
            rsrc = t_splitmix64(st, base + 4 * e + 3)
            pick = _t_shr(rsel, 11).to(torch.float64) * 2.0 ** -53 < dup_frac
            src = offs[seg] + _t_umod_t(rsrc, sz[seg])
            picked.append(e[pick])
            sources.append(src[pick])
        idx, src = torch.cat(picked), torch.cat(sources)
        keys[idx] = keys[src]
    return keys, offs
