"""Autotuner of librsort's size-dependent choices.

The paper picks its sorting algorithm by input size (Section 6: a handful of
algorithms cover the whole range of n/p; Appendix "Parameter Tuning": the
number of levels and the splitter counts are tuned per size).  On one GPU the
same choice is made per segment and per bucket, and this module measures it on
the device instead of fixing it by hand:

* the scatter of a sort's deeper levels: staged, or ranked by shared-memory
  atomics in a small-footprint kernel (``atomic_scatter``);
* the in-SM sort of a bucket, per bucket-size class: the rank-by-counting
  threshold (``rank_max``), bins or bitonic for the small class
  (``sort_small``), bins, quicksort or bitonic for the mid and medium classes
  (``sort_mid``, ``sort_medium``), and the class cut-offs that pick the CTA
  shape (``small_cap``: 128 threads of 8 slots up to it, ``mid_cap``: 128
  threads of 16 slots up to it, 256 threads of 16 slots above);
* the sample-sort fan-out of a segment, per segment-size class
  c = ceil(log2 m): the bucket size it aims at (``target_bucket@c``, i.e. the
  bucket count k = ceil(m / target)).

Every candidate is timed on the device (CUDA events, median of a few runs)
through the C ABI on synthetic batches of float64 N(0, 1) keys with 10 % exact
duplicates (the batched-sort workload):

* the in-SM knobs act on every bucket of a class, most of which come out of
  the partition levels (narrow key ranges), so they are timed on two mixed
  batches -- segment sizes log-uniform in [1, 2^15] and in [1, 2^20], the
  batched configurations scaled down -- by the sum of both times;
* ``target_bucket@c`` acts only on segments of class c, so it is timed on a
  batch of such segments.

The search is coordinate descent from the defaults: a knob moves to a
candidate only if that candidate is more than ``MIN_GAIN`` faster than the
current value, so measurement noise cannot pull the table away from a plan
that is as good.  A last pass times the whole table against the defaults on
the mixed batches and keeps whichever is faster.

``write_table`` writes the "name value" tune table that ``rsort_create``
(``Context(tune_table=...)``) loads.  Tunables change speed, never results:
every choice sorts to the same bytes.
"""
from __future__ import annotations

import math
import statistics
from dataclasses import dataclass, field

import torch

from .binding import Context

# Knobs timed on the mixed batches -- the scatter of the deeper levels, then
# the in-SM sort: (name, candidates, default).  Tuned in this order, each with
# the choices made before it in place.
IN_SM_KNOBS = (
    ("atomic_scatter", (0, 1), 0),
    ("rank_max", (0, 16, 32, 64, 128), 64),
    ("sort_small", (0, 2), 0),
    ("small_cap", (256, 512, 768, 1024), 1024),
    ("sort_mid", (0, 1, 2), 0),
    ("mid_cap", (1024, 1536, 2048), 2048),
    ("sort_medium", (0, 1, 2), 0),
)
# The mixed batches the in-SM knobs are timed on: segment sizes log-uniform in
# (lo, hi] (the batched configurations' size ranges).
MIXED = ((1, 1 << 15), (1, 1 << 20))
MIN_GAIN = 0.01         # a knob moves only for a gain above 1 %
# Fan-out targets tried for segments that run the sample-sort levels.
TARGET_CANDIDATES = (768, 1024, 1280, 1536, 1792, 2048, 2560)
DEFAULT_CLASSES = tuple(range(13, 23))  # segments of 4097 .. 2^22 keys


@dataclass
class KnobResult:
    name: str
    workload: str
    ms: dict            # candidate value -> median milliseconds
    chosen: int
    default: int


@dataclass
class TuneResult:
    device: int
    knobs: list = field(default_factory=list)
    default_ms: float = 0.0     # mixed batches, defaults
    tuned_ms: float = 0.0       # mixed batches, the tuned table
    reverted: bool = False      # the table lost to the defaults and was reset

    def table(self) -> dict:
        return {k.name: k.chosen for k in self.knobs}

    def as_dict(self) -> dict:
        return {"device": self.device, "default_ms": self.default_ms,
                "tuned_ms": self.tuned_ms, "reverted": self.reverted,
                "knobs": [{"name": k.name, "workload": k.workload, "chosen": k.chosen,
                           "default": k.default,
                           "ms": {str(v): t for v, t in k.ms.items()}} for k in self.knobs]}


def segment_batch(lo: int, hi: int, total: int, seed: int, device) -> tuple:
    """A batch of segments with sizes log-uniform in (lo, hi], about `total`
    keys in all: float64 N(0, 1) keys (10 % of each segment overwritten by a
    copy of another key of the segment) and their int64 offsets, on device."""
    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    mean = (hi - lo) / max(math.log(hi / max(lo, 1)), 1e-9) if hi > lo else hi
    nseg = max(1, int(total / max(mean, 1.0)))
    u = torch.rand(nseg, generator=g, dtype=torch.float64)
    sizes = torch.floor(torch.exp(math.log(max(lo, 1)) + u * math.log(hi / max(lo, 1))))
    sizes = torch.clamp(sizes.to(torch.int64) + 1, min=max(lo, 0) + 1, max=hi)
    offs = torch.zeros(nseg + 1, dtype=torch.int64)
    offs[1:] = torch.cumsum(sizes, 0)
    n = int(offs[-1])
    keys = torch.randn(n, generator=g, dtype=torch.float64)
    seg = torch.repeat_interleave(torch.arange(nseg), sizes)
    pick = torch.rand(n, generator=g) < 0.1
    src = offs[:-1][seg] + (torch.rand(n, generator=g, dtype=torch.float64)
                            * sizes[seg].to(torch.float64)).to(torch.int64)
    keys[pick] = keys[src[pick]]
    return keys.to(device), offs.to(device)


def _time_segmented(ctx: Context, keys, offs, ko, po, reps: int) -> float:
    """Median device time (ms) of rsort_segmented on one batch."""
    stream = torch.cuda.current_stream(keys.device)
    ctx.segmented(keys, offs, keys_out=ko, perm_out=po)  # warm-up (sizes the scratch)
    ts = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.segmented(keys, offs, keys_out=ko, perm_out=po)
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    ctx.check()
    return statistics.median(ts)


def _time_batches(ctx: Context, batches, reps: int) -> float:
    """Sum over the batches of the median device time (ms)."""
    t = 0.0
    for keys, offs, ko, po in batches:
        t += _time_segmented(ctx, keys, offs, ko, po, reps)
    return t


def _batches(specs):
    out = []
    for keys, offs in specs:
        out.append((keys, offs, torch.empty_like(keys),
                    torch.empty(keys.numel(), dtype=torch.int32, device=keys.device)))
    return out


def _tune_knob(ctx: Context, name: str, candidates, batches, reps: int, default: int,
               current: int, workload: str) -> KnobResult:
    """Times every candidate; moves from `current` only for a gain above
    MIN_GAIN.  `chosen` is always the fastest candidate timed or ties it
    within that margin (the current value wins such ties)."""
    ms = {}
    for v in candidates:
        ctx.set_tunable(name, v)
        ms[v] = _time_batches(ctx, batches, reps)
    best = min(ms, key=lambda v: ms[v])
    chosen = best if (current not in ms or ms[best] < ms[current] * (1 - MIN_GAIN)) else current
    ctx.set_tunable(name, chosen)
    return KnobResult(name, workload, ms, chosen, default)


def tune(device: int = 0, classes=DEFAULT_CLASSES, keys_per_class: int = 1 << 23,
         reps: int = 3, in_sm: bool = True, seed: int = 7) -> TuneResult:
    """Times the candidates of every knob on the device and returns the
    choices (a private context is used; the defaults are its start)."""
    dev = torch.device("cuda", device)
    res = TuneResult(device)
    with torch.cuda.device(dev), Context(device) as ctx:
        mixed = _batches([segment_batch(lo, hi, keys_per_class, seed + j, dev)
                          for j, (lo, hi) in enumerate(MIXED)])
        mixed_desc = " + ".join(f"{int(b[1].numel()) - 1} float64 segments of ({lo}, {hi}] keys"
                                for b, (lo, hi) in zip(mixed, MIXED))
        default_ms = _time_batches(ctx, mixed, reps)
        if in_sm:
            for name, cands, default in IN_SM_KNOBS:
                res.knobs.append(_tune_knob(ctx, name, cands, mixed, reps, default,
                                            ctx.get_tunable(name), mixed_desc))
        for c in classes:
            lo, hi = 1 << (c - 1), 1 << c
            one = _batches([segment_batch(lo, hi, max(keys_per_class, 4 * hi),
                                          seed + 100 + c, dev)])
            name = f"target_bucket@{c}"
            res.knobs.append(_tune_knob(
                ctx, name, TARGET_CANDIDATES, one, reps, 0, ctx.get_tunable("target_bucket"),
                f"{int(one[0][1].numel()) - 1} float64 segments of ({lo}, {hi}] keys"))
            del one
        # the whole table against the defaults on the mixed batches
        tuned_ms = _time_batches(ctx, mixed, reps)
        res.default_ms, res.tuned_ms = default_ms, tuned_ms
        if tuned_ms > default_ms:
            for k in res.knobs:
                k.chosen = k.default if not k.name.startswith("target_bucket@") else 0
            res.reverted = True
        del mixed
        torch.cuda.empty_cache()
    return res


def write_table(result: TuneResult, path: str) -> str:
    """Writes the tune table ("name value" lines) that rsort_create loads."""
    with open(path, "w") as fh:
        fh.write("# librsort tune table written by paper_1606_08766_gb300.autotune\n")
        for k in result.knobs:
            fh.write(f"# {k.name}: {k.workload}; " +
                     ", ".join(f"{v}: {t:.3f} ms" for v, t in k.ms.items()) +
                     f"; chosen {k.chosen}\n")
            fh.write(f"{k.name} {k.chosen}\n")
    return path


def main():
    import argparse
    import json
    ap = argparse.ArgumentParser(description="Tune librsort on this GPU and write a tune table")
    ap.add_argument("--device", type=int, default=0)
    ap.add_argument("--out", default="rsort.tune")
    ap.add_argument("--keys", type=int, default=1 << 23, help="keys per workload")
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args()
    r = tune(args.device, keys_per_class=args.keys, reps=args.reps)
    write_table(r, args.out)
    print(json.dumps(r.as_dict()))


if __name__ == "__main__":
    main()
