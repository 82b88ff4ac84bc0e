"""Benchmark: robust sample sort of 2^28 uint64 keys (p = 1024 virtual
partitions, Uniform instance, seed 1) on one GB300, through the C ABI.

Prints ONE JSON line (rank 0).  A step is one full rsort_sort call (all
partition levels and the in-SM bucket sorts) over the resident input.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl rsort|reference]

--impl reference times the CPU oracle (a textbook merge sort on (key,
position)) on the host cores, on bounded samples of the same workload.
With N > 1 (torchrun) every rank sorts its own instance (weak scaling, no
collective on the data path); the timed region is bracketed by barriers and
the slowest rank's time is reported.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_KEYS = 1 << 28
P_VIRTUAL = 1024
WORKLOAD = "Uniform uint64 keys, n=2^28, p=1024 virtual partitions, seed 1"
METRIC = "GKeys/s"
CPU_SAMPLE = 1 << 24   # cpu_baseline leg: 3 runs of this many keys
REF_SAMPLE = 1 << 24   # --impl reference: keys per step (all-core oracle)

# algorithmic HBM bytes per key of each kernel's input (8 B key, 4 B position)
ALGO_BYTES_PER_KEY = {
    "L1.classify": 8,       # read keys
    "L1.scatter": 20,       # read keys, write (key, position)
    "L2.classify": 8,       # read keys (positions only on key ties)
    "L2.scatter": 24,       # read + write (key, position)
    "L3.classify": 8,
    "L3.scatter": 24,
    "local_sort": 24,       # read + write (key, position), buckets <= 1024 keys
    "local_sort_mid": 24,   # buckets of 1025..2048 keys
    "local_sort_medium": 24,  # buckets of 2049..4096 keys
}


# DRAM bytes (read + write) per input key of a kernel, from one ncu capture of
# the current kernel code on a smaller case of the same workload (traffic
# grows in proportion to the keys; the capture and command are summarised in
# profiles/).  Remove an entry whenever its kernel changes.
MEASURED_TRAFFIC_PER_KEY = {
    "L1.scatter": 23.64,       # 0.7696 + 0.8171 GB at 2^26 keys (k_scatter_units<512,12,0,0>)
    "L1.classify": 9.50,       # 0.5473 + 0.0897 GB (k_classify_ids, ids included)
    "L2.scatter": 25.35,       # 0.9512 + 0.7498 GB (k_scatter_units<512,12,1,0>)
    "L2.classify": 9.39,       # 0.5517 + 0.0787 GB (k_classify_count<2>)
    "local_sort_mid": 23.15,   # 0.6691 + 0.6138 GB over 55.4 M keys of the class
    "local_sort_medium": 18.42,  # 0.1037 + 0.0548 GB over 8.6 M keys (writes left in L2)
    "local_sort": 13.08,       # 0.0379 + 0.0025 GB over 3.1 M keys (writes left in L2)
}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self.t = None
        self.first = 0

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # nvidia-smi needs a moment before its first sample: wait for it so
            # that the samples kept (from mark() on) cover the timed region
            t0 = time.time()
            while not self.lines and time.time() - t0 < 5 and self.proc.poll() is None:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        self.first = 0

    def mark(self):
        """Samples before this call (start-up, warm-up) are not reported."""
        self.first = len(self.lines)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines[self.first:]:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(value: float, dist, device) -> float:
    """The slowest rank's value (weak scaling: every rank sorts its own
    instance and the job takes as long as its slowest rank)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gkeys(keys_per_rank: int, world: int, ms_step: float) -> float:
    """Keys sorted by all ranks per second of the slowest rank, in GKeys/s."""
    return keys_per_rank * world / (ms_step / 1e3) / 1e9


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    """The CPU oracle as it stands, on bounded samples of the same workload,
    on every host core (its all-core merge sort: nproc chunks sorted by their
    own threads, then pairwise merges)."""
    import numpy as np

    import instances
    import oracle

    ws, rank, _ = _dist()
    if rank != 0:
        return
    n = args.n
    chunk = min(REF_SAMPLE, max(1, n // 2))
    keys = instances.generate("uniform", n, p=P_VIRTUAL, seed=1)
    cores = os.cpu_count() or 1
    times = []
    for step in range(args.warmup + args.steps):
        lo = (step * chunk) % max(1, n - chunk)
        sample = np.ascontiguousarray(keys[lo:lo + chunk])
        t0 = time.perf_counter()
        oracle.sort_parallel(sample, threads=cores)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
    ms = 1e3 * statistics.mean(times)
    value = chunk / (ms / 1e3) / 1e9
    sample_desc = (f"{chunk} consecutive keys of the n = {n} Uniform input per step, "
                   f"all-core merge sort on {cores} threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC,
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD if n == N_KEYS else
                   f"Uniform uint64 keys, n={n}, p={P_VIRTUAL} virtual partitions, seed 1",
                   "n": n, "p": P_VIRTUAL},
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": cores, "kind": "oracle",
                         "sample": sample_desc},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }))


def cpu_baseline_leg():
    """Oracle timed on the host on a bounded sample (rank 0, N = 1 only): the
    all-core merge sort (nproc equal chunks sorted by their own threads, then
    pairwise merges) and the single-thread one."""
    import numpy as np

    import instances
    import oracle

    sample = np.ascontiguousarray(instances.generate("uniform", CPU_SAMPLE, p=P_VIRTUAL, seed=1))
    cores = os.cpu_count() or 1
    ts = []
    for _ in range(3):
        t0 = time.perf_counter()
        oracle.sort_parallel(sample, threads=cores)
        ts.append(time.perf_counter() - t0)
    t0 = time.perf_counter()
    oracle.sort(sample)
    t1 = time.perf_counter() - t0
    v = CPU_SAMPLE / statistics.median(ts) / 1e9
    return {"value": v, "unit": METRIC, "cores": cores, "kind": "oracle",
            "sample": f"first {CPU_SAMPLE} keys of the Uniform instance; all-core merge sort "
                      f"({cores} threads), median of 3",
            "single_core_value": CPU_SAMPLE / t1 / 1e9, "nproc": cores}


def _event_ms(fn, stream, reps):
    import torch
    ts = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def config1_leg(ctx, dev, n=1 << 20, p=64, reps=20):
    """Plain sort of 2^20 uniform uint64 keys as p = 64 virtual partitions."""
    import torch

    import instances

    keys = instances.generate_torch("uniform", n, p=p, seed=1, device=dev)
    ko = torch.empty_like(keys)
    po = torch.empty(n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    fn = lambda: ctx.sort(keys, p=p, keys_out=ko, perm_out=po)
    for _ in range(3):
        fn()
    ms = _event_ms(fn, stream, reps)
    ref_k, ref_p = ko.clone(), po.clone()
    # the same call's ~30 launches captured once in a CUDA graph and replayed
    # (the launch sequence of a sort this small costs about what its kernels do)
    side = torch.cuda.Stream(dev)
    with torch.cuda.stream(side):
        ctx.sort(keys, p=p, keys_out=ko, perm_out=po, stream=side)
    torch.cuda.synchronize(dev)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        ctx.sort(keys, p=p, keys_out=ko, perm_out=po, stream=side)
    ko.zero_()
    po.zero_()
    g.replay()
    torch.cuda.synchronize(dev)
    same = bool(torch.equal(ko, ref_k)) and bool(torch.equal(po, ref_p))
    ms_graph = _event_ms(g.replay, stream, reps)
    return {"workload": f"Uniform uint64 keys, n=2^20, p={p}, seed 1", "ms": ms,
            "gkeys_s": n / (ms / 1e3) / 1e9, "graph_replay_ms": ms_graph,
            "graph_replay_gkeys_s": n / (ms_graph / 1e3) / 1e9, "graph_identical": same}


def instances_leg(ctx, dev, n=1 << 28, p=1024, reps=3):
    """Configs 2 and 3: the full sort on every input instance at 2^28 keys and
    p = 1024 (Section 6's robustness claim: duplicates, skew and presorted
    orders should neither unbalance nor slow the sort).  Device time (median
    of reps after one warm-up), GKeys/s and the level-1 balance (largest
    virtual partition over the mean n/p)."""
    import torch

    import instances

    out = {"workload": f"rsort_sort of n=2^{n.bit_length() - 1} u64 keys, p={p}, per instance"}
    stream = torch.cuda.current_stream(dev)
    ko = torch.empty(n, dtype=torch.int64, device=dev)
    po = torch.empty(n, dtype=torch.int32, device=dev)
    for name in instances.NAMES:
        keys = instances.generate_torch(name, n, p=p, seed=1, device=dev)
        _, _, st = ctx.sort(keys, p=p, keys_out=ko, perm_out=po, stats=True)
        ms = _event_ms(lambda: ctx.sort(keys, p=p, keys_out=ko, perm_out=po), stream, reps)
        out[name] = {"ms": ms, "gkeys_s": n / (ms / 1e3) / 1e9,
                     "max_over_mean": st.max_over_mean}
        del keys
    return out


def partition_leg(ctx, dev, n=1 << 26, k=1024, over=10, reps=3):
    """The partition step alone on duplicate-heavy and unique inputs: the
    robust step, the NTB ablation (classification by key only) and AMS
    overpartitioning (b = 10: eps = 0.2 with one level).  Reports device time
    and the largest partition over the mean n/k."""
    import torch

    import instances

    out = {"workload": f"one partition step, n=2^{n.bit_length() - 1}, k={k}, seed 1",
           "variants": {"robust": "tie_break=1, b=1", "ntb": "tie_break=0, b=1",
                        f"over{over}": f"tie_break=1, b={over}"}}
    stream = torch.cuda.current_stream(dev)
    for name in ("uniform", "zero", "deter_dupl", "rand_dupl"):
        keys = instances.generate_torch(name, n, p=k, seed=1, device=dev)
        row = {}
        for label, kw in (("robust", {}), ("ntb", {"tie_break": False}),
                          (f"over{over}", {"overpartition": over})):
            res = ctx.partition_ex(keys, k, seed=1, **kw)
            ms = _event_ms(lambda: ctx.partition_ex(keys, k, seed=1, **kw), stream, reps)
            sizes = torch.diff(res[2]).max().item()
            row[label] = {"ms": ms, "max_over_mean": sizes / (n / k)}
            del res
        out[name] = row
        del keys
        torch.cuda.empty_cache()
    return out


def autotune_leg(dev, path):
    """Runs the autotuner on this GPU and writes its table (bounded: about
    a dozen seconds)."""
    from paper_1606_08766_gb300 import autotune

    t0 = time.perf_counter()
    r = autotune.tune(dev.index, keys_per_class=1 << 24, reps=3)
    autotune.write_table(r, path)
    return {"seconds": time.perf_counter() - t0, "table": r.table(),
            "mixed_default_ms": r.default_ms, "mixed_tuned_ms": r.tuned_ms,
            "reverted_to_defaults": r.reverted,
            "knobs": {k.name: {"chosen": k.chosen, "default": k.default,
                               "ms": {str(v): round(t, 4) for v, t in k.ms.items()}}
                      for k in r.knobs}}


def batched_leg(ctx, tuned, dev, nseg, maxlog, total_cap=None, plain_max=20_000, label=""):
    """Batched segmented sort of float64 segments (log-uniform sizes, 10%
    duplicates) in one launch sequence with the default plan and with the
    autotuned one, replayed from a CUDA graph, against one plain rsort_sort
    per segment (all segments, or the first plain_max)."""
    import torch

    import instances

    x, o = instances.segmented_f64_torch(nseg, maxlog, seed=1, total_cap=total_cap, device=dev)
    n = int(x.numel())
    nsegs = int(o.numel() - 1)
    ko = torch.empty_like(x)
    po = torch.empty(n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    res = {}
    for name, c in (("default", ctx), ("tuned", tuned)):
        for _ in range(2):
            c.segmented(x, o, keys_out=ko, perm_out=po)
        res[name] = _event_ms(lambda: c.segmented(x, o, keys_out=ko, perm_out=po), stream, 3)
    # the tuned launch sequence captured once in a CUDA graph and replayed
    side = torch.cuda.Stream(dev)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        tuned.segmented(x, o, keys_out=ko, perm_out=po, stream=side)
    torch.cuda.synchronize(dev)
    with torch.cuda.graph(g, stream=side):
        tuned.segmented(x, o, keys_out=ko, perm_out=po, stream=side)
    g.replay()
    torch.cuda.synchronize(dev)
    ms_graph = _event_ms(g.replay, stream, 3)
    # one plain sort per segment (pointer-level calls, same stream)
    offs_l = o.cpu().tolist()
    nplain = min(plain_max, nsegs)
    m = offs_l[nplain]
    ko2 = torch.empty(m, dtype=torch.float64, device=dev)
    po2 = torch.empty(m, dtype=torch.int32, device=dev)
    xp, kp, pp, sh = x.data_ptr(), ko2.data_ptr(), po2.data_ptr(), stream.cuda_stream

    def plain_pass():
        for s in range(nplain):
            a, b = offs_l[s], offs_l[s + 1]
            ctx.sort_raw(1, xp + 8 * a, kp + 8 * a, pp + 4 * a, b - a, 1, 1, sh)

    plain_pass()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    plain_pass()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_plain = e0.elapsed_time(e1)
    wall_plain = time.perf_counter() - t0
    tuned.segmented(x, o, keys_out=ko, perm_out=po)
    same = bool(torch.equal(ko2, ko[:m])) and bool(torch.equal(po2, po[:m]))
    gk = lambda keys_, ms_: keys_ / (ms_ / 1e3) / 1e9
    plain_gk = m / max(wall_plain, ms_plain / 1e3) / 1e9
    return {"workload": f"{label}{nsegs} float64 segments, sizes floor(exp(U ln 2^{maxlog})), "
                        f"10% duplicates, {n} keys",
            "keys": n, "segments": nsegs,
            "default_gkeys_s": gk(n, res["default"]), "default_ms": res["default"],
            "tuned_gkeys_s": gk(n, res["tuned"]), "tuned_ms": res["tuned"],
            "tuned_over_default": res["default"] / res["tuned"],
            "graph_replay_gkeys_s": gk(n, ms_graph),
            "plain_per_segment_gkeys_s": plain_gk,
            "plain_subset": f"first {nplain} segments ({m} keys), one rsort_sort each",
            "speedup_vs_plain": gk(n, res["tuned"]) / plain_gk,
            "identical_to_plain": same}


def serving_leg(dev, requests=1000, slots=1000, lo_log2=4, hi_log2=26,
                loads=(0.5, 0.8, 0.95, 1.2), budget=64 << 30, seed=5):
    """Config 5: a stream of sort requests with sizes log-uniform in
    [2^lo, 2^hi], u64 or f64 keys (50/50), each drawing one of the 11
    instances, p_virtual = min(1024, ceil(n / 2^8)), served by continuous
    batching under an HBM budget, against serial plain sorts of the same
    requests.  Capacity = everything offered at once; then Poisson arrivals
    at the given fractions of that capacity, each with p50 / p99 latency.

    The requests' device buffers stay resident: min(requests, slots) distinct
    requests are drawn, and arrival i reuses the buffers of request
    i mod slots, once the arrival that used them before has finished (an
    arrival that has to wait for that is counted as blocked: the stream is
    then no longer open-loop for it)."""
    import math
    import random

    import torch

    import instances
    from paper_1606_08766_gb300 import Context

    rng = random.Random(seed)
    nslots = min(requests, slots)
    sizes = [int(math.exp(rng.uniform(lo_log2 * math.log(2), hi_log2 * math.log(2))))
             for _ in range(nslots)]
    reqs = []
    for i, n in enumerate(sizes):
        name = instances.NAMES[rng.randrange(len(instances.NAMES))]
        p = min(1024, -(-n // 256))
        k = instances.generate_torch(name, n, p=max(p, 1), seed=seed + i, device=dev)
        if rng.random() < 0.5:
            t, kt = k, 0
        else:
            t, kt = k.to(torch.float64), 1
        reqs.append((t, torch.empty_like(t), torch.empty(n, dtype=torch.int32, device=dev), kt, p))
    total = sum(sizes)
    torch.cuda.synchronize(dev)
    ctx = Context(dev.index, hbm_budget_bytes=budget)
    assert requests <= ctx.get_tunable("serve_history"), "every ticket must stay readable"

    def offer_all():
        t0 = time.perf_counter()
        ts = [ctx.submit(t, o, pm, p=p, key_type=kt) for t, o, pm, kt, p in reqs]
        for t in ts:
            assert ctx.wait(t, 300) == 0
        return time.perf_counter() - t0

    offer_all()                        # warm-up: every request once through the server
    ctx.reset_serve_stats()
    wall = offer_all()
    sat = ctx.serve_stats()
    # serial plain sorts, one rsort_sort per request on one stream
    stream = torch.cuda.current_stream(dev)
    plain = Context(dev.index)
    for t, o, pm, kt, p in reqs[:50]:
        plain.sort_raw(kt, t.data_ptr(), o.data_ptr(), pm.data_ptr(), t.numel(), p, 1,
                       stream.cuda_stream)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for t, o, pm, kt, p in reqs:
        plain.sort_raw(kt, t.data_ptr(), o.data_ptr(), pm.data_ptr(), t.numel(), p, 1,
                       stream.cuda_stream)
    torch.cuda.synchronize(dev)
    wall_plain = time.perf_counter() - t0
    plain.close()
    cap_rate = nslots / wall
    out = {"workload": f"{requests} requests (of the 200,000 of the stated stream) cycling "
                       f"through {nslots} distinct resident requests, sizes "
                       f"log-uniform in [2^{lo_log2}, 2^{hi_log2}], u64/f64 50/50, a random "
                       f"instance each, p_virtual = min(1024, ceil(n/2^8)), {total} keys "
                       f"in the distinct requests, HBM budget {budget >> 30} GiB",
           "capacity_requests_s": cap_rate, "served_gkeys_s": total / wall / 1e9,
           "plain_serial_requests_s": nslots / wall_plain,
           "plain_serial_gkeys_s": total / wall_plain / 1e9,
           "speedup_vs_plain": wall_plain / wall,
           "saturated_p50_us": sat["p50_us"], "saturated_p99_us": sat["p99_us"],
           "mean_batch_requests": sat["mean_batch_requests"], "loads": {}}
    for load in loads:
        rate = load * cap_rate
        ctx.reset_serve_stats()
        ts = []
        blocked = 0
        keys_served = 0
        t_start = time.perf_counter()
        t_next = t_start
        for i in range(requests):
            t_next += rng.expovariate(rate)
            while time.perf_counter() < t_next:
                pass
            t, o, pm, kt, p = reqs[i % nslots]
            if i >= nslots:  # this request's buffers: their previous user must be done
                prev = ts[i - nslots]
                blocked += ctx.poll(prev)[0] == 1
                assert ctx.wait(prev, 300) == 0
            ts.append(ctx.submit(t, o, pm, p=p, key_type=kt))
            keys_served += t.numel()
        for t in ts[max(0, requests - nslots):]:
            assert ctx.wait(t, 300) == 0
        el = time.perf_counter() - t_start
        st = ctx.serve_stats()
        assert st["completed"] == requests
        out["loads"][str(load)] = {"offered_requests_s": rate, "served_requests_s": requests / el,
                                   "served_gkeys_s": keys_served / el / 1e9, "p50_us": st["p50_us"],
                                   "p99_us": st["p99_us"], "max_us": st["max_us"],
                                   "blocked_arrivals": blocked}
    ctx.close()
    del reqs
    torch.cuda.empty_cache()
    return out


def run_rsort(args):
    import numpy as np
    import torch

    import instances
    from paper_1606_08766_gb300 import Context

    ws, rank, local = _dist()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = args.n
    keys_h = instances.generate("uniform", n, p=P_VIRTUAL, seed=1 + rank)
    keys = torch.from_numpy(keys_h.view(np.int64)).to(dev)
    keys_out = torch.empty_like(keys)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    ctx = Context(local)
    tunables = {}
    for kv in args.tunable:
        name, val = kv.split("=", 1)
        ctx.set_tunable(name, int(val))
        tunables[name] = int(val)
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream

    def step():
        ctx.sort_raw(0, keys.data_ptr(), keys_out.data_ptr(), perm.data_ptr(), n, P_VIRTUAL,
                     1, sh)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize(dev)
    ctx.check()

    # -- timed region: device time with CUDA events; per-kernel events inside
    ctx.set_profiling(True)
    ctx.phase_times()
    launches0 = ctx.launch_count()
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks.mark()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms_total = ev0.elapsed_time(ev1)
    launches = ctx.launch_count() - launches0
    phases = ctx.phase_times()
    ctx.set_profiling(False)
    ctx.check()
    ms_step = max_over_ranks(ms_total / args.steps, dist, dev)
    value = whole_job_gkeys(n, ws, ms_step)

    # -- per-kernel roofline (dominant kernel)
    _, _, st = ctx.sort(keys, p=P_VIRTUAL, seed=1, keys_out=keys_out, perm_out=perm, stats=True)
    torch.cuda.synchronize(dev)
    elems = {"L1": n, "L2": st.level_elems[1] if len(st.level_elems) > 1 else n,
             "L3": st.level_elems[2] if len(st.level_elems) > 2 else 0,
             "local_copy": st.class_elems[0], "local_sort": st.class_elems[1],
             "local_sort_mid": st.class_elems[2], "local_sort_medium": st.class_elems[3],
             "local_big": st.class_elems[4]}
    peak, peak_kind = _peaks()
    kernels = {}
    for name, (ms, cnt) in phases.items():
        per = ms / max(cnt, 1)
        info = {"ms_per_launch": per, "launches": cnt, "share": ms / max(ms_total, 1e-9)}
        if name in ALGO_BYTES_PER_KEY:
            units = elems.get(name.split(".")[0] if "." in name else name, n)
            info["algo_bytes"] = ALGO_BYTES_PER_KEY[name] * units
            info["gbs"] = info["algo_bytes"] / (per / 1e3) / 1e9
        kernels[name] = info
    dom = max((k for k in kernels if "gbs" in kernels[k]), key=lambda k: kernels[k]["ms_per_launch"]
              * kernels[k]["launches"])

    def roofline_of(name):
        t = MEASURED_TRAFFIC_PER_KEY.get(name)
        return {"kernel": name, "bound": "hbm", "achieved": kernels[name]["gbs"], "peak": peak,
                "unit": "GB/s", "frac": kernels[name]["gbs"] / peak, "peak_kind": peak_kind,
                "algo_bytes_per_launch": kernels[name]["algo_bytes"],
                "traffic": (t * elems.get(name.split(".")[0] if "." in name else name, n)
                            if t else None)}

    roof = roofline_of(dom)
    # the same entry for every kernel with algorithmic bytes (classify and
    # scatter of each level, the in-SM sort classes), largest first
    rooflines = [roofline_of(k) for k in sorted(
        (k for k in kernels if "gbs" in kernels[k]),
        key=lambda k: -kernels[k]["ms_per_launch"] * kernels[k]["launches"])]

    # -- end to end through the C ABI with host buffers (pinned): every step
    # copies its input up and its result (keys + permutation) down, inside the
    # timed region.  Serial: one stream, copy / sort / copy in turn.
    # Pipelined: consecutive steps overlap on three streams (upload, sort,
    # download) with three device buffer sets, as a streaming caller would
    # run; the host link (both directions at once) is the bound.
    NSETS = 3
    keys_pin = torch.from_numpy(keys_h.view(np.int64)).pin_memory()
    outs_pin = [(torch.empty(n, dtype=torch.int64).pin_memory(),
                 torch.empty(n, dtype=torch.int32).pin_memory()) for _ in range(NSETS)]
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    serial_steps = max(1, min(args.steps, 3))
    # one untimed pass through every pinned buffer first (first DMA to or
    # from a freshly pinned buffer can cost more than the copy)
    for j in range(NSETS):
        keys.copy_(keys_pin, non_blocking=True)
        outs_pin[j][0].copy_(keys_out, non_blocking=True)
        outs_pin[j][1].copy_(perm, non_blocking=True)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(serial_steps):
        keys.copy_(keys_pin, non_blocking=True)
        step()
        outs_pin[0][0].copy_(keys_out, non_blocking=True)
        outs_pin[0][1].copy_(perm, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    serial_ms = max_over_ranks(e0.elapsed_time(e1) / serial_steps, dist, dev)

    dev_in = [keys] + [torch.empty_like(keys) for _ in range(NSETS - 1)]
    dev_out = [(keys_out, perm)] + [(torch.empty_like(keys_out), torch.empty_like(perm))
                                    for _ in range(NSETS - 1)]
    s_up, s_sort, s_down = (torch.cuda.Stream(dev), torch.cuda.Stream(dev),
                            torch.cuda.Stream(dev))
    up_done = [torch.cuda.Event() for _ in range(NSETS)]
    sort_done = [torch.cuda.Event() for _ in range(NSETS)]
    down_done = [torch.cuda.Event() for _ in range(NSETS)]
    pipe_steps = max(6, min(args.steps, 12))
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(s_up)
    for i in range(pipe_steps):
        j = i % NSETS
        with torch.cuda.stream(s_up):
            if i >= NSETS:
                s_up.wait_event(sort_done[j])      # step i-NSETS has read dev_in[j]
            dev_in[j].copy_(keys_pin, non_blocking=True)
            up_done[j].record(s_up)
        s_sort.wait_event(up_done[j])
        if i >= NSETS:
            s_sort.wait_event(down_done[j])        # dev_out[j] is downloaded
        ctx.sort_raw(0, dev_in[j].data_ptr(), dev_out[j][0].data_ptr(),
                     dev_out[j][1].data_ptr(), n, P_VIRTUAL, 1, s_sort.cuda_stream)
        sort_done[j].record(s_sort)
        with torch.cuda.stream(s_down):
            s_down.wait_event(sort_done[j])
            outs_pin[j][0].copy_(dev_out[j][0], non_blocking=True)
            outs_pin[j][1].copy_(dev_out[j][1], non_blocking=True)
            down_done[j].record(s_down)
    p1.record(s_down)
    torch.cuda.synchronize(dev)
    ctx.check()
    pipe_ms = max_over_ranks(p0.elapsed_time(p1) / pipe_steps, dist, dev)
    for j in range(1, NSETS):
        assert bool(torch.equal(outs_pin[0][0], outs_pin[j][0])), "pipelined outputs differ"
    e2e = {"value": (n * ws) / (pipe_ms / 1e3) / 1e9, "unit": METRIC,
           "h2d_bytes_per_step": n * 8, "d2h_bytes_per_step": n * 8 + n * 4,
           "mode": "pipelined over 3 streams and 3 buffer sets (upload / sort / download of "
                   "consecutive steps overlap)",
           "serial_value": (n * ws) / (serial_ms / 1e3) / 1e9, "steps": pipe_steps}
    del dev_in, dev_out, outs_pin

    cpu = cpu_baseline_leg() if (rank == 0 and ws == 1) else None
    extra = {}
    if rank == 0 and ws == 1 and not args.skip_systems:
        import tempfile

        from paper_1606_08766_gb300 import Context as _Ctx
        del keys_pin, keys, keys_out, perm
        torch.cuda.empty_cache()
        extra["config1"] = config1_leg(ctx, dev)
        extra["instances"] = instances_leg(ctx, dev)
        torch.cuda.empty_cache()
        extra["partition_variants"] = partition_leg(ctx, dev)
        table = os.path.join(tempfile.mkdtemp(), "gb300.tune")
        extra["autotune"] = autotune_leg(dev, table)
        tuned = _Ctx(local, tune_table=table)
        extra["batched"] = {
            "4a": batched_leg(ctx, tuned, dev, 100_000, 15, label="config 4a: "),
            "4b": batched_leg(ctx, tuned, dev, 100_000, 20, total_cap=N_KEYS,
                              label="config 4b: ")}
        tuned.close()
        torch.cuda.empty_cache()
        extra["serving"] = serving_leg(dev, requests=args.serving_requests)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD if n == N_KEYS else
                       f"Uniform uint64 keys, n={n}, p=1024 virtual partitions, seed 1",
                       "n": n, "p": P_VIRTUAL,
                       "l2": "inputs (2 GiB keys) larger than L2 (129 MB); no flush needed",
                       "max_over_mean": st.max_over_mean, "levels": st.levels,
                       "tunables": {"classifier": ctx.get_tunable("classifier")}},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
            "gpu_launches": launches, "rooflines": rooflines, "kernels": kernels, **extra,
        }))
    ctx.close()
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="rsort", choices=["rsort", "reference"])
    ap.add_argument("--skip-systems", action="store_true",
                    help="skip the batched-segmented and serving legs")
    ap.add_argument("--tunable", action="append", default=[],
                    help="name=value tunable of the library context (repeatable)")
    ap.add_argument("--serving-requests", type=int, default=1000,
                    help="arrivals of the serving leg (the stated stream has 200,000; "
                         "its buffers cycle through at most 1,000 resident requests)")
    ap.add_argument("--n", type=int, default=N_KEYS,
                    help="keys per GPU (default 2^28; smaller values are for profiling)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_rsort(args)


if __name__ == "__main__":
    main()
