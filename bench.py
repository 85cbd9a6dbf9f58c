#!/usr/bin/env python
"""Adaptive Hybrid Sort on GB300: throughput of the whole hot path.

One step = the AUTO pipeline (features -> selector -> strategy) over the six
single-array workloads of size n = 2^28 uint32 (uniform k=4096; Zipf(1.1)
over 1,024 distinct values; uniform 32-bit; sorted; 1% swapped; reversed),
inputs resident in HBM.  Prints one JSON line (rank 0).

  --impl ours       the CUDA library (default)
  --impl reference  the CPU oracle on a bounded sample of the same workload
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

VARIANTS = "abcdef"
METRIC = "Gkeys/s & % HBM roofline per strategy; batched vs per-array on 1 GB300; p50/p99"

# Algorithmic bytes per key of each kernel (w = key bytes, v = payload bytes):
# what the method must move, not what a kernel happens to move.
def algo_bytes_per_item(kernel: str, w: int, v: int) -> float:
    table = {
        "features_minmax": w, "features_histogram": w, "counting_fill": w,
        "radix_digit_hist": w, "radix_onesweep": 2 * (w + v), "sample_count": w,
        "sample_scatter": 2 * (w + v), "bucket_sort_1k": 2 * (w + v), "bucket_sort_2k": 2 * (w + v),
        "segradix_count": w, "segradix_scatter": 2 * (w + v),
        "bucket_sort_3k": 2 * (w + v), "bucket_sort_4k": 2 * (w + v),
        "bucket_sort_4.5k": 2 * (w + v), "bucket_sort_6k": 2 * (w + v), "bucket_sort_8k": 2 * (w + v),
        "blocksort_single": 2 * (w + v), "copy": 8, "reverse": 2 * w,
        "msd_scatter": 2 * w, "msd_bin_minmax": w,
        "sparse_count": w, "sparse_fill": w,
    }
    return table.get(kernel, 0.0)


def kernel_table(kt, peak, w: int = 4, v: int = 0):
    """Per kernel: launches, total ms, share of kernel time and, where the
    kernel's algorithmic bytes per key are known, its GB/s over all launches
    and that as a fraction of `peak` (the per-pass roofline)."""
    total = sum(x[1] for x in kt.values()) or 1.0
    out = {}
    for k, (c, m, items) in sorted(kt.items(), key=lambda kv: -kv[1][1]):
        e = {"launches": c, "ms": round(m, 3), "share": round(m / total, 4)}
        per = algo_bytes_per_item(k, w, v)
        if per and items and m > 0:
            gbs = per * items / (m / 1e3) / 1e9
            e["gbs"] = round(gbs, 1)
            e["frac"] = round(gbs / peak, 4) if peak else None
        out[k] = e
    return out


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d.get("hbm_gbs"), "measured"
    return 6800.0, "fallback"


def kernel_source_hash(kernel: str):
    files = {"radix": "radix.cu", "sample": "samplesort.cu", "msd": "samplesort.cu",
             "bucket": "blocksort.cuh", "sparse_count": "sparse.cu", "sparse_fill": "counting.cu",
             "features": "features.cu", "counting": "counting.cu", "copy": "counting.cu",
             "reverse": "counting.cu"}
    for pre, f in files.items():
        if kernel.startswith(pre):
            with open(os.path.join(ROOT, "paper_2506_20677_gb300", "csrc", f), "rb") as fh:
                return hashlib.sha256(fh.read()).hexdigest()[:16]
    return None


def ncu_traffic(kernel: str, items_per_launch: float):
    """DRAM bytes per launch from the committed ncu summary, scaled to this
    launch's size; None when absent or when the kernel source changed since."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    e = d.get(kernel)
    if not e or e.get("source_hash") != kernel_source_hash(kernel):
        return None
    return e["dram_bytes_per_item"] * items_per_launch


class ClockSampler:
    def __init__(self):
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def start(self):
        def run():
            q = ("--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap")
            dev = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0] or "0"
            while not self._stop.is_set():
                try:
                    out = subprocess.run(["nvidia-smi", q, "--format=csv,noheader,nounits", "-i",
                                          str(int(os.environ.get("LOCAL_RANK", "0")))
                                          if dev.isdigit() else "0"],
                                         capture_output=True, text=True, timeout=5).stdout
                    for line in out.strip().splitlines():
                        f = [x.strip() for x in line.split(",")]
                        if len(f) >= 6:
                            self.samples.append(f)
                except Exception:
                    pass
                self._stop.wait(0.2)
        self._t = threading.Thread(target=run, daemon=True)
        self._t.start()

    def stop(self):
        self._stop.set()
        if self._t:
            self._t.join(timeout=10)
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if s[2 + i].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


def bind_gpu_local_cpus(local: int):
    """Run on the CPUs next to the GPU, so that pinned host buffers (placed
    where they are first touched) sit in that CPU's memory; skipped when the
    topology cannot be read."""
    try:
        bus = subprocess.run(["nvidia-smi", "--query-gpu=pci.bus_id", "--format=csv,noheader",
                              "-i", str(local)], capture_output=True, text=True, timeout=10).stdout.strip()
        dom, rest = bus.split(":", 1)
        path = f"/sys/bus/pci/devices/{int(dom, 16):04x}:{rest.lower()}/local_cpulist"
        with open(path) as fh:
            spec = fh.read().strip()
        cpus = set()
        for part in spec.split(","):
            a, _, b = part.partition("-")
            cpus.update(range(int(a), int(b or a) + 1))
        if cpus:
            os.sched_setaffinity(0, cpus)
            return sorted(cpus)
    except Exception:
        pass
    return None


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        # Replicas exchange only a barrier and one timing value.
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return world, rank, local


def job_value(world: int, keys_per_step: int, steps: int, ms_max: float) -> float:
    """Whole-job Gkeys/s of weakly scaled replicas: every rank sorts its own
    keys_per_step keys per step; the job time is the slowest rank's."""
    return world * keys_per_step * steps / (ms_max / 1e3) / 1e9


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, x: float) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------- CPU oracle arm
def oracle_sample_run(n_sample: int, seed_offset: int = 0):
    """Time the oracle (features -> PAPER FSM -> strategy) on the first
    n_sample keys of each workload array.  Returns (keys, seconds, picks)."""
    import numpy as np

    import oracle
    from gen import host as gen
    keys_total, secs, picks = 0, 0.0, {}
    for v in VARIANTS:
        if v in "abc":
            a = gen.config2(v, n_sample)
        else:
            # sorted / swapped / reversed variants of a uniform sample
            a = gen.config2(v, n_sample)
        t0 = time.perf_counter()
        _, _, chosen, _ = oracle.sort(a, profile=oracle.PAPER)
        secs += time.perf_counter() - t0
        keys_total += len(a)
        picks[v] = oracle.STRATEGY_NAMES[chosen]
    return keys_total, secs, picks


def std_sort_context(n_sample: int):
    """libstdc++ std::sort on the first n_sample keys of each array, one core
    (context beside the oracle; Gkeys/s)."""
    import oracle
    from gen import host as gen
    keys, secs = 0, 0.0
    for v in VARIANTS:
        a = gen.config2(v, n_sample)
        t0 = time.perf_counter()
        oracle.std_sort(a)
        secs += time.perf_counter() - t0
        keys += len(a)
    return round(keys / secs / 1e9, 4)


def _c4_oracle_worker(share, n_seg, barrier, q):
    """One process of the all-core oracle baseline: generate this worker's
    config-4 segments, wait for the others, then sort them with the oracle."""
    import oracle
    from gen import host as gen
    lengths, types, _ = gen.config4_layout()
    segs = [gen.config4_segment(s, int(lengths[s]), int(types[s])) for s in range(share, n_seg, q[1])]
    oracle.lib()
    barrier.wait()
    t0 = time.time()
    keys = 0
    for a in segs:
        oracle.sort(a, profile=oracle.PAPER)
        keys += len(a)
    q[0].put((t0, time.time(), keys))


def oracle_config4_all_cores(n_seg: int):
    """The oracle on the first n_seg segments of config 4, one segment at a
    time per process, on every host core (processes started with spawn, after
    the GPU is in use).  Gkeys/s = keys / wall time of the sorting phase."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(cores)
    q = ctx.Queue()
    procs = [ctx.Process(target=_c4_oracle_worker, args=(i, n_seg, barrier, (q, cores)))
             for i in range(cores)]
    for p in procs:
        p.start()
    res = [q.get(timeout=600) for _ in procs]
    for p in procs:
        p.join(timeout=60)
    start = min(r[0] for r in res)
    end = max(r[1] for r in res)
    keys = sum(r[2] for r in res)
    return {"value": round(keys / (end - start) / 1e9, 4), "unit": "Gkeys/s", "cores": cores,
            "kind": "oracle", "sample": f"first {n_seg} segments of config 4 ({keys} keys, "
                                        f"{end - start:.1f} s), one segment per process at a time"}


def run_reference(args, world, rank):
    if rank != 0:
        return
    import oracle
    oracle.build()
    n_sample = args.ref_sample
    for _ in range(args.warmup):
        oracle_sample_run(n_sample // 4)
    times, keys = [], 0
    picks = {}
    for _ in range(args.steps):
        k, s, picks = oracle_sample_run(n_sample)
        times.append(s)
        keys = k
    tot = sum(times)
    value = keys * args.steps / tot / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gkeys/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "config2 a-f (uint32; oracle on a bounded sample)",
                   "n_per_array_sample": n_sample, "profile": "PAPER", "picks": picks},
        "cpu_baseline": {"value": value, "unit": "Gkeys/s", "cores": 1, "kind": "oracle",
                         "sample": f"first {n_sample} keys of each of the 6 arrays"},
        "e2e": {"value": value, "unit": "Gkeys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    bound = bind_gpu_local_cpus(local)
    import paper_2506_20677_gb300 as ahs
    from gen import device as gdev

    n = args.n
    inputs = {}
    for v in VARIANTS:
        inputs[v] = gdev.config2(v, n)
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()

    ctx = ahs.Context(local, select_mode=ahs.AHS_SEL_GB300)
    stream = torch.cuda.current_stream()

    def step(record=None):
        picks = {}
        for v in VARIANTS:
            if record is not None:
                ev0 = torch.cuda.Event(enable_timing=True)
                ev1 = torch.cuda.Event(enable_timing=True)
                ev0.record(stream)
            r = ctx.sort(inputs[v], out=out, key_type=ahs.AHS_U32, stream=stream)
            if record is not None:
                ev1.record(stream)
                record.append((v, ev0, ev1))
            picks[v] = ahs.STRATEGY_NAMES[r.strategy]
        return picks

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # Timed region: K steps, tracing each kernel launch on its stream.
    ctx.trace(True)
    clocks = ClockSampler()
    clocks.start()
    per_variant = []
    barrier(world)
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    picks = {}
    for _ in range(args.steps):
        picks = step(per_variant)
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ctx.trace(False)
    trace = ctx.trace_collect()
    ms_total = t_start.elapsed_time(t_end)
    ms_total = max_over_ranks(world, ms_total)
    keys_per_step = len(VARIANTS) * n
    value = job_value(world, keys_per_step, args.steps, ms_total)

    # Per-variant p50 / p99 and per-kernel totals.
    import collections
    vt = collections.defaultdict(list)
    for v, a, b in per_variant:
        vt[v].append(a.elapsed_time(b))
    per_strategy = {}
    for v in VARIANTS:
        xs = sorted(vt[v])
        p50 = statistics.median(xs)
        p99 = xs[min(len(xs) - 1, int(round(0.99 * (len(xs) - 1))))]
        per_strategy[v] = {"strategy": picks[v], "ms_p50": round(p50, 4), "ms_p99": round(p99, 4),
                           "gkeys_s_p50": round(n / (p50 / 1e3) / 1e9, 3)}
        if picks[v] == "IDENTITY":
            per_strategy[v]["note"] = ("input found in order by the min/max pass and returned as "
                                       "a copy (GB300 profile's presorted rule)")
        if picks[v] == "REVERSE":
            per_strategy[v]["note"] = ("input found in reverse order by the min/max pass and "
                                       "returned reversed (GB300 profile's presorted rule)")
    presorted = ("IDENTITY", "REVERSE")
    ms_sorting = sum(statistics.median(vt[v]) for v in VARIANTS if picks[v] not in presorted)
    n_sorting = sum(1 for v in VARIANTS if picks[v] not in presorted)
    kt = collections.defaultdict(lambda: [0, 0.0, 0])
    for name, items, ms, _ in trace:
        kt[name][0] += 1
        kt[name][1] += ms
        kt[name][2] += items
    peak, peak_kind = measured_peaks()
    dom = max(kt.items(), key=lambda kv: kv[1][1])[0]
    launches, ms_k, items_k = kt[dom]
    avg_ms = ms_k / launches
    items_per_launch = items_k / launches
    bytes_per_launch = algo_bytes_per_item(dom, 4, 0) * items_per_launch
    achieved = bytes_per_launch / (avg_ms / 1e3) / 1e9
    kernels = kernel_table(kt, peak)

    # End to end through the public API with host buffers: every step copies
    # each input from pinned host memory to the device, sorts it and copies the
    # sorted keys back (ahs_sort_host overlaps the copies of neighbouring
    # arrays with the sort in between).
    host_in = [torch.empty(n, dtype=torch.int32, pin_memory=True) for _ in VARIANTS]
    host_out = [torch.empty(n, dtype=torch.int32, pin_memory=True) for _ in VARIANTS]
    for h, v in zip(host_in, VARIANTS):
        h.copy_(inputs[v])
    torch.cuda.synchronize()

    def e2e_step():
        # One C-ABI call (ahs_sort_host) per step; consecutive steps overlap
        # (the next step's first copy in runs during this step's last copy
        # out); the timed region ends after ahs_wait_host.
        ctx.sort_host(host_in, host_out, key_type=ahs.AHS_U32, stream=stream, wait=False)

    for _ in range(max(2, args.warmup)):
        e2e_step()
    torch.cuda.synchronize()
    barrier(world)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    ctx.wait_host(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(world, e0.elapsed_time(e1))
    e2e_value = job_value(world, keys_per_step, args.steps, e2e_ms)

    batched = served = cfg1 = cfg3 = None
    if not args.no_extras:
        cfg1 = run_config1(ctx, 100, stream)
        cfg3 = run_config3(ctx, 30, stream, peak)
        batched = run_batched(ctx, args.batch_segments, 10)
        served = [run_served(local, load, args.serve_seconds)
                  for load in args.serve_loads]

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        k, s, _ = oracle_sample_run(args.ref_sample)
        cpu = {"value": k / s / 1e9, "unit": "Gkeys/s", "cores": 1, "kind": "oracle",
               "sample": f"first {args.ref_sample} keys of each of the 6 arrays ({k} keys, {s:.1f} s)",
               "cpu_model": host_cpu_model(), "host_cores": os.cpu_count(),
               "std_sort_gkeys_s": std_sort_context(args.ref_sample)}
        if not args.no_extras:
            cpu["config4_all_cores"] = oracle_config4_all_cores(args.cpu_segments)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 4), "unit": "Gkeys/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms_total / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "config2 a-f: six uint32 arrays of n keys, AUTO pipeline, GB300 profile",
                       "n_per_array": n, "keys_per_step": keys_per_step, "picks": picks,
                       "l2": "inputs (1 GiB each) larger than the 129 MB L2; no flush",
                       "parallelism": f"replicas x{world}",
                       "host_cpus": f"{len(bound)} GPU-local" if bound else "unbound"},
            "per_strategy": per_strategy,
            "sorting_arrays_gkeys_s": round(n_sorting * n / (ms_sorting / 1e3) / 1e9, 3),
            "config1": cfg1,
            "config3": cfg3,
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1),
                         "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                         "peak_kind": peak_kind,
                         "traffic": ncu_traffic(dom, items_per_launch),
                         "algorithmic_bytes_per_launch": bytes_per_launch,
                         "avg_launch_ms": round(avg_ms, 4)},
            "kernels": kernels,
            "gpu_launches": len(trace),
            "e2e": {"value": round(e2e_value, 4), "unit": "Gkeys/s",
                    "h2d_bytes_per_step": keys_per_step * 4, "d2h_bytes_per_step": keys_per_step * 4},
            "clocks": clk,
            "cpu_baseline": cpu,
            "batched": batched,
            "served": served,
        }
        print(json.dumps(line), flush=True)
    ctx.close()


def host_cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the CPU baseline."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def percentiles(xs):
    xs = sorted(xs)
    return statistics.median(xs), xs[min(len(xs) - 1, int(round(0.99 * (len(xs) - 1))))]


def timed_calls(fn, reps: int, stream):
    """Device time of each of `reps` calls of fn(), CUDA events on `stream`."""
    import torch
    times = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
    return times


def run_config1(ctx, reps: int, stream):
    """Config 1: 2^20 uint32 keys uniform in [0, 255] (seed 0), AUTO pipeline
    (features -> selector -> counting sort).  Latency-bound and L2-resident:
    reported in microseconds with p50 / p99 over `reps` calls."""
    import torch
    import paper_2506_20677_gb300 as ahs
    from gen import device as gdev
    keys = gdev.config1()
    out = torch.empty_like(keys)
    n = keys.numel()
    call = lambda: ctx.sort(keys, out=out, key_type=ahs.AHS_U32, stream=stream)
    for _ in range(5):
        r = call()
    torch.cuda.synchronize()
    p50, p99 = percentiles(timed_calls(call, reps, stream))
    return {"n": n, "strategy": ahs.STRATEGY_NAMES[r.strategy], "us_p50": round(1e3 * p50, 1),
            "us_p99": round(1e3 * p99, 1), "gkeys_s_p50": round(n / (p50 / 1e3) / 1e9, 3),
            "calls": reps, "note": "latency-bound, L2-resident (12 MiB of algorithmic traffic)"}


def run_config3(ctx, reps: int, stream, peak: float):
    """Config 3: 2^27 uint64 timestamp-ramp keys (5% replaced by uniform draws
    over the ramp's range) with a uint32 payload = original index, forced
    RADIX (stable LSD digit passes).  p50 / p99 and per-kernel fractions of
    the HBM peak; the path's fraction is against the minimum bytes the paper's
    radix needs with 11-bit digits (16 + 4 x 24 = 112 B/key, Eq. 4 with r = 11)."""
    import collections
    import torch
    import paper_2506_20677_gb300 as ahs
    from gen import device as gdev
    keys, vals = gdev.config3()
    n = keys.numel()
    out, vout = torch.empty_like(keys), torch.empty_like(vals)
    call = lambda: ctx.sort(keys, vals=vals, out=out, vals_out=vout, force=ahs.AHS_RADIX,
                            key_type=ahs.AHS_U64, stream=stream)
    for _ in range(3):
        r = call()
    torch.cuda.synchronize()
    ctx.trace(True)
    times = timed_calls(call, reps, stream)
    ctx.trace(False)
    trace = ctx.trace_collect()
    p50, p99 = percentiles(times)
    kt = collections.defaultdict(lambda: [0, 0.0, 0])
    for name, items, ms, _ in trace:
        kt[name][0] += 1
        kt[name][1] += ms
        kt[name][2] += items
    path_bytes = 112 * n
    res = {"n": n, "strategy": ahs.STRATEGY_NAMES[r.strategy], "passes": int(r.info.passes),
           "ms_p50": round(p50, 4), "ms_p99": round(p99, 4),
           "gkeys_s_p50": round(n / (p50 / 1e3) / 1e9, 3),
           "path_frac_112B": round(path_bytes / (p50 / 1e3) / 1e9 / peak, 4),
           "kernels": kernel_table(kt, peak, 8, 4)}
    del keys, vals, out, vout
    torch.cuda.empty_cache()
    return res


def run_batched(ctx, n_seg: int, steps: int, per_array: bool = True):
    """Config 4's recipe with n_seg segments: the batched call against a loop
    of per-array calls on the same stream, same keys."""
    import torch
    import paper_2506_20677_gb300 as ahs
    from gen import device as gdev
    keys, offs, lengths, types = gdev.config4(n_seg=n_seg)
    out = torch.empty_like(keys)
    total = int(offs[-1])
    offs_l = offs.tolist()
    ctx.sort_batch(keys, offs_l, out=out, key_type=ahs.AHS_U32)        # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    info = None
    for _ in range(steps):
        e0.record()
        _, _, info = ctx.sort_batch(keys, offs_l, out=out, key_type=ahs.AHS_U32)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    # one more call, traced: per-kernel device time and the host gaps between launches
    import collections
    ctx.trace(True)
    e0.record()
    ctx.sort_batch(keys, offs_l, out=out, key_type=ahs.AHS_U32)
    e1.record()
    torch.cuda.synchronize()
    ctx.trace(False)
    tr = ctx.trace_collect()
    kt = collections.defaultdict(lambda: [0, 0.0, 0])
    for name, items, ms_, _ in tr:
        kt[name][0] += 1
        kt[name][1] += ms_
        kt[name][2] += items
    busy = sum(x[1] for x in kt.values())
    # the largest host gaps between consecutive launches of the traced call
    ev = sorted(tr, key=lambda e: e[3])
    gaps = []
    for a, b in zip(ev, ev[1:]):
        g = b[3] - (a[3] + a[2])
        if g > 0.2:
            gaps.append((round(g, 3), a[0], b[0]))
    gaps.sort(reverse=True)
    times_sorted = sorted(times)
    res = {"segments": n_seg, "keys": total, "batched_ms_p50": round(statistics.median(times), 3),
           "batched_ms_p99": round(times_sorted[min(len(times_sorted) - 1, int(0.99 * len(times_sorted)))], 3),
           "batched_gkeys_s": round(total / (statistics.median(times) / 1e3) / 1e9, 3),
           "seg_per_strategy": {ahs.STRATEGY_NAMES[i]: int(info.seg_per_strategy[i]) for i in range(1, 6)},
           "traced_call_ms": round(e0.elapsed_time(e1), 3), "kernel_ms": round(busy, 3),
           "host_ms": {"features": round(info.ms_features, 3), "select": round(info.ms_select, 3),
                       "sort": round(info.ms_sort, 3)},
           "kernels": {k: {"launches": c, "ms": round(m, 3)} for k, (c, m, _) in
                       sorted(kt.items(), key=lambda kv: -kv[1][1])},
           "host_gaps_ms": gaps[:12]}
    if per_array:
        torch.cuda.synchronize()
        e0.record()
        for s in range(n_seg):
            b, e = offs_l[s], offs_l[s + 1]
            if e > b:
                ctx.sort(keys[b:e], out=out[b:e], key_type=ahs.AHS_U32)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        res["per_array_ms"] = round(ms, 3)
        res["per_array_gkeys_s"] = round(total / (ms / 1e3) / 1e9, 3)
        res["batched_over_per_array"] = round(ms / statistics.median(times), 2)
        # The served form on the same segments: every segment is one request,
        # all submitted at once (the offered load exceeds capacity), sorted
        # by the serving loop's continuous batching.
        sv = run_served_segments(ctx.device, keys, out, offs_l, n_seg)
        sv["served_over_per_array"] = round(sv["sustained_gkeys_s"] / res["per_array_gkeys_s"], 2)
        res["served_same_segments"] = sv
    del keys, out
    torch.cuda.empty_cache()
    return res


def run_served_segments(device: int, keys, out, offs_l, n_seg: int, budget: int = 64 << 30):
    """Config 4's segments as served requests, all submitted at t = 0 from the
    host: sustained Gkeys/s (wall time from the first submission to the last
    completion) and latency percentiles."""
    import ctypes
    import torch
    import paper_2506_20677_gb300 as ahs
    ctx = ahs.Context(device)
    cfg = ahs.ahs_serve_config_t(budget, 1024, 100)
    ahs.check(ahs.lib.ahs_serve_start(ctx.handle, ctypes.byref(cfg)), "ahs_serve_start")
    base_in, base_out = keys.data_ptr(), out.data_ptr()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tickets = []
    for s_ in range(n_seg):
        b, e = offs_l[s_], offs_l[s_ + 1]
        if e == b:
            continue
        req = ahs.ahs_request_t()
        req.d_keys_in = base_in + 4 * b
        req.d_keys_out = base_out + 4 * b
        req.n = e - b
        req.type = ahs.AHS_U32
        tk = ctypes.c_uint64()
        ahs.check(ahs.lib.ahs_serve_submit(ctx.handle, ctypes.byref(req), ctypes.byref(tk)), "submit")
        tickets.append(tk.value)
    for tk in tickets:
        r = ahs.ahs_result_t()
        ahs.check(ahs.lib.ahs_serve_poll(ctx.handle, tk, 600000, ctypes.byref(r)), "poll")
        ahs.check(r.status, "served request")
    elapsed = time.perf_counter() - t0
    st = ahs.ahs_serve_stats_t()
    ahs.check(ahs.lib.ahs_serve_stats(ctx.handle, ctypes.byref(st)), "stats")
    ahs.check(ahs.lib.ahs_serve_stop(ctx.handle), "stop")
    ctx.close()
    return {"requests": len(tickets), "seconds": round(elapsed, 3),
            "sustained_gkeys_s": round(st.keys / elapsed / 1e9, 3),
            "p50_ms": round(st.p50_ms, 3), "p99_ms": round(st.p99_ms, 3),
            "batches": int(st.batches)}


def run_served(ctx_device: int, load_gkeys: float, seconds: float, seed: int = 5,
               pool: int = 48, max_keys: int = 10**8):
    """Config 5: Poisson arrivals of uint32 sort requests at an offered load
    in Gkeys/s; request r has a log-uniform size in [10^3, max_keys] and a
    config-4 shape, and its keys are generated by the library on the device
    from (seed 5, r) (AHS_REQ_GENERATE) into one of `pool` output buffers;
    64 GB admission budget.  Against it: the first `pool` requests sorted
    serially one by one (device time of ahs_sort alone)."""
    import ctypes
    import torch
    import numpy as np
    import paper_2506_20677_gb300 as ahs
    from gen import device as gdev
    from gen import host as gh
    rng = np.random.default_rng(seed)
    n_max = 1 << 18
    sizes = gh.log_uniform_lengths(n_max, seed, 7, 1000, max_keys)
    kinds = gh.below32(gh.draws(seed, 8, 0, n_max), 4).astype(np.int64)
    outs = [torch.empty(max_keys, dtype=torch.int32, device="cuda") for _ in range(pool)]
    torch.cuda.synchronize()
    mean = float(np.mean(sizes))
    rate = load_gkeys * 1e9 / mean                       # requests per second
    ctx = ahs.Context(ctx_device)
    cfg = ahs.ahs_serve_config_t(64 << 30, 256, 100)
    ahs.check(ahs.lib.ahs_serve_start(ctx.handle, ctypes.byref(cfg)), "ahs_serve_start")
    busy = [False] * pool
    pending = []
    t_start = time.perf_counter()
    t_next = t_start
    submitted = skipped = 0
    while True:
        now = time.perf_counter()
        if now - t_start >= seconds or submitted >= n_max:
            break
        still = []
        for tk, i in pending:
            r = ahs.ahs_result_t()
            if ahs.lib.ahs_serve_poll(ctx.handle, tk, 0, ctypes.byref(r)) == ahs.AHS_OK:
                ahs.check(r.status, "served request")
                busy[i] = False
            else:
                still.append((tk, i))
        pending = still
        if now < t_next:
            time.sleep(min(t_next - now, 0.0005))
            continue
        t_next += rng.exponential(1.0 / rate)
        free = [i for i in range(pool) if not busy[i]]
        if not free:
            skipped += 1
            continue
        i = free[0]
        req = ahs.ahs_request_t()
        req.d_keys_out, req.n, req.type = outs[i].data_ptr(), int(sizes[submitted]), ahs.AHS_U32
        req.flags, req.gen_seed, req.gen_id = ahs.AHS_REQ_GENERATE, seed, submitted
        req.gen_kind = int(kinds[submitted])
        tk = ctypes.c_uint64()
        ahs.check(ahs.lib.ahs_serve_submit(ctx.handle, ctypes.byref(req), ctypes.byref(tk)), "submit")
        busy[i] = True
        pending.append((tk.value, i))
        submitted += 1
    for tk, i in pending:
        r = ahs.ahs_result_t()
        ahs.lib.ahs_serve_poll(ctx.handle, tk, 600000, ctypes.byref(r))
    elapsed = time.perf_counter() - t_start
    st = ahs.ahs_serve_stats_t()
    ahs.check(ahs.lib.ahs_serve_stats(ctx.handle, ctypes.byref(st)), "stats")
    ahs.check(ahs.lib.ahs_serve_stop(ctx.handle), "stop")
    del outs
    torch.cuda.empty_cache()
    # Serial per-request baselines over the first requests: (1) each request
    # generated on the device (the workload module's generators) and sorted
    # by ahs_sort, one at a time, wall clock -- the served form's work
    # without the loop; (2) the device time of ahs_sort alone on those keys.
    stream = torch.cuda.current_stream()
    n_ser = min(pool, max(submitted, 1))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    serial_keys = 0
    for rid in range(n_ser):
        keys = gdev.request_keys(seed, rid, int(kinds[rid]), int(sizes[rid]))
        ctx.sort(keys, out=keys, key_type=ahs.AHS_U32, stream=stream)
        torch.cuda.synchronize()
        serial_keys += int(sizes[rid])
        del keys
    serial_wall = serial_keys / (time.perf_counter() - t0) / 1e9
    serial_ms = 0.0
    for rid in range(n_ser):
        keys = gdev.request_keys(seed, rid, int(kinds[rid]), int(sizes[rid]))
        out = torch.empty_like(keys)
        ctx.sort(keys, out=out, key_type=ahs.AHS_U32, stream=stream)   # warm
        serial_ms += statistics.median(
            timed_calls(lambda: ctx.sort(keys, out=out, key_type=ahs.AHS_U32, stream=stream), 3, stream))
        del keys, out
    ctx.close()
    serial = serial_keys / (serial_ms / 1e3) / 1e9
    sustained = st.keys / elapsed / 1e9
    return {"offered_gkeys_s": load_gkeys, "seconds": round(elapsed, 2), "submitted": submitted,
            "dropped_no_free_buffer": skipped, "completed": int(st.completed),
            "sustained_gkeys_s": round(sustained, 3),
            "p50_ms": round(st.p50_ms, 3), "p99_ms": round(st.p99_ms, 3),
            "batches": int(st.batches), "peak_reserved_gb": round(st.peak_reserved_bytes / 2**30, 2),
            "serial_per_request_gkeys_s": round(serial_wall, 3),
            "serial_sort_device_gkeys_s": round(serial, 3),
            "served_over_serial": round(sustained / serial_wall, 3),
            "requests": "log-uniform [1e3, %d] keys, config-4 shapes, keys generated by the library "
                        "per (seed %d, request id); %d output buffers" % (max_keys, seed, pool)}


def run_case(args, local):
    """One workload array with one (possibly forced) strategy: per-kernel
    device times from the library trace.  Used for per-strategy rooflines and
    as the small case under ncu."""
    import torch
    torch.cuda.set_device(local)
    import paper_2506_20677_gb300 as ahs
    from gen import device as gdev
    force = {"auto": ahs.AHS_AUTO, "counting": ahs.AHS_COUNTING, "radix": ahs.AHS_RADIX,
             "general": ahs.AHS_GENERAL}[args.force]
    if args.case == "3":
        keys, vals = gdev.config3(args.n)
        kt, w, v = ahs.AHS_U64, 8, 4
    else:
        keys, vals = gdev.config2(args.case, args.n), None
        kt, w, v = ahs.AHS_U32, 4, 0
    out = torch.empty_like(keys)
    vout = torch.empty_like(vals) if vals is not None else None
    ctx = ahs.Context(local, tuning_path=args.tuning if args.tuning else "shipped")
    for _ in range(args.warmup):
        ctx.sort(keys, vals=vals, out=out, vals_out=vout, force=force, key_type=kt)
    torch.cuda.synchronize()
    ctx.trace(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        r = ctx.sort(keys, vals=vals, out=out, vals_out=vout, force=force, key_type=kt)
    e1.record()
    torch.cuda.synchronize()
    trace = ctx.trace_collect()
    ms = e0.elapsed_time(e1) / args.steps
    peak, kind = measured_peaks()
    import collections
    kt_ = collections.defaultdict(lambda: [0, 0.0, 0])
    for name, items, t, _ in trace:
        kt_[name][0] += 1
        kt_[name][1] += t
        kt_[name][2] += items
    kernels = {}
    for name, (c, t, items) in sorted(kt_.items(), key=lambda kv: -kv[1][1]):
        b = algo_bytes_per_item(name, w, v) * items / c
        kernels[name] = {"launches": c, "avg_ms": round(t / c, 4),
                         "gbs": round(b / (t / c / 1e3) / 1e9, 1) if b else None,
                         "frac": round(b / (t / c / 1e3) / 1e9 / peak, 4) if b else None}
    line = {"case": args.case, "force": args.force, "n": args.n,
            "strategy": ahs.STRATEGY_NAMES[r.strategy], "ms_per_sort": round(ms, 4),
            "gkeys_s": round(args.n / (ms / 1e3) / 1e9, 3), "peak_gbs": peak,
            "peak_kind": kind, "kernels": kernels}
    if args.launches:
        # every launch of the last call: kernel, keys, device ms, start offset
        per = len(trace) // max(1, args.steps)
        line["last_call"] = [(k, it, round(t, 4), round(s0, 4)) for k, it, t, s0 in trace[-per:]]
    print(json.dumps(line), flush=True)
    ctx.close()


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--n", type=int, default=1 << 28, help="keys per array (default 2^28)")
    p.add_argument("--ref-sample", type=int, default=1 << 22,
                   help="keys per array the CPU oracle sorts")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--case", choices=list(VARIANTS) + ["3"], default=None,
                   help="diagnostic: one array of config 2 (a-f) or config 3, see --force")
    p.add_argument("--force", choices=["auto", "counting", "radix", "general"], default="auto")
    p.add_argument("--no-extras", action="store_true", help="skip the batched and served sections")
    p.add_argument("--launches", action="store_true", help="with --case: list the last call's launches")
    p.add_argument("--tuning", default=None, help="with --case: tuned-shape table to load")
    p.add_argument("--batch-segments", type=int, default=100_000,
                   help="segments of the config-4 batch in the default run")
    p.add_argument("--serve-loads", type=float, nargs="+", default=[2.0, 5.0, 10.0, 40.0],
                   help="offered Gkeys/s of the served runs (the last one above capacity)")
    p.add_argument("--serve-seconds", type=float, default=6.0)
    p.add_argument("--cpu-segments", type=int, default=2000,
                   help="config-4 segments the all-core oracle baseline sorts")
    p.add_argument("--batch", action="store_true", help="config 4 at full size: batched vs per-array")
    p.add_argument("--serve", action="store_true", help="config 5: offered loads 2/5/10 Gkeys/s")
    args = p.parse_args()
    world, rank, local = dist_setup()
    if args.case is not None:
        run_case(args, local)
        return
    if args.batch or args.serve:
        import torch
        torch.cuda.set_device(local)
        import paper_2506_20677_gb300 as ahs
        out = {}
        if args.batch:
            ctx = ahs.Context(local)
            out["batched"] = run_batched(ctx, 100_000, args.steps)
            ctx.close()
        if args.serve:
            out["served"] = [run_served(local, load, args.serve_seconds) for load in args.serve_loads]
        print(json.dumps(out), flush=True)
        return
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
