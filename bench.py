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
        "sample_scatter": 2 * (w + v), "bucket_sort_1k": 2 * (w + v),
        "bucket_sort_4k": 2 * (w + v), "bucket_sort_8k": 2 * (w + v),
        "blocksort_single": 2 * (w + v), "copy": 8,
    }
    return table.get(kernel, 0.0)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d.get("hbm_gbs"), "measured"
    return 6800.0, "fallback"


def kernel_source_hash(kernel: str):
    files = {"radix": "radix.cu", "sample": "samplesort.cu", "bucket": "blocksort.cuh",
             "features": "features.cu", "counting": "counting.cu", "copy": "counting.cu"}
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


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, x: float) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
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
    value = world * keys_per_step * args.steps / (ms_total / 1e3) / 1e9

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
    kt = collections.defaultdict(lambda: [0, 0.0, 0])
    for name, items, ms in trace:
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
    kernels = {k: {"launches": c, "ms": round(m, 3), "share": round(m / sum(x[1] for x in kt.values()), 4)}
               for k, (c, m, _) in sorted(kt.items(), key=lambda kv: -kv[1][1])}

    # End to end through the public API with host buffers: H2D of each input,
    # the sort, D2H of each sorted output, every step.
    host_in = {v: torch.empty(n, dtype=torch.int32, pin_memory=True) for v in VARIANTS}
    for v in VARIANTS:
        host_in[v].copy_(inputs[v])
    host_out = torch.empty(n, dtype=torch.int32, pin_memory=True)
    dev_in = torch.empty(n, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()

    def e2e_step():
        for v in VARIANTS:
            dev_in.copy_(host_in[v], non_blocking=True)
            ctx.sort(dev_in, out=out, key_type=ahs.AHS_U32, stream=stream)
            host_out.copy_(out, non_blocking=True)

    for _ in range(max(1, args.warmup // 2)):
        e2e_step()
    torch.cuda.synchronize()
    barrier(world)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(world, e0.elapsed_time(e1))
    e2e_value = world * keys_per_step * args.steps / (e2e_ms / 1e3) / 1e9

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        k, s, _ = oracle_sample_run(args.ref_sample)
        cpu = {"value": k / s / 1e9, "unit": "Gkeys/s", "cores": 1, "kind": "oracle",
               "sample": f"first {args.ref_sample} keys of each of the 6 arrays ({k} keys, {s:.1f} s)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 4), "unit": "Gkeys/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms_total / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "config2 a-f: six uint32 arrays of n keys, AUTO pipeline, GB300 profile",
                       "n_per_array": n, "keys_per_step": keys_per_step, "picks": picks,
                       "l2": "inputs (1 GiB each) larger than the 129 MB L2; no flush",
                       "parallelism": f"replicas x{world}"},
            "per_strategy": per_strategy,
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
        }
        print(json.dumps(line), flush=True)
    ctx.close()


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
    ctx = ahs.Context(local)
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
    for name, items, t in trace:
        kt_[name][0] += 1
        kt_[name][1] += t
        kt_[name][2] += items
    kernels = {}
    for name, (c, t, items) in sorted(kt_.items(), key=lambda kv: -kv[1][1]):
        b = algo_bytes_per_item(name, w, v) * items / c
        kernels[name] = {"launches": c, "avg_ms": round(t / c, 4),
                         "gbs": round(b / (t / c / 1e3) / 1e9, 1) if b else None,
                         "frac": round(b / (t / c / 1e3) / 1e9 / peak, 4) if b else None}
    print(json.dumps({"case": args.case, "force": args.force, "n": args.n,
                      "strategy": ahs.STRATEGY_NAMES[r.strategy], "ms_per_sort": round(ms, 4),
                      "gkeys_s": round(args.n / (ms / 1e3) / 1e9, 3), "peak_gbs": peak,
                      "peak_kind": kind, "kernels": kernels}), flush=True)
    ctx.close()


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--n", type=int, default=1 << 28, help="keys per array (default 2^28)")
    p.add_argument("--ref-sample", type=int, default=1 << 22,
                   help="keys per array the CPU oracle sorts")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--case", choices=list(VARIANTS) + ["3"], default=None,
                   help="diagnostic: one array of config 2 (a-f) or config 3, see --force")
    p.add_argument("--force", choices=["auto", "counting", "radix", "general"], default="auto")
    args = p.parse_args()
    world, rank, local = dist_setup()
    if args.case is not None:
        run_case(args, local)
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
