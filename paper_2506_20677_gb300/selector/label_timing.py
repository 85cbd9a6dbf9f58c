"""Label synthetic inputs with the fastest strategy on this GPU.

For each synthetic set (size n, range k, distribution, key type, payload) the
features are taken with ahs_features and every strategy that can run on the
input (counting only for k <= 2^16, the one-block sort only up to its
capacity) is timed with CUDA events, median of `reps` runs; the label is the
fastest.  This is the training protocol of the learned selector of Section
III-H, with GB300 timings instead of the paper's CPU timings.

    python -m paper_2506_20677_gb300.selector.label_timing --out labels.json

Inputs are seeded and synthetic: uniform over ranges from 10 to 2^64, Zipf
over a few hundred to thousands of values spread over wide ranges, Gaussian
N(0, k/4) (the paper's Gaussian sets), timestamp-like ramps, and presorted /
nearly sorted arrays.
"""
from __future__ import annotations

import argparse
import json
import math
import statistics

import numpy as np


def make_input(rng, torch, n, kind, key64):
    dt = torch.int64 if key64 else torch.int32
    g = torch.Generator(device="cuda")
    g.manual_seed(int(rng.integers(0, 2**31)))
    if kind == "uniform":
        bits = int(rng.integers(3, 64 if key64 else 32))
        hi = 1 << bits
        x = torch.randint(0, min(hi, 2**62), (n,), generator=g, device="cuda", dtype=torch.int64)
    elif kind == "zipf":
        m = int(rng.integers(16, 4096))
        vals = torch.randint(0, 2**62 if key64 else 2**31, (m,), generator=g, device="cuda",
                             dtype=torch.int64)
        p = 1.0 / torch.arange(1, m + 1, device="cuda", dtype=torch.float64) ** float(rng.uniform(0.8, 1.6))
        idx = torch.multinomial(p / p.sum(), n, replacement=True, generator=g)
        x = vals[idx]
    elif kind == "gauss":
        k = 10 ** float(rng.uniform(1, 9))
        x = (torch.randn(n, generator=g, device="cuda", dtype=torch.float64) * math.sqrt(k / 4)).round()
        x = (x - x.min()).to(torch.int64)
    elif kind == "ramp":
        steps = torch.randint(0, 1001, (n,), generator=g, device="cuda", dtype=torch.int64)
        x = torch.cumsum(steps, 0)
        rep = torch.rand(n, generator=g, device="cuda") < 0.05
        x[rep] = torch.randint(0, int(x[-1].item()) + 1, (int(rep.sum().item()),), generator=g,
                               device="cuda", dtype=torch.int64)
    else:   # nearly sorted
        x = torch.sort(torch.randint(0, 2**31, (n,), generator=g, device="cuda", dtype=torch.int64)).values
        sw = max(1, n // 100)
        i = torch.randint(0, n, (sw,), generator=g, device="cuda")
        j = torch.randint(0, n, (sw,), generator=g, device="cuda")
        x[i], x[j] = x[j].clone(), x[i].clone()
    if not key64:
        x = (x & 0xFFFFFFFF).to(torch.int64)
        x = torch.where(x >= 2**31, x - 2**32, x).to(torch.int32)
    return x.to(dt).contiguous()


def time_strategy(ctx, ahs, torch, keys, vals, force, kt, reps):
    out = torch.empty_like(keys)
    vout = torch.empty_like(vals) if vals is not None else None
    ctx.sort(keys, vals=vals, out=out, vals_out=vout, force=force, key_type=kt)   # warm-up
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.sort(keys, vals=vals, out=out, vals_out=vout, force=force, key_type=kt)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def main():
    import torch
    import paper_2506_20677_gb300 as ahs
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--sets", type=int, default=360)
    ap.add_argument("--max-log2n", type=int, default=26)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--seed", type=int, default=2506)
    a = ap.parse_args()
    rng = np.random.default_rng(a.seed)
    rows = []
    with ahs.Context(0) as ctx:
        for s in range(a.sets):
            n = int(2 ** rng.uniform(10, a.max_log2n))
            kind = ["uniform", "zipf", "gauss", "ramp", "nearly"][s % 5]
            key64 = bool(rng.random() < 0.3)
            payload = bool(rng.random() < 0.25)
            keys = make_input(rng, torch, n, kind, key64)
            kt = ahs.AHS_I64 if key64 else ahs.AHS_I32
            vals = torch.arange(n, dtype=torch.int32, device="cuda") if payload else None
            f = ctx.features(keys, key_type=kt)
            cand = [ahs.AHS_RADIX, ahs.AHS_GENERAL]
            if f.span < 65536:
                cand.append(ahs.AHS_COUNTING)
            if n <= ahs.lib.ahs_small_capacity(kt, int(payload)):
                cand.append(ahs.AHS_SMALL)
            times = {}
            for c in cand:
                times[ahs.STRATEGY_NAMES[c]] = time_strategy(ctx, ahs, torch, keys, vals, c, kt, a.reps)
            best = min(times, key=times.get)
            rows.append({"n": n, "span": int(f.span), "entropy_bits": f.entropy_bits,
                         "entropy_norm": f.entropy_norm, "nbins": int(f.nbins),
                         "key_bytes": 8 if key64 else 4, "payload": int(payload), "kind": kind,
                         "times_ms": times, "label": best})
            if s % 40 == 0:
                print(s, n, kind, best, {k: round(v, 3) for k, v in times.items()}, flush=True)
    with open(a.out, "w") as fh:
        json.dump({"protocol": "median of %d CUDA-event timings per forced strategy" % a.reps,
                   "device": torch.cuda.get_device_name(0), "rows": rows}, fh, indent=0)
    print("wrote", len(rows), "rows to", a.out)


if __name__ == "__main__":
    main()
