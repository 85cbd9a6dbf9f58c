"""Autotuner: measure kernel shapes on this GPU and write the tuned-shape table.

The table (selector/tuning_gb300.txt, loaded by every Context) holds
  - the largest digit width r of the stable LSD radix passes, per key width,
    payload and key range: Eq. 4 gives d = ceil(D / r) passes over a D-bit
    range, and wider digits trade fewer passes for larger per-tile counters,
    so r is chosen by time among 4, 8, 9, 10 and 11 bits;
  - the batched form's one-block cutoff: segments up to that many keys are
    sorted by one CTA whatever strategy the selector picked.
Each candidate is timed with CUDA events on the launching stream (median of
`reps` calls after warm-up) on seeded uniform keys of the given range.

    python -m paper_2506_20677_gb300.autotune [--n 33554432] [--out path]
"""
from __future__ import annotations

import argparse
import os
import statistics
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_OUT = os.path.join(HERE, "selector", "tuning_gb300.txt")
WIDTHS = (4, 8, 9, 10, 11)
SPANS = {4: (12, 16, 20, 24, 28, 32), 8: (16, 24, 32, 36, 40, 48, 56, 64)}
CUTOFFS = (0, 1024, 2048, 4096, 8192)
MARGIN = 0.03   # a candidate must beat the default by more than this to be chosen


def _write_table(path, radix_rows, cutoff):
    with open(path, "w") as fh:
        fh.write("ahs-tuning 1\n")
        for kb, pay, span, bits in radix_rows:
            fh.write(f"radix_bits {kb} {pay} {span} {bits}\n")
        fh.write(f"batch_small_cutoff {cutoff}\n")


def _time(fn, reps, stream):
    import torch
    for _ in range(2):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def tune_radix(ctx, n, n_kv, reps, log):
    """Best digit width per (key bytes, payload, span bits); key-value cases
    at n_kv keys (the stable passes matter most for large key-value arrays)."""
    import torch
    import paper_2506_20677_gb300 as ahs
    stream = torch.cuda.current_stream()
    rows = []
    tmp = tempfile.mkdtemp(prefix="ahs_tune_")
    g = torch.Generator(device="cuda")
    for kb in (4, 8):
        dt = torch.int32 if kb == 4 else torch.int64
        kt = ahs.AHS_U32 if kb == 4 else ahs.AHS_U64
        for span in SPANS[kb]:
            g.manual_seed(1000 * kb + span)
            if kb == 4:
                hi = (1 << span) if span < 32 else (1 << 32)
                keys = (torch.randint(0, hi, (n,), device="cuda", dtype=torch.int64, generator=g)
                        .to(torch.int32) if span < 32 else
                        torch.randint(-2**31, 2**31, (n,), device="cuda", dtype=torch.int64,
                                      generator=g).to(torch.int32))
            else:
                lo = -(1 << 63) if span == 64 else 0
                hi = (1 << 63) - 1 if span == 64 else (1 << span) - 1
                keys = torch.randint(lo, hi, (n,), device="cuda", dtype=torch.int64, generator=g)
            for pay in (0, 1):
                m = n_kv if pay else n
                k_m = keys if m == n else torch.cat([keys] * (m // n) + [keys[: m % n]])
                vals = torch.arange(m, device="cuda", dtype=torch.int32)
                out, vout = torch.empty_like(k_m), torch.empty_like(vals)
                best = None
                times = {}
                for r in WIDTHS:
                    path = os.path.join(tmp, f"t{kb}_{span}_{pay}_{r}.txt")
                    _write_table(path, [(kb, pay, 64, r)], 0)
                    ctx.load_tuning(path)
                    v, vo = (vals, vout) if pay else (None, None)
                    ms = _time(lambda: ctx.sort(k_m, vals=v, out=out, vals_out=vo,
                                                force=ahs.AHS_RADIX, key_type=kt, stream=stream),
                               reps, stream)
                    log(f"radix kb={kb} payload={pay} span_bits={span} r={r}: {ms:.4f} ms")
                    times[r] = ms
                    if best is None or ms < best[1]:
                        best = (r, ms)
                # Base 256 (the default path) unless a width beats it clearly.
                if times[8] <= (1.0 + MARGIN) * best[1]:
                    best = (8, times[8])
                rows.append((kb, pay, span, best[0]))
                del k_m, vals, out, vout
            del keys
            torch.cuda.empty_cache()
    ctx.load_tuning(None)
    return rows


def tune_batch_cutoff(ctx, n_seg, reps, log):
    import torch
    import paper_2506_20677_gb300 as ahs
    from gen import device as gdev
    keys, offs, _, _ = gdev.config4(n_seg=n_seg)
    out = torch.empty_like(keys)
    offs_l = offs.tolist()
    stream = torch.cuda.current_stream()
    tmp = tempfile.mkdtemp(prefix="ahs_tune_")
    best = None
    for c in CUTOFFS:
        path = os.path.join(tmp, f"c{c}.txt")
        _write_table(path, [], c)
        ctx.load_tuning(path)
        ms = _time(lambda: ctx.sort_batch(keys, offs_l, out=out, key_type=ahs.AHS_U32), reps, stream)
        log(f"batch cutoff={c}: {ms:.3f} ms ({n_seg} segments)")
        if best is None or ms < best[1] * (1.0 - MARGIN) or (c == 0 and ms <= best[1]):
            best = (c, ms)
    ctx.load_tuning(None)
    del keys, out
    torch.cuda.empty_cache()
    return best[0]


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--n", type=int, default=1 << 25, help="keys per keys-only radix timing")
    p.add_argument("--n-kv", type=int, default=1 << 27, help="keys per key-value radix timing")
    p.add_argument("--reps", type=int, default=5)
    p.add_argument("--segments", type=int, default=5000, help="config-4 segments for the cutoff")
    p.add_argument("--out", default=DEFAULT_OUT)
    args = p.parse_args(argv)
    sys.path.insert(0, os.path.dirname(HERE))
    import torch
    import paper_2506_20677_gb300 as ahs
    torch.cuda.set_device(0)
    lines = []

    def log(s):
        print(s, flush=True)
        lines.append(s)

    with ahs.Context(0, tuning_path=None) as ctx:
        rows = tune_radix(ctx, args.n, args.n_kv, args.reps, log)
        cutoff = tune_batch_cutoff(ctx, args.segments, args.reps, log)
    name = torch.cuda.get_device_name(0)
    with open(args.out, "w") as fh:
        fh.write("ahs-tuning 1\n")
        fh.write(f"# measured by paper_2506_20677_gb300/autotune.py on {name}: stable LSD radix on\n")
        fh.write(f"# {args.n} uniform keys per range ({args.n_kv} with a payload), median of "
                 f"{args.reps} CUDA-event timings per\n")
        fh.write("# candidate digit width; batched cutoff on the first "
                 f"{args.segments} segments of config 4.\n")
        for kb, pay, span, bits in rows:
            fh.write(f"radix_bits {kb} {pay} {span} {bits}\n")
        fh.write(f"batch_small_cutoff {cutoff}\n")
        for s in lines:
            fh.write(f"# {s}\n")
    print(f"wrote {args.out}")


if __name__ == "__main__":
    main()
