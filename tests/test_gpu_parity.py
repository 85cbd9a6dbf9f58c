"""GPU parity: the CUDA path through the C ABI against the oracle.

Keys and payload permutations are compared bit for bit; the entropy within
1e-9 relative (1e-12 absolute near zero): both sides sum -p log2 p in fp64
over the same integer counts, only the summation order differs.
"""
import math

import numpy as np
import pytest

from gpu_util import check_sorted_permutation, check_stable_kv, dev, host, key_type

pytestmark = pytest.mark.gpu

ENT_REL, ENT_ABS = 1e-9, 1e-12


@pytest.fixture(scope="module")
def ahs():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    import paper_2506_20677_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(ahs):
    c = ahs.Context(0)
    yield c
    c.close()


def _gen(kind, n, dt, seed):
    rng = np.random.default_rng(seed)
    info = np.iinfo(dt)
    if kind == "uniform_full":
        return rng.integers(info.min, info.max, size=n, dtype=dt, endpoint=True)
    if kind == "small_range":
        return rng.integers(0, 300, size=n, dtype=dt) + dt(5 if info.min == 0 else -150)
    if kind == "k4096":
        return rng.integers(0, 4096, size=n, dtype=dt)
    if kind == "k65536":
        return rng.integers(0, 65536, size=n, dtype=dt)
    if kind == "zipf_wide":
        vals = rng.integers(info.min, info.max, size=64, dtype=dt, endpoint=True)
        p = 1.0 / np.arange(1, 65) ** 1.1
        return vals[rng.choice(64, size=n, p=p / p.sum())]
    if kind == "clustered":
        # 90% of the keys in a range narrower than one histogram bin (a heavy
        # bin holding many values), the rest spread over the whole type.
        lo = info.min // 2 + info.max // 2
        c = lo + rng.integers(0, 4096, size=n).astype(dt)
        wide = rng.integers(info.min, info.max, size=n, dtype=dt, endpoint=True)
        return np.where(rng.random(n) < 0.9, c, wide).astype(dt)
    if kind == "two_in_bin":
        # Two heavy values inside one bin, plus a spread of others.
        v0 = dt(info.max // 3)
        pick = rng.random(n)
        wide = rng.integers(info.min, info.max, size=n, dtype=dt, endpoint=True)
        return np.where(pick < 0.45, v0, np.where(pick < 0.9, dt(v0 + 3), wide)).astype(dt)
    if kind == "dup_spread":
        # About four copies of each of n/4 values spread over the whole type:
        # equal keys share a sub-bucket of the keys-only bucket sort.
        vals = rng.integers(info.min, info.max, size=max(n // 4, 1), dtype=dt, endpoint=True)
        return vals[rng.integers(0, len(vals), size=n)]
    if kind == "half_equal":
        # Half the keys one value, the rest within 2^20 above it: one
        # sub-bucket of the keys-only bucket sort holds far more keys than the
        # comparison rank takes, so the bucket falls back to LSD passes.
        v0 = dt(info.max // 2 + 1)
        spread = (v0 + rng.integers(0, 1 << 20, size=n)).astype(dt)
        return np.where(rng.random(n) < 0.5, v0, spread).astype(dt)
    if kind == "all_equal":
        return np.full(n, dt(7), dtype=dt)
    if kind == "extremes":
        return rng.choice(np.array([info.min, info.max, 0, 1], dtype=dt), size=n)
    if kind == "sorted":
        return np.sort(rng.integers(info.min, info.max, size=n, dtype=dt, endpoint=True))
    if kind == "reversed":
        return np.sort(rng.integers(info.min, info.max, size=n, dtype=dt, endpoint=True))[::-1].copy()
    raise ValueError(kind)


def _check_features(f, of):
    assert (f.n, f.min_bits, f.max_bits, f.span, f.hist_shift, f.nbins, f.descents) == \
        (of.n, of.min_bits, of.max_bits, of.span, of.shift, of.nbins, of.descents)
    assert math.isclose(f.entropy_bits, of.entropy, rel_tol=ENT_REL, abs_tol=ENT_ABS)
    assert math.isclose(f.entropy_norm, of.entropy_norm, rel_tol=ENT_REL, abs_tol=ENT_ABS)


DTS = [np.uint32, np.int32, np.uint64, np.int64]
SIZES = [1, 2, 3, 17, 20, 21, 33, 1000, 8191, 8192, 8193, 65537, 300_001]
KINDS = ["uniform_full", "small_range", "k65536", "zipf_wide", "all_equal", "extremes",
         "sorted", "reversed", "clustered"]


@pytest.mark.parametrize("dt", DTS, ids=lambda d: np.dtype(d).name)
@pytest.mark.parametrize("kind", KINDS)
def test_features(ctx, orc, dt, kind):
    for i, n in enumerate(SIZES):
        a = _gen(kind, n, dt, 100 + i)
        _check_features(ctx.features(dev(a), key_type=key_type(a)), orc.features(a))


def test_features_misaligned_and_large(ctx, orc):
    import torch
    rng = np.random.default_rng(5)
    base = rng.integers(0, 2**32, size=(1 << 22) + 7, dtype=np.uint32)
    t = dev(base)
    for off in range(4):
        a = base[off:]
        _check_features(ctx.features(t[off:], key_type=key_type(a)), orc.features(a))
    b = rng.integers(0, 2**64, size=(1 << 21) + 3, dtype=np.uint64)
    tb = dev(b)
    _check_features(ctx.features(tb[1:], key_type=key_type(b)), orc.features(b[1:]))


def _sort_case(ahs, ctx, orc, a, force, kv, inplace=False):
    import torch
    vals = np.arange(len(a), dtype=np.uint32) if kv else None
    ka = dev(a)
    va = dev(vals) if kv else None
    if inplace:
        r = ctx.sort(ka, vals=va, out=ka, vals_out=va, force=force, key_type=key_type(a))
    else:
        r = ctx.sort(ka, vals=va, force=force, key_type=key_type(a))
    torch.cuda.synchronize()
    ko = host(r.keys, a.dtype)
    if force == ahs.AHS_IDENTITY:
        assert np.array_equal(ko, a)
        return r
    ok, ov, _, _ = orc.sort(a, vals, force=orc.RADIX)
    assert np.array_equal(ko, ok)
    if kv:
        assert np.array_equal(host(r.vals, np.uint32), ov)
    return r


@pytest.mark.parametrize("kv", [False, True], ids=["keys", "kv"])
@pytest.mark.parametrize("dt", DTS, ids=lambda d: np.dtype(d).name)
def test_forced_radix(ahs, ctx, orc, dt, kv):
    for i, n in enumerate(SIZES + [(1 << 20) + 5]):
        for kind in ("uniform_full", "zipf_wide", "extremes", "k65536", "all_equal", "clustered",
                     "two_in_bin", "dup_spread"):
            r = _sort_case(ahs, ctx, orc, _gen(kind, n, dt, i), ahs.AHS_RADIX, kv)
            assert r.strategy == ahs.AHS_RADIX


@pytest.mark.parametrize("kv", [False, True], ids=["keys", "kv"])
@pytest.mark.parametrize("dt", DTS, ids=lambda d: np.dtype(d).name)
def test_forced_general(ahs, ctx, orc, dt, kv):
    for i, n in enumerate(SIZES + [(1 << 21) + 9]):
        for kind in ("uniform_full", "zipf_wide", "extremes", "sorted", "reversed", "all_equal",
                     "clustered", "two_in_bin", "dup_spread", "half_equal"):
            _sort_case(ahs, ctx, orc, _gen(kind, n, dt, 7 + i), ahs.AHS_GENERAL, kv)


@pytest.mark.parametrize("kv", [False, True], ids=["keys", "kv"])
@pytest.mark.parametrize("dt", DTS, ids=lambda d: np.dtype(d).name)
def test_forced_counting(ahs, ctx, orc, dt, kv):
    for i, n in enumerate(SIZES + [(1 << 20) + 3]):
        for kind in ("small_range", "k4096", "k65536", "all_equal"):
            _sort_case(ahs, ctx, orc, _gen(kind, n, dt, 30 + i), ahs.AHS_COUNTING, kv)


def test_counting_range_refused(ahs, ctx):
    a = np.array([0, 70000] * 50, dtype=np.uint32)
    with pytest.raises(ahs.AhsError) as e:
        ctx.sort(dev(a), force=ahs.AHS_COUNTING, key_type=ahs.AHS_U32)
    assert e.value.status == ahs.AHS_ERR_RANGE


@pytest.mark.parametrize("kv", [False, True], ids=["keys", "kv"])
@pytest.mark.parametrize("dt", DTS, ids=lambda d: np.dtype(d).name)
def test_forced_small(ahs, ctx, orc, dt, kv):
    cap = int(ahs.lib.ahs_small_capacity(key_type(np.zeros(1, dt)), int(kv)))
    for i, n in enumerate([1, 2, 5, 16, 20, 21, 31, 32, 33, 500, 1024, 1025, 4095, cap - 1, cap]):
        for kind in ("uniform_full", "small_range", "extremes", "all_equal", "reversed",
                     "dup_spread", "half_equal"):
            _sort_case(ahs, ctx, orc, _gen(kind, n, dt, 50 + i), ahs.AHS_SMALL, kv)
    with pytest.raises(ahs.AhsError):
        ctx.sort(dev(_gen("uniform_full", cap + 1, dt, 0)), force=ahs.AHS_SMALL,
                 key_type=key_type(np.zeros(1, dt)))


def test_identity_and_empty(ahs, ctx, orc):
    import torch
    a = _gen("uniform_full", 1001, np.uint64, 1)
    _sort_case(ahs, ctx, orc, a, ahs.AHS_IDENTITY, True)
    e = torch.empty(0, dtype=torch.int32, device="cuda")
    r = ctx.sort(e, key_type=ahs.AHS_U32)
    assert r.strategy == ahs.AHS_IDENTITY and r.keys.numel() == 0


@pytest.mark.parametrize("force", ["RADIX", "GENERAL", "COUNTING", "AUTO"])
def test_in_place(ahs, ctx, orc, force):
    """In place (output buffer = input buffer), keys only and with payload, on
    inputs whose histogram-guided levels finish buckets after one pass (heavy
    bins, clustered keys) as well as on uniform keys."""
    f = getattr(ahs, "AHS_" + force)
    for dt in (np.uint32, np.int64):
        kinds = ["k4096"] if force == "COUNTING" else ["uniform_full", "zipf_wide", "clustered",
                                                        "two_in_bin", "half_equal"]
        for kind in kinds:
            for n in (100_003, 1 << 20):
                _sort_case(ahs, ctx, orc, _gen(kind, n, dt, n), f, True, inplace=True)
                _sort_case(ahs, ctx, orc, _gen(kind, n, dt, n + 1), f, False, inplace=True)


def test_misaligned_sort(ahs, ctx, orc):
    import torch
    rng = np.random.default_rng(9)
    base = rng.integers(0, 4096, size=(1 << 20) + 9, dtype=np.uint32)
    t = dev(base)
    for off in (1, 2, 3):
        for force in (ahs.AHS_COUNTING, ahs.AHS_RADIX, ahs.AHS_GENERAL):
            out = torch.empty(len(base) + 8, dtype=torch.int32, device="cuda")
            r = ctx.sort(t[off:], out=out[off + 1: off + 1 + len(base) - off], force=force,
                         key_type=ahs.AHS_U32)
            torch.cuda.synchronize()
            assert np.array_equal(host(r.keys, np.uint32), np.sort(base[off:])), (off, force)


def test_auto_picks_match_oracle(ahs, ctx, orc):
    g = ahs.profile_thresholds(ahs.AHS_SEL_GB300)
    prof = orc.Profile(g.n_t, g.k_t, g.k_max, g.h_max, bool(g.use_entropy), bool(g.sorted_identity))
    cases = [("small_range", 5000), ("k65536", 100_000), ("uniform_full", 50_000),
             ("zipf_wide", 200_000), ("sorted", 70_000), ("all_equal", 9000), ("uniform_full", 15),
             ("extremes", 100)]
    for kind, n in cases:
        for dt in DTS:
            a = _gen(kind, n, dt, n)
            r = ctx.sort(dev(a), key_type=key_type(a))
            import torch
            torch.cuda.synchronize()
            ko, _, chosen, _ = orc.sort(a, force=orc.AUTO, profile=prof)
            assert r.strategy == chosen, (kind, n, dt)
            assert np.array_equal(host(r.keys, a.dtype), ko)


def test_repeated_calls_reuse_context(ahs, ctx, orc):
    """Self-resetting counters and the reused workspace give identical results."""
    a = _gen("zipf_wide", 1 << 20, np.uint32, 77)
    first = None
    for force in (ahs.AHS_RADIX, ahs.AHS_GENERAL, ahs.AHS_RADIX, ahs.AHS_GENERAL):
        r = ctx.sort(dev(a), force=force, key_type=ahs.AHS_U32)
        out = host(r.keys, np.uint32)
        if first is None:
            first = out
        assert np.array_equal(out, first)


def test_sort_host_pipeline(ahs, ctx):
    """Host arrays through Context.sort_host (copies overlapped with sorts)."""
    import torch
    rng = np.random.default_rng(11)
    sizes = [300_001, 1, 0, 70_000, (1 << 20) + 3, 5]
    arrays = [rng.integers(0, 2**32, size=m, dtype=np.uint32) for m in sizes]
    arrays[3] = rng.integers(0, 4000, size=sizes[3], dtype=np.uint32)
    host_in = [torch.from_numpy(a.view(np.int32)).pin_memory() for a in arrays]
    host_out = [torch.empty_like(h).pin_memory() for h in host_in]
    for _ in range(2):   # the second call reuses the first one's streams and buffers
        picks = ctx.sort_host(host_in, host_out, key_type=ahs.AHS_U32)
        torch.cuda.synchronize()
        assert len(picks) == len(arrays)
        for a, o in zip(arrays, host_out):
            assert np.array_equal(o.numpy().view(np.uint32), np.sort(a))
    # Back-to-back calls that do not wait overlap; outputs are complete after
    # wait_host, each call's into its own outputs.
    outs = [[torch.empty_like(h).pin_memory() for h in host_in] for _ in range(3)]
    for o in outs:
        for t in o:
            t.fill_(-1)
        ctx.sort_host(host_in, o, key_type=ahs.AHS_U32, wait=False)
    ctx.wait_host()
    torch.cuda.synchronize()
    for o in outs:
        for a, t in zip(arrays, o):
            assert np.array_equal(t.numpy().view(np.uint32), np.sort(a))


def test_sort_host_payload_against_oracle(ahs, ctx, orc):
    """ahs_sort_host with a payload: every array in the unique stable order."""
    import torch
    rng = np.random.default_rng(12)
    arrays = [rng.integers(0, 3000 if i % 2 else 2**32, size=m, dtype=np.uint32)
              for i, m in enumerate([200_003, 17, (1 << 19) + 1])]
    vals = [np.arange(len(a), dtype=np.uint32)[::-1].copy() for a in arrays]
    hk = [torch.from_numpy(a.view(np.int32)).pin_memory() for a in arrays]
    hv = [torch.from_numpy(v.view(np.int32)).pin_memory() for v in vals]
    ok = [torch.empty_like(h).pin_memory() for h in hk]
    ov = [torch.empty_like(h).pin_memory() for h in hv]
    ctx.sort_host(hk, ok, key_type=ahs.AHS_U32, host_vals=hv, host_vals_out=ov)
    for a, v, k2, v2 in zip(arrays, vals, ok, ov):
        ek, ev = orc.merge_sort(a, v)
        assert np.array_equal(k2.numpy().view(np.uint32), ek)
        assert np.array_equal(v2.numpy().view(np.uint32), ev)


def test_sorted_input_skips_histogram_only_when_identity(ahs, orc):
    """Under GB300 an input in order is returned as it is without its
    histogram (entropy NaN); under PAPER, or when a strategy is forced, the
    histogram is built and the result is the oracle's."""
    import torch
    a = np.sort(_gen("uniform_full", 300_001, np.uint32, 5))
    g = ahs.Context(0, select_mode=ahs.AHS_SEL_GB300)
    p = ahs.Context(0, select_mode=ahs.AHS_SEL_PAPER)
    try:
        r = g.sort(dev(a), key_type=ahs.AHS_U32)
        torch.cuda.synchronize()
        assert r.strategy == ahs.AHS_IDENTITY
        assert math.isnan(r.info.features.entropy_bits) and math.isnan(r.info.features.entropy_norm)
        assert r.info.features.descents == 0
        assert np.array_equal(host(r.keys, np.uint32), a)
        of = orc.features(a)
        rp = p.sort(dev(a), key_type=ahs.AHS_U32)
        torch.cuda.synchronize()
        assert math.isclose(rp.info.features.entropy_bits, of.entropy, rel_tol=ENT_REL, abs_tol=ENT_ABS)
        assert np.array_equal(host(rp.keys, np.uint32), a)
        for force in (ahs.AHS_GENERAL, ahs.AHS_RADIX):
            rf = g.sort(dev(a), force=force, key_type=ahs.AHS_U32)
            torch.cuda.synchronize()
            assert math.isclose(rf.info.features.entropy_bits, of.entropy, rel_tol=ENT_REL,
                                abs_tol=ENT_ABS)
            assert np.array_equal(host(rf.keys, np.uint32), a)
    finally:
        g.close()
        p.close()
