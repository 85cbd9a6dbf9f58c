"""Batched form (ahs_sort_batch) against the oracle, segment by segment."""
import ctypes

import numpy as np
import pytest

from gen import host as gen
from gpu_util import check_sorted_permutation, dev, host, key_type

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ahs():
    import paper_2506_20677_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(ahs):
    c = ahs.Context(0)
    yield c
    c.close()


def _mixed_segments(dt, seed):
    """Segments of every class and awkward size, one buffer."""
    rng = np.random.default_rng(seed)
    info = np.iinfo(dt)
    sizes = [0, 1, 2, 16, 17, 20, 21, 1000, 4095, 4096, 4097, 8192, 8193, 20000, 65535, 65536,
             70001, 300_001, 3, 0, 50]
    parts = []
    for i, n in enumerate(sizes):
        kind = i % 6
        if kind == 0:
            a = rng.integers(0, 4096, size=n, dtype=dt)                      # counting
        elif kind == 1:
            vals = rng.integers(info.min, info.max, size=1024, dtype=dt, endpoint=True)
            p = 1.0 / np.arange(1, 1025) ** 1.1
            a = vals[rng.choice(1024, size=n, p=p / p.sum())]                # radix (low entropy)
        elif kind == 2:
            a = rng.integers(info.min, info.max, size=n, dtype=dt, endpoint=True)  # general
        elif kind == 3:
            a = np.sort(rng.integers(info.min, info.max, size=n, dtype=dt, endpoint=True))  # identity
        elif kind == 4:
            a = rng.integers(0, 40000, size=n, dtype=dt)                     # wide counting -> radix
        else:
            a = np.full(n, dt(5), dtype=dt)                                  # all equal
        parts.append(a.astype(dt))
    offs = np.zeros(len(parts) + 1, dtype=np.uint64)
    np.cumsum([len(p) for p in parts], out=offs[1:])
    return np.concatenate(parts).astype(dt), offs


@pytest.mark.parametrize("kv", [False, True], ids=["keys", "kv"])
@pytest.mark.parametrize("dt", [np.uint32, np.int32, np.uint64, np.int64], ids=lambda d: np.dtype(d).name)
def test_batch_mixed_against_oracle(ahs, ctx, orc, dt, kv):
    keys, offs = _mixed_segments(dt, 11)
    vals = np.arange(len(keys), dtype=np.uint32) if kv else None
    out, vout, info = ctx.sort_batch(dev(keys), offs.tolist(), vals=dev(vals) if kv else None,
                                     key_type=key_type(keys))
    ko = host(out, dt)
    vo = host(vout, np.uint32) if kv else None
    for s in range(len(offs) - 1):
        b, e = int(offs[s]), int(offs[s + 1])
        seg = keys[b:e]
        if kv:
            ek, ev, _, _ = orc.sort(seg, np.arange(b, e, dtype=np.uint32), force=orc.RADIX)
            assert np.array_equal(ko[b:e], ek), s
            assert np.array_equal(vo[b:e], ev), s
        else:
            assert np.array_equal(ko[b:e], orc.radix_sort(seg)), s
    assert info.n_seg == len(offs) - 1
    assert sum(info.seg_per_strategy) == len(offs) - 1
    assert info.seg_per_strategy[ahs.AHS_COUNTING] + info.seg_per_strategy[ahs.AHS_RADIX] > 0


def test_batch_equals_per_array_calls(ahs, ctx):
    """The batched result is the per-array result, array by array."""
    import torch
    keys, offs = _mixed_segments(np.uint32, 3)
    d = dev(keys)
    out, _, _ = ctx.sort_batch(d, offs.tolist(), key_type=ahs.AHS_U32)
    ko = host(out, np.uint32)
    for s in range(len(offs) - 1):
        b, e = int(offs[s]), int(offs[s + 1])
        if e == b:
            continue
        r = ctx.sort(d[b:e].clone(), key_type=ahs.AHS_U32)
        torch.cuda.synchronize()
        assert np.array_equal(host(r.keys, np.uint32), ko[b:e]), s


def test_batch_offsets_not_starting_at_zero(ahs, ctx, orc):
    rng = np.random.default_rng(2)
    keys = rng.integers(0, 2**32, size=100_000, dtype=np.uint32)
    offs = [1000, 1000, 5000, 60_000, 99_000]
    out, _, _ = ctx.sort_batch(dev(keys), offs, key_type=ahs.AHS_U32)
    ko = host(out, np.uint32)
    for b, e in zip(offs[:-1], offs[1:]):
        assert np.array_equal(ko[b:e], np.sort(keys[b:e]))


def test_batch_rejects_bad_arguments(ahs, ctx):
    import torch
    t = torch.zeros(100, dtype=torch.int32, device="cuda")
    offs = (ctypes.c_uint64 * 3)(0, 60, 40)
    rc = ahs.lib.ahs_sort_batch(ctx.handle, ctypes.c_void_p(t.data_ptr()),
                                ctypes.c_void_p(torch.empty_like(t).data_ptr()), None, None, offs, 2,
                                ahs.AHS_U32, None, None)
    assert rc == ahs.AHS_ERR_INVALID_ARG
    offs = (ctypes.c_uint64 * 2)(0, 100)
    rc = ahs.lib.ahs_sort_batch(ctx.handle, ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                None, None, offs, 1, ahs.AHS_U32, None, None)
    assert rc == ahs.AHS_ERR_INVALID_ARG   # out of place only


def test_config4_scaled(ahs, ctx, orc):
    """Config 4's recipe with 2,000 segments of up to 2^16 keys: every segment."""
    from gen import device as gdev
    keys, offs, lengths, types = gdev.config4(n_seg=2000, hi=1 << 16)
    out, _, info = ctx.sort_batch(keys, offs.tolist(), key_type=ahs.AHS_U32)
    ko = host(out, np.uint32)
    for s in range(2000):
        seg = gen.config4_segment(s, int(lengths[s]), int(types[s]))
        b, e = int(offs[s]), int(offs[s + 1])
        assert np.array_equal(host(keys[b:e], np.uint32), seg), s   # generator parity
        assert np.array_equal(ko[b:e], orc.radix_sort(seg)), s


def test_config4_full(ahs, ctx, orc):
    """Config 4 at full size (100,000 segments, ~9.5e9 keys): sampled segments
    regenerated on the host and sorted by the oracle; the rest by properties."""
    import torch
    from gen import device as gdev
    keys, offs, lengths, types = gdev.config4()
    out = torch.empty_like(keys)
    out, _, info = ctx.sort_batch(keys, offs.tolist(), out=out, key_type=ahs.AHS_U32)
    torch.cuda.synchronize()
    rng = np.random.default_rng(4)
    sample = sorted(set(rng.integers(0, 100_000, size=60).tolist()) | {int(np.argmax(lengths))})
    for s in sample:
        b, e = int(offs[s]), int(offs[s + 1])
        seg = gen.config4_segment(s, int(lengths[s]), int(types[s]))
        assert np.array_equal(host(out[b:e], np.uint32), orc.radix_sort(seg)), s
    # every segment non-decreasing (checked on the device in chunks, no oracle value involved)
    total = int(offs[-1])
    bounds = torch.from_numpy(offs[1:-1].astype(np.int64)).cuda()   # first key of each segment
    chunk = 1 << 28
    for a in range(0, total - 1, chunk):
        b = min(total, a + chunk + 1)
        o = out[a:b].to(torch.int64) & 0xFFFFFFFF
        bad = torch.nonzero(o[1:] < o[:-1]).flatten() + a + 1     # index of the smaller key
        if bad.numel():
            assert bool(torch.isin(bad, bounds).all()), "a segment is out of order"
    assert info.n_keys == total


def test_batch_device_offsets_against_oracle(ahs, ctx, orc):
    """ahs_sort_batch_dev: offsets resident on the device give the same result
    as host offsets, segment by segment the oracle's sort (with a payload)."""
    import torch
    keys, offs = _mixed_segments(np.uint32, 5)
    vals = np.arange(len(keys), dtype=np.uint32)
    d_offs = torch.from_numpy(np.asarray(offs, dtype=np.uint64).view(np.int64)).cuda()
    out, vout, info = ctx.sort_batch(dev(keys), d_offs, vals=dev(vals), key_type=ahs.AHS_U32)
    ko, vo = host(out, np.uint32), host(vout, np.uint32)
    for s in range(len(offs) - 1):
        b, e = int(offs[s]), int(offs[s + 1])
        ek, ev = orc.merge_sort(keys[b:e], vals[b:e])
        assert np.array_equal(ko[b:e], ek), s
        assert np.array_equal(vo[b:e], ev), s
    assert info.n_seg == len(offs) - 1
