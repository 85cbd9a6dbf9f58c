"""Presorted inputs in reverse order (Section III-B's descending edge case)
under the GB300 profile: found by the min/max pass (no ascents) and returned
reversed, against the oracle's pick and sort of the same arrays.

Keys only, ties allowed; with a payload only strictly decreasing keys are
reversed (the reversal is then the stable order), otherwise the profile's
rules sort them stably.  Ragged and odd sizes, misaligned and in-place
buffers, the four key types; the PAPER profile never reverses."""
import numpy as np
import pytest

import oracle
from gpu_util import dev, host

pytestmark = pytest.mark.gpu

GB = oracle.Profile(4096, 65536, 10**6, sorted_identity=True)


@pytest.fixture(scope="module")
def ahs():
    import paper_2506_20677_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(ahs):
    c = ahs.Context(0)   # GB300 profile by default
    yield c
    c.close()


def _desc(rng, n, dtype, distinct):
    info = np.iinfo(dtype)
    if distinct:
        a = np.unique(rng.integers(0, 2**31 - 1, size=n + n // 8 + 100)).astype(dtype)
        rng.shuffle(a)
        a = a[:n]
        assert len(a) == n
    else:
        a = rng.integers(info.min // 2, info.max // 2, size=n, dtype=dtype)
        a = a[rng.integers(0, max(1, n // 3), size=n)]   # ties
    return np.sort(a)[::-1].copy()


@pytest.mark.parametrize("dtype", [np.uint32, np.int32, np.uint64, np.int64])
@pytest.mark.parametrize("n", [2, 3, 1000, (1 << 20) + 7])
def test_reversed_keys(ahs, ctx, dtype, n):
    import torch
    rng = np.random.default_rng(n + np.dtype(dtype).itemsize)
    a = _desc(rng, n, dtype, distinct=False)
    kt = {np.uint32: ahs.AHS_U32, np.int32: ahs.AHS_I32, np.uint64: ahs.AHS_U64,
          np.int64: ahs.AHS_I64}[dtype]
    ko, _, chosen, of = oracle.sort(a, profile=GB)
    r = ctx.sort(dev(a), key_type=kt)
    torch.cuda.synchronize()
    assert np.array_equal(host(r.keys, dtype), ko)
    expect = "REVERSE" if of.descents > 0 else "IDENTITY"
    assert ahs.STRATEGY_NAMES[r.strategy] == oracle.STRATEGY_NAMES[chosen] == expect
    f = r.info.features
    assert (f.descents, f.ascents) == (of.descents, of.ascents) and f.ascents == 0
    assert np.isnan(f.entropy_bits)   # no histogram pass for a presorted input


def test_payload_strict_and_tied(ahs, ctx):
    import torch
    rng = np.random.default_rng(5)
    n = (1 << 19) + 3
    v = np.arange(n, dtype=np.uint32)
    for distinct, expect_reverse in ((True, True), (False, False)):
        a = _desc(rng, n, np.uint32, distinct)
        ko, vo, chosen, _ = oracle.sort(a, v, profile=GB)
        r = ctx.sort(dev(a), vals=dev(v), key_type=ahs.AHS_U32)
        torch.cuda.synchronize()
        assert np.array_equal(host(r.keys, np.uint32), ko)
        assert np.array_equal(host(r.vals, np.uint32), vo)
        assert (ahs.STRATEGY_NAMES[r.strategy] == "REVERSE") == expect_reverse
        assert ahs.STRATEGY_NAMES[r.strategy] == oracle.STRATEGY_NAMES[chosen]


def test_in_place_and_misaligned(ahs, ctx):
    import torch
    rng = np.random.default_rng(6)
    n = (1 << 20) + 1
    a = _desc(rng, n, np.uint32, distinct=False)
    d = dev(a)
    r = ctx.sort(d, out=d, key_type=ahs.AHS_U32)
    torch.cuda.synchronize()
    assert ahs.STRATEGY_NAMES[r.strategy] == "REVERSE"
    assert np.array_equal(host(d, np.uint32), np.sort(a))
    big = torch.zeros(n + 8, dtype=torch.int32, device="cuda")
    src = big[1:n + 1]
    src.copy_(torch.from_numpy(a.view(np.int32)))
    obig = torch.zeros(n + 8, dtype=torch.int32, device="cuda")
    out = obig[3:n + 3]
    r = ctx.sort(src, out=out, key_type=ahs.AHS_U32)
    torch.cuda.synchronize()
    assert np.array_equal(host(out, np.uint32), np.sort(a))
    assert int(obig[:3].abs().sum()) == 0 and int(obig[n + 3:].abs().sum()) == 0


def test_paper_profile_sorts(ahs):
    import torch
    c = ahs.Context(0, select_mode=ahs.AHS_SEL_PAPER)
    try:
        a = _desc(np.random.default_rng(7), 1 << 18, np.uint32, distinct=False)
        ko, _, chosen, _ = oracle.sort(a, profile=oracle.PAPER)
        r = c.sort(dev(a), key_type=ahs.AHS_U32)
        torch.cuda.synchronize()
        assert np.array_equal(host(r.keys, np.uint32), ko)
        assert ahs.STRATEGY_NAMES[r.strategy] == oracle.STRATEGY_NAMES[chosen] != "REVERSE"
    finally:
        c.close()


def test_ascents_of_unsorted_input(ahs, ctx):
    rng = np.random.default_rng(8)
    for n in (5, 4099, (1 << 20) + 9):
        a = rng.integers(0, 1000, size=n, dtype=np.uint32)
        f = ctx.features(dev(a), key_type=ahs.AHS_U32)
        assert f.ascents == int(np.count_nonzero(a[:-1] < a[1:]))
        assert f.descents == int(np.count_nonzero(a[:-1] > a[1:]))
