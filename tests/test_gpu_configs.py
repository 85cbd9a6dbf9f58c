"""The workload configurations on the GPU.

At 1/64 scale every output is compared with the oracle element by element; at
full size (n = 2^28, 2^27), in the launch configuration bench.py times, the
output is checked through properties that fix it exactly (order, multiset,
sampled order statistics; for key-value, permutation + gather + stability).
"""
import numpy as np
import pytest

from gen import host as gen
from gpu_util import check_sorted_permutation, check_stable_kv, dev, host

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


EXPECT_GB300 = {"a": "COUNTING", "b": "RADIX", "c": "GENERAL", "d": "IDENTITY", "e": "GENERAL",
                "f": "REVERSE"}
NAMED = {"a": "COUNTING", "b": "RADIX", "c": "GENERAL", "d": "GENERAL", "e": "GENERAL",
         "f": "GENERAL"}


def test_config1_full(ahs, ctx, orc):
    a = gen.config1()
    r = ctx.sort(dev(a), key_type=ahs.AHS_U32)
    ko, _, chosen, f = orc.sort(a, force=orc.AUTO, profile=orc.PAPER)
    assert ahs.STRATEGY_NAMES[r.strategy] == "COUNTING" == orc.STRATEGY_NAMES[chosen]
    assert np.array_equal(host(r.keys, np.uint32), ko)
    assert abs(r.info.features.entropy_bits - f.entropy) <= 1e-9 * f.entropy


@pytest.mark.parametrize("variant", list("abcdef"))
def test_config2_scaled(ahs, ctx, orc, variant):
    n = (1 << 28) // 64
    a = gen.config2(variant, n)
    r = ctx.sort(dev(a), key_type=ahs.AHS_U32)
    assert ahs.STRATEGY_NAMES[r.strategy] == EXPECT_GB300[variant]
    ko = orc.radix_sort(a)
    assert np.array_equal(host(r.keys, np.uint32), ko)
    forced = getattr(ahs, "AHS_" + NAMED[variant])
    r2 = ctx.sort(dev(a), force=forced, key_type=ahs.AHS_U32)
    assert np.array_equal(host(r2.keys, np.uint32), ko)


@pytest.mark.parametrize("variant", list("abcef"))
def test_config2_full(ahs, ctx, variant):
    from gen import device as gdev   # bit-identical to gen.host (tests/test_gpu_gen.py)
    d = gdev.config2(variant)
    forced = getattr(ahs, "AHS_" + NAMED[variant])
    r = ctx.sort(d, force=forced, key_type=ahs.AHS_U32)
    check_sorted_permutation(host(d, np.uint32), host(r.keys, np.uint32))


def test_config3_scaled(ahs, ctx, orc):
    keys, vals = gen.config3((1 << 27) // 64)
    r = ctx.sort(dev(keys), vals=dev(vals), force=ahs.AHS_RADIX, key_type=ahs.AHS_U64)
    ko, vo = orc.radix_sort(keys, vals)
    assert np.array_equal(host(r.keys, np.uint64), ko)
    assert np.array_equal(host(r.vals, np.uint32), vo)


def test_config3_full(ahs, ctx):
    from gen import device as gdev
    keys, vals = gdev.config3()
    r = ctx.sort(keys, vals=vals, force=ahs.AHS_RADIX, key_type=ahs.AHS_U64)
    check_stable_kv(host(keys, np.uint64), host(r.keys, np.uint64), host(r.vals, np.uint32))


@pytest.mark.slow
@pytest.mark.parametrize("variant", list("abcdef"))
def test_config2_full_against_oracle(ahs, ctx, orc, variant):
    """Config 2 at n = 2^28 in the launch configuration the bench times (AUTO
    under the GB300 profile), element by element against the oracle's sort of
    the host generator's keys (the oracle's counting sort for the k = 4096
    array, its LSD radix sort for the others)."""
    a = gen.config2(variant)
    r = ctx.sort(dev(a), key_type=ahs.AHS_U32)
    assert ahs.STRATEGY_NAMES[r.strategy] == EXPECT_GB300[variant]
    out = host(r.keys, np.uint32)
    del r
    ko = orc.counting_sort(a) if variant == "a" else orc.radix_sort(a)
    assert np.array_equal(out, ko)
