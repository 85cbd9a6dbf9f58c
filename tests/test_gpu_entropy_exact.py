"""The device exact-entropy mode (entropy over every distinct value, and the
distinct count k') against the oracle's exact entropy (sort + run lengths in
plain C) and distinct count; for k <= 2^16 it equals the feature pass's
histogram entropy.  Tolerance: 1e-9 relative, 1e-12 absolute (fp64 sums in
different orders)."""
import math

import numpy as np
import pytest

import oracle
from gen import host as gen
from gpu_util import dev, key_type

pytestmark = pytest.mark.gpu

REL, ABS = 1e-9, 1e-12


@pytest.fixture(scope="module")
def ahs():
    import paper_2506_20677_gb300 as m
    return m


def _cases():
    rng = np.random.default_rng(77)
    yield "one", np.array([42], np.uint32)
    yield "all_equal", np.full(300_001, 9, np.uint64)
    yield "two_values", np.where(rng.random(100_000) < 0.25, 3, 8).astype(np.int32)
    yield "uniform32", gen.uniform_u32(1 << 20, 5, 1, 1 << 32)
    yield "k4096", gen.uniform_u32((1 << 20) + 7, 5, 2, 4096)
    yield "zipf", gen.zipf_u32((1 << 21) + 3, 5, 3, 4)
    yield "runs_long", np.repeat(rng.integers(0, 2**40, 50, dtype=np.uint64), 10_000)
    yield "ramp", gen.ramp_u64(1 << 20, 6)
    yield "kmers", gen.kmer_u64((1 << 20) + 1, 5, 30)
    yield "gauss", gen.gaussian_i32(1 << 20, 5, 40, 10**6)


@pytest.mark.parametrize("name,a", list(_cases()))
def test_exact_entropy_against_oracle(ahs, name, a):
    with ahs.Context(0) as ctx:
        d = dev(a)
        h, k = ctx.entropy_exact(d, key_type=key_type(a))
        assert k == oracle.distinct(a), name
        assert math.isclose(h, oracle.entropy_exact(a), rel_tol=REL, abs_tol=ABS), name
        f = ctx.features(d, key_type=key_type(a))
        if f.span < 65536:       # bins are values: the two entropies are one quantity
            assert math.isclose(h, f.entropy_bits, rel_tol=REL, abs_tol=ABS), name
        # the input itself is untouched
        assert np.array_equal(d.cpu().numpy().view(a.dtype), a)


def test_exact_entropy_feeds_the_lemma32_profile(ahs):
    """k' from the device mode drives Table V's skewed-range rule."""
    a = gen.zipf_u32(1 << 20, 8, 3, 4, n_values=600)     # 600 distinct values over 2^32
    with ahs.Context(0, select_mode=ahs.AHS_SEL_LEMMA32) as ctx:
        d = dev(a)
        f = ctx.features(d, key_type=ahs.AHS_U32)
        h, k = ctx.entropy_exact(d, key_type=ahs.AHS_U32)
        assert k == oracle.distinct(a) <= 600
        assert ctx.select(f, ahs.AHS_SEL_LEMMA32) == ahs.AHS_RADIX      # k' unknown
        f.distinct = k
        assert ctx.select(f, ahs.AHS_SEL_LEMMA32) == ahs.AHS_COUNTING   # k' <= 1000
        # an AUTO sort under the profile is the unique sorted order
        r = ctx.sort(d, key_type=ahs.AHS_U32)
        assert np.array_equal(r.keys.cpu().numpy().view(np.uint32), oracle.sort(a)[0])
