"""The second workload family (Section III-B, Table VII) through every
strategy against the oracle: Gaussian-shaped int32 keys N(0, k/4) for
k = 10^2, 10^4, 10^6, and 60-bit k-mer keys of a repetitive genome
(k = 4^30).  Keys and payload permutations bit-exact."""
import numpy as np
import pytest

import oracle
from gen import device as gdev
from gen import host as gen
from gpu_util import dev, host

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


def _check(ahs, ctx, a, kt, forces):
    import torch
    v = np.arange(len(a), dtype=np.uint32)
    ko, vo = oracle.merge_sort(a, v)
    for force in forces:
        r = ctx.sort(dev(a), force=force, key_type=kt)
        torch.cuda.synchronize()
        assert np.array_equal(host(r.keys, a.dtype), ko), (force, "keys")
        r = ctx.sort(dev(a), vals=dev(v), force=force, key_type=kt)
        torch.cuda.synchronize()
        assert np.array_equal(host(r.keys, a.dtype), ko), (force, "kv keys")
        assert np.array_equal(host(r.vals, np.uint32), vo), (force, "kv payload")


@pytest.mark.parametrize("k", [10**2, 10**4, 10**6])
def test_gaussian_all_strategies(ahs, ctx, k):
    n = (1 << 20) + 3
    d = gdev.gaussian_i32(n, 11, 70, k)
    a = d.cpu().numpy()
    assert np.array_equal(a, gen.gaussian_i32(n, 11, 70, k))
    f = ctx.features(d, key_type=ahs.AHS_I32)
    of = oracle.features(a)
    assert (f.span, f.nbins, f.min_bits) == (of.span, of.nbins, of.min_bits)
    forces = [ahs.AHS_AUTO, ahs.AHS_RADIX, ahs.AHS_GENERAL]
    if f.span < 65536:
        forces.append(ahs.AHS_COUNTING)
    _check(ahs, ctx, a, ahs.AHS_I32, forces)


def test_kmers_all_strategies(ahs, ctx):
    n = (1 << 20) + 5
    d = gdev.kmer_u64(n, 12, 80)
    a = d.cpu().numpy().view(np.uint64)
    assert np.array_equal(a, gen.kmer_u64(n, 12, 80))
    f = ctx.features(d, key_type=ahs.AHS_U64)
    of = oracle.features(a)
    assert abs(f.entropy_bits - of.entropy) <= 1e-9 * max(1.0, of.entropy)
    _check(ahs, ctx, a, ahs.AHS_U64, [ahs.AHS_AUTO, ahs.AHS_RADIX, ahs.AHS_GENERAL])
