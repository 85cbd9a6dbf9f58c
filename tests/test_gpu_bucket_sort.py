"""GPU parity for the keys-only one-CTA sort on inputs built for its hard cases.

Without a payload a one-CTA sort (the SMALL strategy, and each bucket of the
general path) counts the keys by their leading bits with about one counter per
key, 2^lgc counters for m keys, lgc = bitlen(m - 1 - floor(m / 5)), and then
insertion-sorts the keys that share a counter (a sub-bucket).  The inputs here
span exactly lgc + R bits, so a sub-bucket is the set of keys whose offset from
the minimum agrees above its R trailing bits.  They are filled with 1 to 32
distinct keys each, in descending input order (the most shifts an insertion
sort can meet), and optionally one sub-bucket of more than 32 distinct keys,
which sends the whole CTA to the stable LSD passes instead.  Keys are
compared with the oracle element by element.
"""
import numpy as np
import pytest

from gpu_util import dev, host, key_type

DTS = [np.uint32, np.int32, np.uint64, np.int64]


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


def subbucket_keys(m, dt, seed, r_bits=6, big=False):
    """m >= 64 keys spanning lgc + r_bits bits whose sub-buckets hold many
    distinct keys in descending order (see the module docstring); big adds one
    sub-bucket of 40 (r_bits >= 6)."""
    assert m >= 64 and (not big or r_bits >= 6)
    rng = np.random.default_rng(seed)
    lgc = int(m - 1 - m // 5).bit_length()
    nsub, w = 1 << lgc, 1 << r_bits
    inner = rng.permutation(np.arange(1, nsub - 1))
    offsets = []
    if big:   # more distinct keys in one sub-bucket than the insertion sort takes
        d, inner = int(inner[0]), inner[1:]
        offsets.append(d * w + np.sort(rng.choice(w, size=40, replace=False))[::-1])
    # the span: offset 0 in the first sub-bucket, the largest in the last
    offsets.append(np.array([(nsub - 1) * w + w - 1]))
    offsets.append(np.array([0]))
    have = sum(len(o) for o in offsets)
    for d in inner:
        if have == m:
            break
        s = min(int(rng.choice([1, 2, 3, 5, 6, 8, 11, 16, 23, 32])), w, m - have)
        offsets.append(int(d) * w + np.sort(rng.choice(w, size=s, replace=False))[::-1])
        have += s
    # sub-buckets in random order, each one's keys contiguous and descending
    order = rng.permutation(len(offsets))
    u = np.concatenate([offsets[i] for i in order]).astype(np.int64)
    assert len(u) == m and u.min() == 0 and u.max() == nsub * w - 1
    info = np.iinfo(dt)
    base = -(nsub * w // 2) if info.min < 0 else (1 << 33) + 5 if info.bits == 64 else 1000
    return (u + base).astype(dt)


def _check_against_oracle(ahs, ctx, a, force):
    import oracle
    import torch
    r = ctx.sort(dev(a), force=force, key_type=key_type(a))
    torch.cuda.synchronize()
    ok = oracle.sort(a, force=oracle.RADIX)[0]
    assert np.array_equal(host(r.keys, a.dtype), ok)
    return r


def test_builder_makes_the_intended_sub_buckets():
    """CPU check of the construction: span, counter count and sub-bucket sizes."""
    for m in (64, 1000, 4000, 8192):
        for r_bits, big in ((6, False), (6, True), (3, False), (8, True)):
            a = subbucket_keys(m, np.int32, m + r_bits, r_bits=r_bits, big=big)
            u = a.astype(np.int64) - int(a.min())
            lgc = int(m - 1 - m // 5).bit_length()
            assert len(a) == m
            assert int(u.max()).bit_length() == lgc + r_bits
            sizes = np.sort(np.bincount(u >> r_bits))
            if big:
                assert sizes[-1] == 40 and sizes[-2] <= 32
            else:
                assert sizes[-1] <= 32
            assert np.count_nonzero(sizes >= 5) > 0 or m < 1000
            assert len(np.unique(u)) == m   # distinct keys: every inversion shifts


@pytest.mark.gpu
@pytest.mark.parametrize("dt", DTS, ids=lambda d: np.dtype(d).name)
def test_small_sort_sub_buckets(ahs, ctx, dt):
    cap = int(ahs.lib.ahs_small_capacity(key_type(np.zeros(1, dt)), 0))
    for i, m in enumerate([64, 1000, 1024, 1025, 3000, 4000, 4097, cap - 3, cap]):
        for big in (False, True):
            a = subbucket_keys(m, dt, 100 + i, big=big)
            r = _check_against_oracle(ahs, ctx, a, ahs.AHS_SMALL)
            assert r.strategy == ahs.AHS_SMALL


@pytest.mark.gpu
@pytest.mark.parametrize("dt", DTS, ids=lambda d: np.dtype(d).name)
def test_general_sort_sub_bucket_blocks(ahs, ctx, dt):
    """Blocks of the same shape side by side: the partition passes cut them
    into buckets of every size class."""
    rng = np.random.default_rng(7)
    blocks = []
    for b in range(48):
        m = int(rng.integers(600, 4600))
        r_bits = int(rng.integers(3, 9))
        x = subbucket_keys(m, dt, 200 + b, r_bits=r_bits, big=(b % 5 == 0 and r_bits >= 6))
        shift = (b - 24) * (1 << 22)
        blocks.append((x.astype(np.int64) + shift).astype(dt))
    a = np.concatenate(blocks)
    _check_against_oracle(ahs, ctx, a, ahs.AHS_GENERAL)
