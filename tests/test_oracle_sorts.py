"""Pins for the oracle's sorts (Listings 1-4, 7) and its pipeline.

Each forced strategy must produce the unique non-decreasing permutation of
the input (Python's ``sorted``) and, with a payload, the unique stable order
(Python's ``sorted`` is stable).  Brute force covers every sequence over small
alphabets, mapped onto values that include the extremes of each key type.
"""
import itertools

import numpy as np
import pytest

from conftest import read_golden

DTS = [np.uint32, np.uint64, np.int32, np.int64]


def _alphabet(dt, size):
    info = np.iinfo(dt)
    pool = sorted({int(info.min), int(info.min) + 1, -7 if info.min < 0 else 3, 0, 1, 2,
                   1000, int(info.max) - 1, int(info.max)})
    idx = np.linspace(0, len(pool) - 1, size).round().astype(int)
    vals = sorted({pool[i] for i in idx})
    while len(vals) < size:           # fill with small distinct values
        vals = sorted(set(vals) | {len(vals) + 10})
    return vals[:size]


def _small_alphabet(dt, size):
    base = -3 if np.iinfo(dt).min < 0 else 5
    return [base + i for i in range(size)]


def _check_all(orc, keys, strategies, kv=True):
    exp_keys = np.array(sorted(keys.tolist()), dtype=keys.dtype)
    order = sorted(range(len(keys)), key=lambda i: keys[i])   # stable
    exp_vals = np.array(order, dtype=np.uint32)
    vals = np.arange(len(keys), dtype=np.uint32)
    for s in strategies:
        if s == "quick":
            assert np.array_equal(orc.quicksort(keys), exp_keys)
            continue
        fn = getattr(orc, s)
        assert np.array_equal(fn(keys), exp_keys), s
        if kv:
            ko, vo = fn(keys, vals)
            assert np.array_equal(ko, exp_keys), s
            assert np.array_equal(vo, exp_vals), s


@pytest.mark.parametrize("dt", DTS)
def test_brute_force_all_sequences(orc, dt):
    """Every sequence of length n <= 5 over an alphabet of n values (n^n inputs)."""
    for n in range(0, 6):
        alpha = _alphabet(dt, max(n, 1))
        small = _small_alphabet(dt, max(n, 1))
        for seq in itertools.product(range(max(n, 1)), repeat=n):
            keys = np.array([alpha[i] for i in seq], dtype=dt)
            _check_all(orc, keys, ["insertion_sort", "radix_sort", "merge_sort", "quick"])
            keys_small = np.array([small[i] for i in seq], dtype=dt)
            _check_all(orc, keys_small, ["counting_sort"])


@pytest.mark.parametrize("dt", [np.uint32, np.int64])
def test_brute_force_permutations_n8(orc, dt):
    """Every permutation of three multisets of size 8 (distinct, pairs, heavy dup)."""
    for ms in ([0, 1, 2, 3, 4, 5, 6, 7], [0, 0, 1, 1, 2, 2, 3, 3], [5, 5, 5, 5, 5, 1, 9, 9]):
        alpha = _alphabet(dt, 10)
        seen = set()
        for perm in itertools.permutations(ms):
            if perm in seen:
                continue
            seen.add(perm)
            keys = np.array([alpha[i] for i in perm], dtype=dt)
            _check_all(orc, keys, ["radix_sort", "merge_sort", "quick"], kv=(len(seen) % 7 == 0))


@pytest.mark.parametrize("dt", DTS)
def test_random_against_numpy(orc, dt):
    rng = np.random.default_rng(1)
    info = np.iinfo(dt)
    for n in (0, 1, 2, 31, 257, 4099):
        for lo, hi in ((info.min, info.max), (0, 300), (info.max - 1000, info.max)):
            keys = rng.integers(lo, hi, size=n, dtype=dt, endpoint=True)
            exp = np.sort(keys, kind="stable")
            exp_idx = np.argsort(keys, kind="stable").astype(np.uint32)
            vals = np.arange(n, dtype=np.uint32)
            for fn in (orc.radix_sort, orc.merge_sort):
                ko, vo = fn(keys, vals)
                assert np.array_equal(ko, exp) and np.array_equal(vo, exp_idx)
            assert np.array_equal(orc.quicksort(keys), exp)
            if hi - lo <= 300:
                ko, vo = orc.counting_sort(keys, vals)
                assert np.array_equal(ko, exp) and np.array_equal(vo, exp_idx)


@pytest.mark.parametrize("dt", [np.int32, np.int64])
def test_listing7_signed(orc, dt):
    rng = np.random.default_rng(2)
    info = np.iinfo(dt)
    for n in (0, 1, 5, 1000):
        keys = rng.integers(info.min, info.max, size=n, dtype=dt, endpoint=True)
        if n > 3:
            keys[0], keys[1] = info.min, info.max
        assert np.array_equal(orc.radix_sort_signed_listing7(keys), np.sort(keys))


def test_quicksort_presorted_and_duplicates(orc):
    """Listing 4's filters drop extra copies of the pivot; the oracle keeps them."""
    a = np.array([3, 3, 3, 1, 3, 2, 3], dtype=np.uint32)
    assert orc.quicksort(a).tolist() == [1, 2, 3, 3, 3, 3, 3]
    b = np.arange(5000, dtype=np.uint32)
    assert np.array_equal(orc.quicksort(b), b)
    assert np.array_equal(orc.quicksort(b[::-1].copy()), b)
    c = np.full(3000, 9, dtype=np.uint64)
    assert np.array_equal(orc.quicksort(c), c)


@pytest.mark.parametrize("row", read_golden("radix_passes_eq4.txt"), ids=lambda r: r[0])
def test_radix_passes_eq4(orc, row):
    k, d = int(row[0]), int(row[1])
    assert orc.radix_passes(k - 1) == d


def test_counting_range_guard(orc):
    a = np.array([0, 2**40], dtype=np.uint64)
    with pytest.raises(RuntimeError):
        orc.counting_sort(a)


@pytest.mark.parametrize("force", [1, 2, 3, 4, 5])
def test_pipeline_forced(orc, force):
    rng = np.random.default_rng(force)
    keys = rng.integers(0, 500, size=3000, dtype=np.uint32)
    vals = np.arange(3000, dtype=np.uint32)
    ko, vo, chosen, f = orc.sort(keys, vals, force=force)
    assert chosen == force
    if force == orc.IDENTITY:
        assert np.array_equal(ko, keys)
    else:
        assert np.array_equal(ko, np.sort(keys, kind="stable"))
        assert np.array_equal(vo, np.argsort(keys, kind="stable").astype(np.uint32))


def test_pipeline_auto_paper(orc):
    rng = np.random.default_rng(9)
    cases = [
        (rng.integers(0, 100, size=15, dtype=np.uint32), orc.SMALL),
        (np.full(100, 7, dtype=np.uint32), orc.IDENTITY),
        (rng.integers(0, 1000, size=5000, dtype=np.uint32), orc.COUNTING),
        (rng.integers(0, 2**32, size=5000, dtype=np.uint64), orc.GENERAL),
    ]
    # low entropy, wide range: 8 distinct values spread over 2^40 (h = 3/16 < 0.7)
    vals8 = np.array([0, 1, 2**20, 2**30, 2**35, 2**38, 2**39, 2**40], dtype=np.uint64)
    cases.append((vals8[rng.integers(0, 8, size=5000)], orc.RADIX))
    for keys, expect in cases:
        ko, _, chosen, _ = orc.sort(keys)
        assert chosen == expect
        assert np.array_equal(ko, np.sort(keys))
