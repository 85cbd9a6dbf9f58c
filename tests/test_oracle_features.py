"""Pins for the oracle's state vector v = (n, k, H) (Section III-A, III-H)."""
import math

import numpy as np
import pytest

from conftest import read_golden

DT = {"u32": np.uint32, "u64": np.uint64, "i32": np.int32, "i64": np.int64}


def _expand(runs, dtype):
    out = []
    for tok in runs.split():
        val, cnt = tok.split("*")
        if val.startswith("range("):
            lo, hi = val[len("range("):-1].split(",")
            out.extend(list(range(int(lo), int(hi))) * int(cnt))
        else:
            out.extend([int(val)] * int(cnt))
    return np.array(out, dtype=dtype)


@pytest.mark.parametrize("row", read_golden("entropy_closed_forms.txt"), ids=lambda r: r[0])
def test_entropy_closed_forms(orc, row):
    name, typ, runs, H, h, shift, nbins = row
    keys = _expand(runs, DT[typ])
    rng = np.random.default_rng(len(keys))
    keys = keys[rng.permutation(len(keys))]        # features are permutation-invariant
    f = orc.features(keys)
    assert f.n == len(keys)
    assert f.shift == int(shift)
    assert f.nbins == int(nbins)
    assert math.isclose(f.entropy, float(H), rel_tol=1e-12, abs_tol=1e-12)
    assert math.isclose(f.entropy_norm, float(h), rel_tol=1e-12, abs_tol=1e-12)


@pytest.mark.parametrize("typ", ["u32", "u64", "i32", "i64"])
def test_min_max_span_against_numpy(orc, typ):
    dt = DT[typ]
    info = np.iinfo(dt)
    rng = np.random.default_rng(7)
    for trial in range(20):
        n = int(rng.integers(1, 3000))
        a = rng.integers(info.min, info.max, size=n, dtype=dt, endpoint=True)
        if trial % 3 == 0:
            a[int(rng.integers(0, n))] = info.min
        if trial % 4 == 0:
            a[int(rng.integers(0, n))] = info.max
        f = orc.features(a)
        mn, mx = int(a.min()), int(a.max())
        assert f.min_bits == mn & ((1 << (8 * a.itemsize)) - 1)
        assert f.max_bits == mx & ((1 << (8 * a.itemsize)) - 1)
        assert f.span == mx - mn
        assert f.descents == int(np.count_nonzero(a[:-1] > a[1:]))


def test_empty_and_single(orc):
    f = orc.features(np.zeros(0, dtype=np.uint32))
    assert f.n == 0 and f.entropy == 0.0
    f = orc.features(np.array([42], dtype=np.uint32))
    assert (f.n, f.span, f.nbins, f.entropy, f.entropy_norm, f.descents) == (1, 0, 1, 0.0, 0.0, 0)


def test_binning_rule(orc):
    """s = max(0, bitlen(span) - 16): spans below 2^16 keep one bin per value."""
    for span, s, nb in [(0, 0, 1), (1, 0, 2), (65535, 0, 65536), (65536, 1, 32769),
                        (131071, 1, 65536), (2**32 - 1, 16, 65536), (2**36 + 5, 21, 32769)]:
        a = np.array([0, span], dtype=np.uint64)
        f = orc.features(a)
        assert (f.shift, f.nbins) == (s, nb), span


def test_binned_entropy_equals_exact_when_k_small(orc):
    """For k <= 2^16 the bins are the values, so the binned H is the per-value H."""
    rng = np.random.default_rng(3)
    for k in (2, 17, 1000, 65536):
        a = rng.integers(0, k, size=20000, dtype=np.uint32)
        assert math.isclose(orc.features(a).entropy, orc.entropy_exact(a), rel_tol=1e-12)


def test_exact_entropy_brute_force(orc):
    """Per-value entropy against counts from Python's collections.Counter."""
    from collections import Counter
    rng = np.random.default_rng(5)
    a = rng.integers(-2**40, 2**40, size=500, dtype=np.int64)
    a[:100] = a[100:200]
    c = Counter(a.tolist())
    n = len(a)
    # closed form for a multiset: H = log2 n - (1/n) sum c log2 c (exact rearrangement)
    expect = math.log2(n) - sum(v * math.log2(v) for v in c.values()) / n
    assert math.isclose(orc.entropy_exact(a), expect, rel_tol=1e-12)


def test_entropy_invariant_under_shift(orc):
    """H depends only on the multiset of differences x - min."""
    rng = np.random.default_rng(11)
    a = rng.integers(0, 5000, size=10000, dtype=np.int64)
    f1 = orc.features(a)
    f2 = orc.features(a + 123456789)
    assert f1.entropy == f2.entropy and f1.span == f2.span


def test_rejects_non_integer(orc):
    with pytest.raises(TypeError):
        orc.features(np.zeros(4, dtype=np.float32))


def test_zipf_sample_entropy_near_population(orc):
    """Config 2b draws Zipf(1.1) over 1,024 distinct values: the exact
    per-value entropy of a 2^22-key sample lies near the population's
    H = -sum p_r log2 p_r, p_r = r^-1.1 / sum_j j^-1.1 (sampling error about
    1e-3 bits here, plug-in bias about 2e-4)."""
    from gen import host as gen
    r = np.arange(1, 1025, dtype=np.float64)
    p = r ** -1.1
    p /= p.sum()
    h_pop = float(-(p * np.log2(p)).sum())
    assert abs(h_pop - 6.8214) < 1e-3            # the population value of this recipe
    a = gen.config2("b", 1 << 22)
    h = orc.entropy_exact(a)
    assert abs(h - h_pop) < 5e-3
    # The 2^16-bin feature entropy cannot exceed the exact one (bins merge values).
    assert orc.features(a).entropy <= h + 1e-9
