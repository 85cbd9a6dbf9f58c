"""Host workload generators: published test vectors and distribution shape."""
import math

import numpy as np

from gen import host as g
from gen import host as H


def test_splitmix64_published_sequence():
    """SplitMix64 seeded with 0 (Vigna's splitmix64.c) starts e220a839..., 6e789e6a..., 06c45d18..."""
    assert g.mix64_int(1 * g.GOLDEN) == 0xE220A8397B1DCDAF
    assert g.mix64_int(2 * g.GOLDEN) == 0x6E789E6AA1B965F4
    assert g.mix64_int(3 * g.GOLDEN) == 0x06C45D188009454F
    z = g.mix64(np.array([g.GOLDEN, (2 * g.GOLDEN) % 2**64], dtype=np.uint64))
    assert z.tolist() == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4]


def test_draws_are_counter_based():
    a = g.draws(4, 9, 0, 1000)
    b = g.draws(4, 9, 500, 500)
    assert np.array_equal(a[500:], b)
    assert g.draw_int(4, 9, 17) == int(a[17])
    assert not np.array_equal(a, g.draws(4, 10, 0, 1000))


def test_mulhi64_against_python_ints():
    rng = np.random.default_rng(0)
    a = rng.integers(0, 2**64, size=2000, dtype=np.uint64, endpoint=False)
    for m in (1, 3, 1001, 2**32 + 7, 2**63 + 12345, 2**64 - 1):
        got = g.below64(a, m)
        exp = np.array([(int(x) * m) >> 64 for x in a], dtype=np.uint64)
        assert np.array_equal(got, exp)


def test_uniform_shape():
    x = g.uniform_u32(1 << 20, 0, 0, 256)
    assert x.dtype == np.uint32 and x.min() == 0 and x.max() == 255
    counts = np.bincount(x, minlength=256)
    assert abs(counts.mean() - 4096) < 1e-9 and counts.std() < 4 * math.sqrt(4096)


def test_zipf_shape():
    vals = g.zipf_values(1, 2, 1024)
    assert len(np.unique(vals)) == 1024        # distinct by construction (bijective hash)
    x = g.zipf_u32(1 << 20, 1, 2, 3)
    assert set(np.unique(x).tolist()) <= set(vals.tolist())
    cdf = g.zipf_cdf(1024, 1.1)
    p1 = cdf[0]
    frac_top = np.count_nonzero(x == vals[0]) / len(x)
    assert abs(frac_top - p1) < 5 * math.sqrt(p1 * (1 - p1) / len(x))
    # population entropy of Zipf(1.1) over 1,024 ranks (sum written from the pmf)
    p = np.diff(np.concatenate([[0.0], cdf]))
    assert abs(-(p * np.log2(p)).sum() - 6.8214) < 1e-3


def test_config2_variants():
    n = 1 << 16
    c = g.config2("c", n)
    d = g.config2("d", n)
    e = g.config2("e", n)
    f = g.config2("f", n)
    assert np.array_equal(d, np.sort(c))
    assert np.array_equal(f, d[::-1])
    assert np.array_equal(np.sort(e), d)
    assert 0 < np.count_nonzero(e != d) <= 2 * (n // 100)
    a = g.config2("a", n)
    assert a.max() <= 4095


def test_ramp_shape():
    t = g.ramp_u64(100000, 2)
    base = 1_700_000_000_000_000_000
    assert t.dtype == np.uint64 and t.min() >= base
    assert t.max() <= base + 1000 * 100000
    inversions = np.count_nonzero(t[:-1] > t[1:])
    assert 0.03 * len(t) < inversions < 0.12 * len(t)


def test_config4_layout():
    L, T, O = g.config4_layout()
    assert L.min() >= 16 and L.max() <= 1 << 20 and len(L) == 100000
    # mean of floor(exp(U(ln16, ln2^20))) ~ (2^20 - 16) / ln(2^16)
    assert abs(L.mean() / ((2**20 - 16) / math.log(2**16)) - 1) < 0.03
    assert int(O[-1]) == int(L.sum())
    assert np.all(np.bincount(T) > 24000)
    s = g.config4_segment(5, int(L[5]), int(T[5]))
    assert len(s) == L[5]


def test_gaussian_shape_and_determinism():
    """Irwin-Hall sum of 12 uniforms: mean ~0 and sd ~sqrt(k/4); a prefix and
    an offset start give the same keys as one call (counter-based)."""
    for k in (10**2, 10**4, 10**6):
        g = H.gaussian_i32(400_000, 1, 30, k)
        sd = (k / 4) ** 0.5
        assert abs(g.std() - sd) < 0.01 * sd + 0.5
        assert abs(g.mean()) < 0.02 * sd + 1.0
        # Irwin-Hall with 12 terms is bounded at 6 sd
        assert g.min() >= -6 * sd - 1 and g.max() <= 6 * sd
    a = H.gaussian_i32(1000, 1, 30, 10**4)
    assert np.array_equal(a[300:], H.gaussian_i32(700, 1, 30, 10**4, start=300))


def test_kmer_shape():
    """60-bit keys, each the next window of the same base sequence."""
    k = H.kmer_u64(50_000, 2, 60)
    assert int(k.max()).bit_length() <= 60
    # consecutive windows overlap in 29 bases: key[i+1] >> 2 == key[i] & (2^58 - 1)
    assert np.array_equal(k[1:] >> np.uint64(2), k[:-1] & np.uint64((1 << 58) - 1))
    assert np.array_equal(k[100:], H.kmer_u64(49_900, 2, 60, start=100))
    # repetitive: far fewer distinct k-mers than keys
    assert len(np.unique(k)) < 0.8 * len(k)
