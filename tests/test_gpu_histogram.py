"""The feature histogram above 43,692 bins (16-bit packed counters per CTA,
flushed at 2^15, with the split layout as the exact fallback) against the
oracle: bins, shift and entropy for inputs whose heavy bins get far more than
2^15 keys per CTA, and the same features when the split layout runs."""
import numpy as np
import pytest

import oracle
from gpu_util import dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ahs():
    import paper_2506_20677_gb300 as m
    return m


def _heavy(rng, n, dtype, share):
    """A wide range (every bin width > 1) with one value holding `share` of
    the keys and a second one a quarter of the rest."""
    info = np.iinfo(dtype)
    a = rng.integers(info.min, info.max, size=n, dtype=dtype)
    m = rng.random(n)
    a[m < share] = dtype(12345)
    a[(m >= share) & (m < share + (1 - share) / 4)] = dtype(-7 if info.min < 0 else 99)
    return a


@pytest.mark.parametrize("dtype", [np.uint32, np.int32, np.uint64])
@pytest.mark.parametrize("share", [0.5, 0.99])
def test_heavy_bins_against_oracle(ahs, dtype, share):
    kt = {np.uint32: ahs.AHS_U32, np.int32: ahs.AHS_I32, np.uint64: ahs.AHS_U64}[dtype]
    rng = np.random.default_rng(int(share * 100) + np.dtype(dtype).itemsize)
    a = _heavy(rng, (1 << 24) + 3, dtype, share)
    of = oracle.features(a)
    assert of.nbins > 43692
    for flags in (0, ahs.AHS_DEBUG_K2_SPLIT):
        c = ahs.Context(0, debug_flags=flags)
        try:
            f = c.features(dev(a), key_type=kt)
        finally:
            c.close()
        assert (f.nbins, f.hist_shift, f.span) == (of.nbins, of.shift, of.span)
        assert abs(f.entropy_bits - of.entropy) <= 1e-9 * of.entropy + 1e-12


def test_sorts_match_with_split_retry(ahs):
    import torch
    rng = np.random.default_rng(3)
    a = _heavy(rng, (1 << 22) + 1, np.uint32, 0.7)
    ko = oracle.radix_sort(a)
    for flags in (0, ahs.AHS_DEBUG_K2_SPLIT):
        c = ahs.Context(0, debug_flags=flags)
        try:
            r = c.sort(dev(a), key_type=ahs.AHS_U32)
            torch.cuda.synchronize()
            assert np.array_equal(r.keys.cpu().numpy().view(np.uint32), ko)
        finally:
            c.close()
