"""The memory-aware choice for large ranges (Section III-I: Lemma 3.2 and
Table V) pinned by a hand-written decision table; the oracle and the library
(host-only context) are each checked against it.  Also the distinct-value
count k' of the oracle against numpy."""
import ctypes

import numpy as np
import pytest

from conftest import read_golden

NAMES = {"IDENTITY": 1, "SMALL": 2, "COUNTING": 3, "RADIX": 4, "GENERAL": 5}


def _rows():
    return [(int(n), int(span), int(d), NAMES[e]) for n, span, d, e in read_golden("lemma32_decisions.txt")]


@pytest.mark.parametrize("row", _rows())
def test_oracle_lemma32(orc, row):
    n, span, distinct, want = row
    f = orc.Features()
    f.n, f.span, f.nbins = n, span, 65536
    assert orc.select_lemma32(f, orc.PAPER, distinct) == want


def test_library_lemma32():
    import paper_2506_20677_gb300 as ahs
    cfg = ahs.ahs_config_t()
    ahs.lib.ahs_default_config(ctypes.byref(cfg))
    cfg.device = -1
    cfg.select_mode = ahs.AHS_SEL_LEMMA32
    h = ctypes.c_void_p()
    ahs.check(ahs.lib.ahs_create(ctypes.byref(h), ctypes.byref(cfg)), "ahs_create")
    try:
        for n, span, distinct, want in _rows():
            f = ahs.ahs_features_t()
            f.n, f.span, f.nbins, f.distinct = n, span, 65536, distinct
            out = ctypes.c_int()
            ahs.check(ahs.lib.ahs_select(h, ctypes.byref(f), ahs.AHS_SEL_LEMMA32, 4, 0,
                                         ctypes.byref(out)), "ahs_select")
            assert out.value == want, (n, span, distinct)
    finally:
        ahs.lib.ahs_destroy(h)


def test_oracle_distinct_against_numpy(orc):
    rng = np.random.default_rng(4)
    for dt in (np.uint32, np.int32, np.uint64, np.int64):
        info = np.iinfo(dt)
        for a in (np.zeros(0, dt), np.array([5], dt), rng.integers(0, 40, 1000).astype(dt),
                  rng.integers(info.min, info.max, 5000, dtype=dt, endpoint=True),
                  np.array([info.min, info.max, info.min, 0], dt)):
            assert orc.distinct(a) == len(np.unique(a))
