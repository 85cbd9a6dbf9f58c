"""The tuned-shape table: loader, lookups and fallbacks (host-only context, no GPU).

The radix rows choose the largest digit width r of the stable LSD passes; the
plan then takes d = ceil(D / r) passes for a D-bit key range (Eq. 4 with base
2^r) and shares the D bits evenly between them."""
import ctypes
import math
import os

import pytest


def _host_ctx(ahs, tuning=None):
    cfg = ahs.ahs_config_t()
    ahs.lib.ahs_default_config(ctypes.byref(cfg))
    cfg.device = -1
    cfg.tuning_path = None if tuning is None else os.fsencode(str(tuning))
    h = ctypes.c_void_p()
    rc = ahs.lib.ahs_create(ctypes.byref(h), ctypes.byref(cfg))
    return rc, h


def _plan(ahs, h, span, kb=8, pay=1):
    p, b = ctypes.c_uint32(), ctypes.c_uint32()
    ahs.check(ahs.lib.ahs_tuned_radix_bits(h, kb, pay, span, ctypes.byref(p), ctypes.byref(b)), "plan")
    return p.value, b.value


def test_defaults_are_base_256():
    import paper_2506_20677_gb300 as ahs
    rc, h = _host_ctx(ahs)
    assert rc == ahs.AHS_OK
    try:
        # Eq. 4: d = ceil(log_256 k)
        for D in (1, 7, 8, 9, 16, 24, 32, 36, 64):
            span = (1 << D) - 1
            p, b = _plan(ahs, h, span)
            assert p == math.ceil(D / 8), D
            assert b == math.ceil(D / p)
        assert _plan(ahs, h, 0) == (0, 0)
    finally:
        ahs.lib.ahs_destroy(h)


def test_table_rows_and_even_split(tmp_path):
    import paper_2506_20677_gb300 as ahs
    t = tmp_path / "t.txt"
    t.write_text("# tuned on a test box\nahs-tuning 1\n"
                 "radix_bits 8 1 40 11\n"
                 "radix_bits 8 1 64 8\n"
                 "radix_bits 4 0 32 4\n"
                 "batch_small_cutoff 2048\n")
    rc, h = _host_ctx(ahs, t)
    assert rc == ahs.AHS_OK
    try:
        assert _plan(ahs, h, (1 << 36) - 1) == (4, 9)      # 36 bits, r <= 11: 4 passes of 9
        assert _plan(ahs, h, (1 << 33) - 1) == (3, 11)     # 33 bits: 3 x 11
        assert _plan(ahs, h, (1 << 40) - 1) == (4, 10)     # 40 bits: 4 x 10
        assert _plan(ahs, h, (1 << 41) - 1) == (6, 7)      # past the first row: r <= 8
        assert _plan(ahs, h, (1 << 32) - 1, 4, 0) == (8, 4)
        assert _plan(ahs, h, (1 << 32) - 1, 4, 1) == (4, 8)  # no row: default base 256
        # a malformed table is refused and leaves the loaded one in place
        bad = tmp_path / "bad.txt"
        bad.write_text("ahs-tuning 1\nradix_bits 8 1 40 12\n")
        assert ahs.lib.ahs_load_tuning(h, os.fsencode(str(bad))) == ahs.AHS_ERR_NOT_FOUND
        assert _plan(ahs, h, (1 << 36) - 1) == (4, 9)
        assert ahs.lib.ahs_load_tuning(h, os.fsencode(str(tmp_path / "missing.txt"))) == \
            ahs.AHS_ERR_NOT_FOUND
        # NULL: back to the compiled defaults
        assert ahs.lib.ahs_load_tuning(h, None) == ahs.AHS_OK
        assert _plan(ahs, h, (1 << 36) - 1) == (5, 8)
    finally:
        ahs.lib.ahs_destroy(h)


@pytest.mark.parametrize("text", ["", "ahs-tuning 2\n", "ahs-tuning 1\nradix_bits 3 0 32 8\n",
                                  "ahs-tuning 1\nbatch_small_cutoff 9000\n",
                                  "ahs-tuning 1\nunknown_key 1\n"])
def test_malformed_tables_refused_at_create(tmp_path, text):
    import paper_2506_20677_gb300 as ahs
    t = tmp_path / "t.txt"
    t.write_text(text)
    rc, h = _host_ctx(ahs, t)
    assert rc == ahs.AHS_ERR_NOT_FOUND and not h.value


def test_shipped_table_loads_when_present():
    import paper_2506_20677_gb300 as ahs
    if not os.path.exists(ahs.SHIPPED_TUNING):
        pytest.skip("no tuned table shipped")
    rc, h = _host_ctx(ahs, ahs.SHIPPED_TUNING)
    assert rc == ahs.AHS_OK
    try:
        for kb in (4, 8):
            for pay in (0, 1):
                for D in range(1, 8 * kb + 1):
                    p, b = _plan(ahs, h, (1 << D) - 1, kb, pay)
                    assert 1 <= b <= 11 and p * b >= D and p <= 8
    finally:
        ahs.lib.ahs_destroy(h)
