"""The MODEL profile's policy (Section III-H, Table IV) pinned by a hand-written
decision table.

tests/golden/model_policy.txt lists (n, k, h, descents, capacity) -> strategy
as Table IV states the split between static thresholds and the learned model,
with a hand-written one-tree table (tests/golden/model_policy_trees.txt) whose
pick depends on h alone.  The oracle and the library (a host-only context, no
GPU) are each checked against the table, not against one another.
"""
import ctypes
import os

import pytest

from conftest import GOLDEN, read_golden

NAMES = {"IDENTITY": 1, "SMALL": 2, "COUNTING": 3, "RADIX": 4, "GENERAL": 5}
TREES = os.path.join(GOLDEN, "model_policy_trees.txt")
# The GB300 rules the policy falls back to (Table IV's "static thresholds" for
# what n <= 20 and k <= 500 leave), as the oracle is given them.
GB300_RULES = dict(n_t=4096, k_t=65536, k_max=10**6, h_max=0.7, use_entropy=True,
                   sorted_identity=True)


def _rows():
    return [(int(n), int(span), float(h), int(d), int(cap), NAMES[e])
            for n, span, h, d, cap, e in read_golden("model_policy.txt")]


def test_tree_table_picks_by_h(orc):
    m = orc.Model(TREES)
    for h, want in ((0.1, 3), (0.14, 3), (0.3, 2), (0.5, 4), (0.7, 5), (0.9, 1)):
        assert m.predict([12.0, 20.0, h, 4.0, 0.0]) == want, h


@pytest.mark.parametrize("row", _rows())
def test_oracle_policy(orc, row):
    n, span, h, desc, cap, want = row
    m = orc.Model(TREES)
    f = orc.Features()
    f.n, f.span, f.entropy_norm, f.descents, f.nbins = n, span, h, desc, 65536
    assert m.select(f, 4, False, orc.Profile(**GB300_RULES), cap) == want


def test_library_policy():
    import paper_2506_20677_gb300 as ahs
    g = ahs.profile_thresholds(ahs.AHS_SEL_GB300)
    assert (g.n_t, g.k_t, g.k_max, bool(g.sorted_identity)) == (4096, 65536, 10**6, True)
    cfg = ahs.ahs_config_t()
    ahs.lib.ahs_default_config(ctypes.byref(cfg))
    cfg.device = -1
    cfg.select_mode = ahs.AHS_SEL_MODEL
    cfg.model_path = os.fsencode(TREES)
    h = ctypes.c_void_p()
    ahs.check(ahs.lib.ahs_create(ctypes.byref(h), ctypes.byref(cfg)), "ahs_create(host-only)")
    try:
        cap = int(ahs.lib.ahs_small_capacity(ahs.AHS_U32, 0))
        checked = 0
        for n, span, hh, desc, rcap, want in _rows():
            if rcap != cap:   # the library's one-block capacity is fixed
                continue
            f = ahs.ahs_features_t()
            f.n, f.span, f.entropy_norm, f.descents, f.nbins = n, span, hh, desc, 65536
            out = ctypes.c_int()
            ahs.check(ahs.lib.ahs_select(h, ctypes.byref(f), ahs.AHS_SEL_MODEL, 4, 0,
                                         ctypes.byref(out)), "ahs_select")
            assert out.value == want, (n, span, hh, desc)
            checked += 1
        assert checked >= 20
    finally:
        ahs.lib.ahs_destroy(h)
