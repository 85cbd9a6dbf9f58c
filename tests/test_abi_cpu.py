"""The C ABI without a GPU: the library loads, exports every declared entry
point, and its host-side logic (the selector) agrees with the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

from conftest import ROOT, read_golden

HEADER = os.path.join(ROOT, "include", "ahs.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(ahs_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def ahs():
    import paper_2506_20677_gb300 as m
    return m


def test_library_exports_every_declared_symbol(ahs):
    declared = _declared_functions()
    assert len(declared) >= 20
    raw = ctypes.CDLL(ahs.LIB_PATH)
    missing = [n for n in declared if not hasattr(raw, n)]
    assert not missing, missing
    unbound = [n for n in declared if n not in ahs.SIGNATURES]
    assert not unbound, unbound


def test_status_strings(ahs):
    for s in range(11):
        assert ahs.lib.ahs_status_str(s)
    assert b"integer" in ahs.lib.ahs_status_str(ahs.AHS_ERR_DTYPE)


def test_default_config_and_profiles(ahs):
    cfg = ahs.ahs_config_t()
    ahs.lib.ahs_default_config(ctypes.byref(cfg))
    assert cfg.select_mode == ahs.AHS_SEL_GB300
    p = ahs.profile_thresholds(ahs.AHS_SEL_PAPER)
    assert (p.n_t, p.k_t, p.k_max, p.h_max, p.use_entropy) == (20, 1000, 10**6, 0.7, 1)
    l6 = ahs.profile_thresholds(ahs.AHS_SEL_LISTING6)
    assert l6.use_entropy == 0
    g = ahs.profile_thresholds(ahs.AHS_SEL_GB300)
    assert g.k_t == 65536 and g.sorted_identity == 1
    assert g.n_t <= ahs.lib.ahs_small_capacity(ahs.AHS_U64, 1)
    t = ahs.ahs_thresholds_t()
    assert ahs.lib.ahs_profile_thresholds(ahs.AHS_SEL_CUSTOM, ctypes.byref(t)) == ahs.AHS_ERR_INVALID_ARG


def _feat(ahs, n, span, h, desc):
    f = ahs.ahs_features_t()
    f.n, f.span, f.entropy_norm, f.descents, f.nbins = n, span, h, desc, 65536
    return f


NAMES = {"IDENTITY": 1, "SMALL": 2, "COUNTING": 3, "RADIX": 4, "GENERAL": 5}


@pytest.mark.parametrize("row", read_golden("fsm_decisions.txt"), ids=lambda r: "-".join(r[:3]))
def test_library_fsm_decision_table(ahs, row):
    profile, n, span, h, desc, expect = row
    mode = {"PAPER": ahs.AHS_SEL_PAPER, "LISTING6": ahs.AHS_SEL_LISTING6}[profile]
    t = ahs.profile_thresholds(mode)
    assert ahs.select_fsm(_feat(ahs, int(n), int(span), float(h), int(desc)), t) == NAMES[expect]


def test_library_fsm_matches_oracle_random(ahs, orc):
    rng = np.random.default_rng(0)
    profiles = [
        (ahs.profile_thresholds(ahs.AHS_SEL_PAPER), orc.PAPER),
        (ahs.profile_thresholds(ahs.AHS_SEL_LISTING6), orc.LISTING6),
    ]
    g = ahs.profile_thresholds(ahs.AHS_SEL_GB300)
    profiles.append((g, orc.Profile(g.n_t, g.k_t, g.k_max, g.h_max, bool(g.use_entropy),
                                    bool(g.sorted_identity))))
    edges_n = [0, 1, 2, 19, 20, 21, 4095, 4096, 4097, 10**6]
    edges_span = [0, 1, 998, 999, 1000, 65534, 65535, 65536, 999999, 10**6, 2**32 - 1, 2**64 - 1]
    for _ in range(4000):
        n = int(rng.choice(edges_n)) if rng.random() < 0.5 else int(rng.integers(0, 10**7))
        span = int(rng.choice(edges_span)) if rng.random() < 0.5 else int(rng.integers(0, 2**40))
        h = float(rng.choice([0.0, 0.5, 0.7, np.nextafter(0.7, 0), 1.0])) if rng.random() < 0.5 \
            else float(rng.random())
        desc = int(rng.choice([0, 1, 5]))
        for lt, op in profiles:
            lf = _feat(ahs, n, span, h, desc)
            of = orc.Features()
            of.n, of.span, of.entropy_norm, of.descents, of.nbins = n, span, h, desc, 65536
            assert ahs.select_fsm(lf, lt) == orc.select(of, op), (n, span, h, desc)


def test_binding_refuses_float_keys(ahs):
    torch = pytest.importorskip("torch")
    with pytest.raises(ahs.AhsError) as e:
        ahs.key_type_of(torch.zeros(4, dtype=torch.float32))
    assert e.value.status == ahs.AHS_ERR_DTYPE


def test_invalid_arguments_without_gpu(ahs):
    """Argument checks happen before any device work."""
    f = ahs.ahs_features_t()
    assert ahs.lib.ahs_features(None, None, 0, 0, None, ctypes.byref(f)) == ahs.AHS_ERR_INVALID_ARG
    assert ahs.lib.ahs_sort(None, None, None, None, None, 0, 0, 0, None, None) == ahs.AHS_ERR_INVALID_ARG
    assert ahs.lib.ahs_select_fsm(None, None, None) == ahs.AHS_ERR_INVALID_ARG
