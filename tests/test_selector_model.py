"""The learned selector (Section III-H, Table IV).

scikit-learn's own predict pins the oracle's tree-table evaluator; the
library's evaluator (host-only context, no GPU) must then pick what the
oracle picks, including at split thresholds."""
import ctypes
import os

import numpy as np
import pytest

from conftest import ROOT

SHIPPED = os.path.join(ROOT, "paper_2506_20677_gb300", "selector", "ahs_trees.txt")


@pytest.fixture(scope="module")
def trained(tmp_path_factory):
    pytest.importorskip("sklearn")
    from paper_2506_20677_gb300.selector import train_trees as tt
    rng = np.random.default_rng(0)
    n = 600
    X = np.column_stack([rng.uniform(10, 28, n), rng.uniform(1, 64, n), rng.uniform(0, 1, n),
                         rng.choice([4.0, 8.0], n), rng.choice([0.0, 1.0], n)])
    # a plausible labelling rule plus noise, classes 3 (counting), 4 (radix), 5 (general)
    y = np.where(X[:, 1] <= 16, 3, np.where(X[:, 2] < 0.6, 4, 5))
    flip = rng.random(n) < 0.05
    y[flip] = rng.choice([3, 4, 5], flip.sum())
    model = tt.fit(X, y, n_estimators=12, max_depth=3)
    path = tmp_path_factory.mktemp("model") / "trees.txt"
    path.write_text(tt.to_table(model))
    return model, str(path), X


def test_oracle_evaluator_equals_sklearn(orc, trained):
    model, path, X = trained
    m = orc.Model(path)
    rng = np.random.default_rng(1)
    pts = np.column_stack([rng.uniform(5, 30, 3000), rng.uniform(0, 66, 3000), rng.uniform(0, 1, 3000),
                           rng.choice([4.0, 8.0], 3000), rng.choice([0.0, 1.0], 3000)])
    # points exactly at split thresholds exercise the <= rule
    thr = []
    for stage in model.estimators_:
        for est in stage:
            t = est.tree_
            for i in range(t.node_count):
                if t.children_left[i] != -1:
                    p = X[i % len(X)].copy()
                    p[t.feature[i]] = t.threshold[i]
                    thr.append(p)
    pts = np.vstack([pts, np.array(thr)])
    ref = model.predict(pts)
    got = np.array([m.predict(p) for p in pts])
    assert np.array_equal(got, ref)


def _host_ctx(ahs, path):
    cfg = ahs.ahs_config_t()
    ahs.lib.ahs_default_config(ctypes.byref(cfg))
    cfg.device = -1
    cfg.select_mode = ahs.AHS_SEL_MODEL
    cfg.model_path = os.fsencode(path)
    h = ctypes.c_void_p()
    ahs.check(ahs.lib.ahs_create(ctypes.byref(h), ctypes.byref(cfg)), "ahs_create(host-only)")
    return h


def _compare_library_with_oracle(orc, path, seed):
    import paper_2506_20677_gb300 as ahs
    h = _host_ctx(ahs, path)
    g = ahs.profile_thresholds(ahs.AHS_SEL_GB300)
    rules = orc.Profile(g.n_t, g.k_t, g.k_max, g.h_max, bool(g.use_entropy), bool(g.sorted_identity))
    m = orc.Model(path)
    rng = np.random.default_rng(seed)
    try:
        for _ in range(4000):
            n = int(2 ** rng.uniform(0, 30))
            span = int(2 ** rng.uniform(0, 64)) - 1 if rng.random() < 0.9 else int(rng.integers(0, 70000))
            h_ = float(rng.random())
            desc = int(rng.choice([0, 3]))
            kb = int(rng.choice([4, 8]))
            pay = bool(rng.random() < 0.3)
            lf = ahs.ahs_features_t()
            lf.n, lf.span, lf.entropy_norm, lf.descents, lf.nbins = n, span, h_, desc, 65536
            of = orc.Features()
            of.n, of.span, of.entropy_norm, of.descents, of.nbins = n, span, h_, desc, 65536
            out = ctypes.c_int()
            ahs.check(ahs.lib.ahs_select(h, ctypes.byref(lf), ahs.AHS_SEL_MODEL, kb, int(pay),
                                         ctypes.byref(out)), "ahs_select")
            cap = int(ahs.lib.ahs_small_capacity(ahs.AHS_U64 if kb == 8 else ahs.AHS_U32, int(pay)))
            assert out.value == m.select(of, kb, pay, rules, cap), (n, span, h_, desc, kb, pay)
    finally:
        ahs.lib.ahs_destroy(h)


def test_library_model_select_equals_oracle(orc, trained):
    _compare_library_with_oracle(orc, trained[1], 2)


@pytest.mark.skipif(not os.path.exists(SHIPPED), reason="no trained table shipped yet")
def test_shipped_table_library_equals_oracle(orc):
    _compare_library_with_oracle(orc, SHIPPED, 3)


def test_host_only_context_refuses_device_work():
    import paper_2506_20677_gb300 as ahs
    cfg = ahs.ahs_config_t()
    ahs.lib.ahs_default_config(ctypes.byref(cfg))
    cfg.device = -1
    h = ctypes.c_void_p()
    ahs.check(ahs.lib.ahs_create(ctypes.byref(h), ctypes.byref(cfg)), "ahs_create")
    f = ahs.ahs_features_t()
    assert ahs.lib.ahs_features(h, ctypes.c_void_p(1), 4, ahs.AHS_U32, None, ctypes.byref(f)) == \
        ahs.AHS_ERR_INVALID_ARG
    assert ahs.lib.ahs_sort(h, ctypes.c_void_p(1), ctypes.c_void_p(1), None, None, 4, ahs.AHS_U32,
                            0, None, None) == ahs.AHS_ERR_INVALID_ARG
    ahs.lib.ahs_destroy(h)


@pytest.mark.skipif(not os.path.exists(SHIPPED), reason="no trained table shipped yet")
def test_shipped_table_matches_its_labels(orc):
    """The shipped table, evaluated by the oracle, reproduces most of the GB300
    timing labels it was trained on (n >= 1000 rows; Table IV)."""
    import json
    from paper_2506_20677_gb300.selector import train_trees as tt
    labels = os.path.join(ROOT, "paper_2506_20677_gb300", "selector", "labels_gb300.json")
    rows, X, y = tt.load(labels)
    m = orc.Model(SHIPPED)
    hit = sum(int(m.predict(list(x)) == int(c)) for x, c in zip(X, y))
    assert hit >= 0.9 * len(rows), (hit, len(rows))
