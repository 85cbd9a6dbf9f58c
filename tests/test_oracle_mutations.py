"""The pins must catch plausible mistakes in the oracle.

Each case plants one mistake in a copy of oracle/ahs_oracle.c (a flipped sign,
a dropped term, a wrong index, a non-strict comparison), builds it with gcc,
and checks that at least one of the oracle's pins fails on the broken build.
The shipped oracle is never modified.
"""
import os
import shutil
import subprocess
import sys

import numpy as np
import pytest

import oracle
from conftest import read_golden
from test_oracle_features import _expand, DT

NAMES = {"IDENTITY": 1, "SMALL": 2, "COUNTING": 3, "RADIX": 4, "GENERAL": 5}

MUTATIONS = {
    "entropy_sign": [("H -= p * log2(p);", "H += p * log2(p);")],
    "entropy_norm_by_k": [("H / log2((double)nbins)", "H / log2((double)span + 1.0)")],
    "bin_width_15": [("bl > 16 ? bl - 16 : 0", "bl > 15 ? bl - 15 : 0")],
    "bins_without_min": [("uint64_t u = (uint64_t)(load_key(keys, i, t) - mn);",
                          "uint64_t u = (uint64_t)(load_key(keys, i, t));")],
    "descent_non_strict": [("if (x > y) ++descents;", "if (x >= y) ++descents;")],
    "ascent_non_strict": [("if (x < y) ++ascents;", "if (x <= y) ++ascents;")],
    "reverse_ignores_tied_payload": [("(!vals || f.descents == n - 1))", "1)")],
    "reverse_under_every_profile": [("if (fsm->sorted_identity && n >= 2", "if (n >= 2")],
    "insertion_unstable": [("a[j - 1] > key", "a[j - 1] >= key")],
    "counting_reverse_placement": [("for (uint64_t i = 0; i < n; ++i) {       /* input order",
                                    "for (uint64_t i = n; i-- > 0;) {       /* input order")],
    "counting_inclusive_start": [("start[c] = before;\n        before += count;",
                                  "before += count;\n        start[c] = before - 1;")],
    "model_rules_at_1000": [("if (f->n < 1000 || !m) {", "if (f->n <= 1000 || !m) {")],
    "model_small_counting_strict": [("else if (k <= 500) s = ORC_COUNTING;",
                                     "else if (k < 500) s = ORC_COUNTING;")],
    "model_counting_clamp_off_by_one": [("if (s == ORC_COUNTING && k > 65536)",
                                         "if (s == ORC_COUNTING && k > 65537)")],
    "model_small_clamp_dropped": [("if (s == ORC_SMALL && f->n > rules->n_t) s = ORC_GENERAL;", "")],
    "model_identity_after_trees": [("} else if (f->span == 0 || (rules->sorted_identity && f->descents == 0)) {\n        s = ORC_IDENTITY;\n    } else {",
                                    "} else {")],
    "radix_digit_stride": [("(u >> (8 * digit)) & 255] += 1", "(u >> (7 * digit)) & 255] += 1"),
                           ("(u >> (8 * digit)) & 255]++", "(u >> (7 * digit)) & 255]++")],
    "radix_without_min": [("uint64_t u = (uint64_t)(a[i] - mn);\n            bucket_size",
                           "uint64_t u = (uint64_t)(a[i]);\n            bucket_size"),
                          ("uint64_t u = (uint64_t)(a[i] - mn);\n            uint64_t pos",
                           "uint64_t u = (uint64_t)(a[i]);\n            uint64_t pos")],
    "radix_passes_off_by_one": [("while (reach < k)", "while (reach <= k / 256)")],
    "quick_drops_pivot_copies": [("else if (a[i] == pivot) tmp[ie++] = a[i];",
                                  "else if (a[i] == pivot) { tmp[ie] = a[i]; }")],
    "merge_unstable": [("if (a[j] < a[i])", "if (a[j] <= a[i])")],
    "fsm_counting_strict": [("if (k <= (uval_t)p->k_t)", "if (k < (uval_t)p->k_t)")],
    "fsm_radix_non_strict": [("f->entropy_norm < p->h_max", "f->entropy_norm <= p->h_max")],
    "fsm_kmax_non_strict": [("k > (uval_t)p->k_max", "k >= (uval_t)p->k_max")],
    "fsm_small_before_identity": [("if (f->n <= 1) return ORC_IDENTITY;", "if (f->n < 1) return ORC_IDENTITY;")],
}


def _pins_pass() -> bool:
    """Run a fast subset of the oracle pins against the currently loaded build."""
    try:
        for row in read_golden("entropy_closed_forms.txt"):
            _, typ, runs, H, h, shift, nbins = row
            keys = _expand(runs, DT[typ])
            keys = keys[np.random.default_rng(len(keys)).permutation(len(keys))]
            f = oracle.features(keys)
            if f.shift != int(shift) or f.nbins != int(nbins):
                return False
            if abs(f.entropy - float(H)) > 1e-12 or abs(f.entropy_norm - float(h)) > 1e-12:
                return False
            if f.descents != int(np.count_nonzero(keys[:-1] > keys[1:])):
                return False
            if f.ascents != int(np.count_nonzero(keys[:-1] < keys[1:])):
                return False
        # Reversed inputs (Section III-B's descending presorted case) under
        # rules that return presorted inputs by a copy: keys only with ties,
        # a payload only when strictly decreasing; never under PAPER.
        rng = np.random.default_rng(1)
        gb = oracle.Profile(4096, 65536, 10**6, sorted_identity=True)
        tied = np.sort(rng.integers(0, 50, size=300).astype(np.uint32))[::-1].copy()
        strict = np.sort(rng.choice(10**6, size=300, replace=False).astype(np.uint32))[::-1].copy()
        v = np.arange(300, dtype=np.uint32)
        k, _, ch, f = oracle.sort(tied, profile=gb)
        if ch != oracle.REVERSE or f.ascents != 0 or not np.array_equal(k, np.sort(tied)):
            return False
        k, vo, ch, _ = oracle.sort(tied, v, profile=gb)
        exp_v = np.array(sorted(range(300), key=lambda i: tied[i]), dtype=np.uint32)
        if ch == oracle.REVERSE or not np.array_equal(vo, exp_v):
            return False
        k, vo, ch, _ = oracle.sort(strict, v, profile=gb)
        if ch != oracle.REVERSE or not np.array_equal(vo, v[::-1]) or not np.array_equal(k, np.sort(strict)):
            return False
        if oracle.sort(tied, profile=oracle.PAPER)[2] == oracle.REVERSE:
            return False
        for row in read_golden("fsm_decisions.txt"):
            profile, n, span, h, desc, expect = row
            f = oracle.Features()
            f.n, f.span, f.entropy_norm, f.descents, f.nbins = int(n), int(span), float(h), int(desc), 65536
            if oracle.select(f, getattr(oracle, profile)) != NAMES[expect]:
                return False
        m = oracle.Model(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                      "model_policy_trees.txt"))
        rules = oracle.Profile(4096, 65536, 10**6, sorted_identity=True)
        for row in read_golden("model_policy.txt"):
            n, span, h, desc, cap, expect = row
            f = oracle.Features()
            f.n, f.span, f.entropy_norm, f.descents, f.nbins = int(n), int(span), float(h), int(desc), 65536
            if m.select(f, 4, False, rules, int(cap)) != NAMES[expect]:
                return False
        for row in read_golden("radix_passes_eq4.txt"):
            if oracle.radix_passes(int(row[0]) - 1) != int(row[1]):
                return False
        rng = np.random.default_rng(0)
        for dt in (np.uint32, np.int64):
            for lo, hi in ((0, 200), (-2**40 if dt == np.int64 else 0, 2**31)):
                keys = rng.integers(lo, hi, size=600, dtype=dt)
                vals = np.arange(600, dtype=np.uint32)
                exp_k = np.array(sorted(keys.tolist()), dtype=dt)
                exp_v = np.array(sorted(range(600), key=lambda i: keys[i]), dtype=np.uint32)
                fns = [oracle.radix_sort, oracle.merge_sort, oracle.insertion_sort]
                if hi - lo <= 200:
                    fns.append(oracle.counting_sort)
                for fn in fns:
                    ko, vo = fn(keys, vals)
                    if not (np.array_equal(ko, exp_k) and np.array_equal(vo, exp_v)):
                        return False
                if not np.array_equal(oracle.quicksort(keys), exp_k):
                    return False
        return True
    except RuntimeError:
        return False


def test_pins_pass_on_shipped_oracle():
    oracle.lib()
    assert _pins_pass()


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, name):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "ahs_oracle.c")).read()
    for old, new in MUTATIONS[name]:
        assert old in src, f"mutation anchor not found: {old!r}"
        src = src.replace(old, new)
    d = tmp_path / name
    d.mkdir()
    shutil.copy(os.path.join(os.path.dirname(oracle.__file__), "ahs_oracle.h"), d)
    (d / "ahs_oracle.c").write_text(src)
    so = str(d / "libmut.so")
    subprocess.check_call(["gcc", "-O1", "-std=gnu99", "-fPIC", "-shared", "-o", so,
                           str(d / "ahs_oracle.c"), "-lm"])
    # A planted out-of-bounds write may crash the process: run the pins in a child.
    tests_dir = os.path.dirname(os.path.abspath(__file__))
    code = ("import sys; sys.path[:0] = [%r, %r]\n"
            "import oracle, test_oracle_mutations as m\n"
            "with oracle.using_library(%r):\n"
            "    sys.exit(0 if m._pins_pass() else 3)\n") % (tests_dir, os.path.dirname(tests_dir), so)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert r.returncode != 0, f"planted mistake {name} was not caught by any pin"
    assert r.returncode == 3 or r.returncode < 0, r.stderr[-2000:]
