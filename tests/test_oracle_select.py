"""Pins for the oracle's decision state machine (Section III-A, Listing 6)."""
import pytest

from conftest import read_golden

NAMES = {"IDENTITY": 1, "SMALL": 2, "COUNTING": 3, "RADIX": 4, "GENERAL": 5}


@pytest.mark.parametrize("row", read_golden("fsm_decisions.txt"),
                         ids=lambda r: "-".join(r[:3]))
def test_decision_table(orc, row):
    profile, n, span, h, desc, expect = row
    f = orc.Features()
    f.n, f.span, f.entropy_norm, f.descents = int(n), int(span), float(h), int(desc)
    f.nbins = 65536
    p = getattr(orc, profile)
    assert orc.select(f, p) == NAMES[expect]


def test_sorted_identity_flag(orc):
    f = orc.Features()
    f.n, f.span, f.entropy_norm, f.descents = 10**6, 2**32 - 1, 1.0, 0
    assert orc.select(f, orc.PAPER) == NAMES["GENERAL"]
    p = orc.Profile(20, 1000, 10**6, sorted_identity=True)
    assert orc.select(f, p) == NAMES["IDENTITY"]
    f.descents = 1
    assert orc.select(f, p) == NAMES["GENERAL"]
