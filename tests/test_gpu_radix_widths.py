"""Stable LSD radix with digits of 4 to 11 bits (Eq. 4 with base 2^r) against
the oracle: the tuned-shape table sets the largest digit width; keys and
payload permutations must be bit-exact for every width, key type and range,
including ragged tiles and in-place sorts."""
import numpy as np
import pytest

import oracle
from gpu_util import dev, host, key_type

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ahs():
    import paper_2506_20677_gb300 as m
    return m


def _table(tmp_path, bits):
    p = tmp_path / f"r{bits}.txt"
    rows = "".join(f"radix_bits {kb} {pay} 64 {bits}\n" for kb in (4, 8) for pay in (0, 1))
    p.write_text("ahs-tuning 1\n" + rows)
    return str(p)


def _keys(dt, n, span_bits, seed):
    rng = np.random.default_rng(seed)
    info = np.iinfo(dt)
    lo = int(info.min) // 3
    hi = lo + (1 << span_bits) - 1
    a = rng.integers(lo, hi, size=n, dtype=dt, endpoint=True)
    a[rng.integers(0, n, size=max(1, n // 50))] = dt(lo)       # duplicates of the minimum
    a[0], a[-1] = dt(lo), dt(hi)                                 # the full span is present
    return a


@pytest.mark.parametrize("bits", [4, 8, 9, 10, 11])
def test_widths_against_oracle(ahs, tmp_path, bits):
    import torch
    with ahs.Context(0, tuning_path=_table(tmp_path, bits)) as ctx:
        cases = [(np.uint32, 32, 300_007), (np.int32, 21, 70_001), (np.uint64, 36, 200_003),
                 (np.int64, 63, 50_000), (np.uint64, 13, 4_097)]
        for i, (dt, span_bits, n) in enumerate(cases):
            a = _keys(dt, n, span_bits, 100 * bits + i)
            v = np.arange(n, dtype=np.uint32)[::-1].copy()
            p, b = ctx.radix_plan((1 << span_bits) - 1, np.dtype(dt).itemsize, True)
            assert b <= bits and p == -(-span_bits // bits) if span_bits // bits < 8 else True
            ko, vo = oracle.radix_sort(a, v)
            r = ctx.sort(dev(a), vals=dev(v), force=ahs.AHS_RADIX, key_type=key_type(a))
            torch.cuda.synchronize()
            assert r.info.passes == p, (dt, span_bits)
            assert np.array_equal(host(r.keys, dt), ko), (bits, dt, span_bits)
            assert np.array_equal(host(r.vals, np.uint32), vo), (bits, dt, span_bits)
            # keys only through the same stable passes (counting range keys too)
            kk = ctx.sort(dev(a), force=ahs.AHS_RADIX, key_type=key_type(a))
            torch.cuda.synchronize()
            assert np.array_equal(host(kk.keys, dt), ko)
        # in place, odd and even pass counts
        for span_bits in (27, 33):
            a = _keys(np.uint64, 123_457, span_bits, bits + span_bits)
            v = np.arange(len(a), dtype=np.uint32)
            ko, vo = oracle.radix_sort(a, v)
            dk, dv = dev(a), dev(v)
            ctx.sort(dk, vals=dv, out=dk, vals_out=dv, force=ahs.AHS_RADIX, key_type=ahs.AHS_U64)
            torch.cuda.synchronize()
            assert np.array_equal(host(dk, np.uint64), ko) and np.array_equal(host(dv, np.uint32), vo)
