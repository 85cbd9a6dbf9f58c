"""Keys-only radix path for inputs with few distinct values (the sparse
counting sort: hash-table counts, ranks, run-by-run fill), against the oracle.

Covers the four key types, distinct counts from 2 to the table's reach,
Zipf-skewed and even counts, ragged sizes, misaligned and in-place buffers,
the span limit (no key may map to the table's empty marker), and inputs whose
distinct values overflow the tables (the partition passes then sort them).
The trace shows which path ran."""
import numpy as np
import pytest

import oracle
from gpu_util import dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ahs():
    import paper_2506_20677_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(ahs):
    c = ahs.Context(0)
    yield c
    c.close()


KT = {"u32": ("AHS_U32", np.uint32), "i32": ("AHS_I32", np.int32),
      "u64": ("AHS_U64", np.uint64), "i64": ("AHS_I64", np.int64)}


def _values(rng, m, dtype):
    bits = np.dtype(dtype).itemsize * 8
    raw = rng.integers(0, 2**bits - 1, size=4 * m, dtype=np.uint64 if bits == 64 else np.uint32)
    vals = np.unique(raw)[:m]
    rng.shuffle(vals)
    return vals.view(dtype) if np.dtype(dtype).kind == "i" else vals.astype(dtype)


def _zipf_keys(rng, n, vals, s=1.1):
    p = np.arange(1, len(vals) + 1, dtype=np.float64) ** -s
    p /= p.sum()
    return vals[rng.choice(len(vals), size=n, p=p)]


def _sort(ahs, ctx, a, kt, out=None):
    import torch
    ctx.trace(True)
    d = dev(a)
    if out == "inplace":
        r = ctx.sort(d, out=d, force=ahs.AHS_RADIX, key_type=getattr(ahs, kt))
    else:
        r = ctx.sort(d, force=ahs.AHS_RADIX, key_type=getattr(ahs, kt))
    torch.cuda.synchronize()
    ctx.trace(False)
    names = [t[0] for t in ctx.trace_collect()]
    return host(r.keys, a.dtype), names


@pytest.mark.parametrize("kt", list(KT))
@pytest.mark.parametrize("m", [2, 37, 1024, 2000])
def test_sparse_zipf_against_oracle(ahs, ctx, kt, m):
    name, dtype = KT[kt]
    rng = np.random.default_rng(1000 + m)
    n = (1 << 20) + 37
    a = _zipf_keys(rng, n, _values(rng, m, dtype))
    got, names = _sort(ahs, ctx, a, name)
    assert np.array_equal(got, oracle.radix_sort(a))
    assert "sparse_fill" in names and "msd_scatter" not in names, names


@pytest.mark.parametrize("kt", ["u32", "u64"])
def test_sparse_even_counts_inplace(ahs, ctx, kt):
    name, dtype = KT[kt]
    rng = np.random.default_rng(7)
    n = (1 << 19) + 5
    vals = _values(rng, 500, dtype)
    a = vals[rng.integers(0, len(vals), size=n)]
    got, names = _sort(ahs, ctx, a, name, out="inplace")
    assert np.array_equal(got, oracle.radix_sort(a))
    assert "sparse_fill" in names


def test_sparse_misaligned_buffers(ahs, ctx):
    import torch
    rng = np.random.default_rng(8)
    n = (1 << 20) + 3
    a = _zipf_keys(rng, n, _values(rng, 300, np.uint32))
    big = torch.zeros(n + 8, dtype=torch.int32, device="cuda")
    src = big[1:n + 1]
    src.copy_(torch.from_numpy(a.view(np.int32)))
    obig = torch.zeros(n + 8, dtype=torch.int32, device="cuda")
    out = obig[3:n + 3]
    r = ctx.sort(src, out=out, force=ahs.AHS_RADIX, key_type=ahs.AHS_U32)
    torch.cuda.synchronize()
    assert np.array_equal(host(r.keys, np.uint32), oracle.radix_sort(a))
    # nothing written outside the output window
    assert int(obig[:3].abs().sum()) == 0 and int(obig[n + 3:].abs().sum()) == 0


def test_span_limit(ahs, ctx):
    """A span of 2^32 - 2 still fits the table's key encoding; the full
    2^32 - 1 span does not and takes the partition passes."""
    rng = np.random.default_rng(9)
    n = 1 << 19
    vals = _values(rng, 60, np.uint32)
    vals[0], vals[1] = 0, 0xFFFFFFFE
    a = _zipf_keys(rng, n, vals)
    a[:2] = [0, 0xFFFFFFFE]
    got, names = _sort(ahs, ctx, a, "AHS_U32")
    assert np.array_equal(got, oracle.radix_sort(a))
    assert "sparse_fill" in names
    a[5] = 0xFFFFFFFF
    got, names = _sort(ahs, ctx, a, "AHS_U32")
    assert np.array_equal(got, oracle.radix_sort(a))
    assert "sparse_count" not in names and "msd_scatter" in names


def test_overflow_falls_back(ahs, ctx):
    """64 histogram bins holding 40,000 distinct values: the tables overflow,
    the fill writes nothing and the partition passes sort the keys."""
    rng = np.random.default_rng(10)
    n = 1 << 20
    bins = rng.choice(1 << 16, size=64, replace=False).astype(np.uint64)
    offs = rng.integers(0, 1 << 16, size=40_000, dtype=np.uint64)
    vals = np.unique(((bins[rng.integers(0, 64, size=40_000)] << np.uint64(16)) + offs)
                     .astype(np.uint32))
    a = vals[rng.integers(0, len(vals), size=n)]
    a[0], a[1] = 0, 0xFFFF0000   # a full-width span: bins of 2^16 values
    got, names = _sort(ahs, ctx, a, "AHS_U32")
    assert np.array_equal(got, oracle.radix_sort(a))
    assert "sparse_count" in names and "msd_scatter" in names, names


def test_config2b_picks_sparse(ahs, ctx):
    """Config 2(b)'s shape (1,024 Zipf(1.1) values) at 1/64 scale."""
    from gen import host as gen
    a = gen.config2("b", (1 << 28) // 64)
    got, names = _sort(ahs, ctx, a, "AHS_U32")
    assert np.array_equal(got, oracle.radix_sort(a))
    assert "sparse_fill" in names
