"""Helpers for the GPU parity tests (host side only)."""
import numpy as np

SIGNED_VIEW = {np.dtype(np.uint32): np.int32, np.dtype(np.int32): np.int32,
               np.dtype(np.uint64): np.int64, np.dtype(np.int64): np.int64}


def key_type(a):
    import paper_2506_20677_gb300 as ahs
    return {np.dtype(np.uint32): ahs.AHS_U32, np.dtype(np.uint64): ahs.AHS_U64,
            np.dtype(np.int32): ahs.AHS_I32, np.dtype(np.int64): ahs.AHS_I64}[a.dtype]


def dev(a):
    """Host numpy array -> CUDA tensor holding the same bits (int32/int64 view)."""
    import torch
    a = np.ascontiguousarray(a)
    return torch.from_numpy(a.view(SIGNED_VIEW[a.dtype])).cuda()


def host(t, dtype):
    return t.cpu().numpy().view(dtype)


def mix64(x):
    x = x.astype(np.uint64)
    with np.errstate(over="ignore"):
        x = (x ^ (x >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        x = (x ^ (x >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return x ^ (x >> np.uint64(31))


def multiset_digest(a):
    """Order-independent digest of a multiset: wrapped sum and xor of a 64-bit
    mix of every element, plus the histogram of the top 16 bits."""
    m = mix64(a.view(np.uint32 if a.itemsize == 4 else np.uint64))
    with np.errstate(over="ignore"):
        s = int(np.sum(m, dtype=np.uint64))
    x = int(np.bitwise_xor.reduce(m)) if len(m) else 0
    u = a.view(np.uint32 if a.itemsize == 4 else np.uint64)
    top = (u >> np.uint64(8 * a.itemsize - 16)).astype(np.int64)
    return s, x, np.bincount(top, minlength=65536)


def order_key(a):
    """Values whose unsigned order is the key type's order."""
    if a.dtype == np.int32:
        return a.view(np.uint32) ^ np.uint32(0x80000000)
    if a.dtype == np.int64:
        return a.view(np.uint64) ^ np.uint64(0x8000000000000000)
    return a


def check_sorted_permutation(inp, out, samples=24, seed=0):
    """Exact properties of the sorted output at any size: non-decreasing,
    same multiset (digest), and sampled order statistics."""
    assert len(inp) == len(out)
    ko = order_key(out)
    assert np.all(ko[:-1] <= ko[1:]), "output not non-decreasing"
    si, xi, hi = multiset_digest(inp)
    so, xo, ho = multiset_digest(out)
    assert si == so and xi == xo and np.array_equal(hi, ho), "output is not a permutation"
    rng = np.random.default_rng(seed)
    ki = order_key(inp)
    for i in rng.integers(0, len(out), size=samples):
        v = ko[i]
        below = int(np.count_nonzero(ki < v))
        upto = int(np.count_nonzero(ki <= v))
        assert below <= i < upto, f"order statistic {i} wrong"


def check_stable_kv(kin, kout, vout):
    """With payload = original index, these properties fix the unique stable order."""
    n = len(kin)
    assert np.array_equal(np.bincount(vout.astype(np.int64), minlength=n), np.ones(n, np.int64))
    assert np.array_equal(kin[vout.astype(np.int64)], kout)
    ko = order_key(kout)
    assert np.all(ko[:-1] <= ko[1:])
    eq = ko[:-1] == ko[1:]
    assert np.all(vout[:-1][eq] < vout[1:][eq]), "equal keys out of input order"
