"""ahs_features_noalloc, the feature pass for callers that cannot allocate.

Some callers cannot call cudaMalloc when they need the features: their device
memory is all reserved up front by another allocator or pool, or they run on a
latency-bound path that cannot afford the synchronisation cudaMalloc / cudaFree
imply.  This entry point serves them; its scratch is a fixed array inside the
library.  Through the C ABI it must return what ahs_features returns for the
same keys, and what the oracle computes, on consecutive calls that reuse the
same scratch.  This file is collected last so that a failure here does not hide
the rest of the suite; it passes alone and after the other tests.
"""
import ctypes
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

ENT_REL, ENT_ABS = 1e-9, 1e-12   # the tolerance of the other parity tests


def _same(a, b):
    assert (a.n, a.min_bits, a.max_bits, a.span, a.hist_shift, a.nbins, a.descents) == \
        (b.n, b.min_bits, b.max_bits, b.span, b.hist_shift, b.nbins, b.descents)
    assert math.isclose(a.entropy_bits, b.entropy_bits, rel_tol=ENT_REL, abs_tol=ENT_ABS)
    assert math.isclose(a.entropy_norm, b.entropy_norm, rel_tol=ENT_REL, abs_tol=ENT_ABS)


def _same_as_oracle(a, o):
    assert (a.n, a.min_bits, a.max_bits, a.span, a.hist_shift, a.nbins, a.descents) == \
        (o.n, o.min_bits, o.max_bits, o.span, o.shift, o.nbins, o.descents)
    assert math.isclose(a.entropy_bits, o.entropy, rel_tol=ENT_REL, abs_tol=ENT_ABS)
    assert math.isclose(a.entropy_norm, o.entropy_norm, rel_tol=ENT_REL, abs_tol=ENT_ABS)


def _raw_noalloc(ahs, t, key_type):
    f = ahs.ahs_features_t()
    rc = ahs.lib.ahs_features_noalloc(ctypes.c_void_p(t.data_ptr()), t.numel(), key_type, None,
                                      ctypes.byref(f))
    return rc, f


def test_noalloc_matches_features_on_consecutive_calls():
    import torch
    import paper_2506_20677_gb300 as ahs
    rng = np.random.default_rng(2024)
    cases = [
        (rng.integers(0, 4096, size=(1 << 22) + 3, dtype=np.uint32), ahs.AHS_U32, torch.int32),
        (rng.integers(0, 2**32, size=(1 << 21) + 5, dtype=np.uint32), ahs.AHS_U32, torch.int32),
        (rng.integers(-2**62, 2**62, size=300_001, dtype=np.int64), ahs.AHS_I64, torch.int64),
    ]
    with ahs.Context(0) as ctx:
        for a, kt, tdt in cases:
            t = torch.from_numpy(a.view(np.int32 if a.itemsize == 4 else np.int64)).cuda()
            ref = ctx.features(t, key_type=kt)
            orc = oracle.features(a)
            for _ in range(2):          # two calls in a row reuse the same scratch
                rc, f = _raw_noalloc(ahs, t, kt)
                assert rc == ahs.AHS_OK
                _same(f, ref)
                _same_as_oracle(f, orc)


def test_noalloc_on_a_non_default_stream():
    """The work runs on the caller's stream, after the work already queued there."""
    import torch
    import paper_2506_20677_gb300 as ahs
    a = np.random.default_rng(7).integers(0, 2**32, size=(1 << 20) + 1, dtype=np.uint32)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        t = torch.from_numpy(a.view(np.int32)).to("cuda", non_blocking=False)
        t2 = t.clone()                      # queued on st before the call
    f = ahs.ahs_features_t()
    for _ in range(2):
        rc = ahs.lib.ahs_features_noalloc(ctypes.c_void_p(t2.data_ptr()), t2.numel(), ahs.AHS_U32,
                                          ctypes.c_void_p(st.cuda_stream), ctypes.byref(f))
        assert rc == ahs.AHS_OK
        _same_as_oracle(f, oracle.features(a))


def test_noalloc_edge_cases():
    import torch
    import paper_2506_20677_gb300 as ahs
    t = torch.zeros(16, dtype=torch.int32, device="cuda")
    f = ahs.ahs_features_t()
    # empty input
    assert ahs.lib.ahs_features_noalloc(ctypes.c_void_p(t.data_ptr()), 0, ahs.AHS_U32, None,
                                        ctypes.byref(f)) == ahs.AHS_OK and f.n == 0
    # beyond the stated maximum: refused before any device work
    assert ahs.lib.ahs_features_noalloc(ctypes.c_void_p(t.data_ptr()), ahs.AHS_NOALLOC_MAX_KEYS + 1,
                                        ahs.AHS_U32, None, ctypes.byref(f)) == ahs.AHS_ERR_RANGE
    assert ahs.lib.ahs_features_noalloc(ctypes.c_void_p(t.data_ptr()), 16, 7, None,
                                        ctypes.byref(f)) == ahs.AHS_ERR_DTYPE
    f = ahs.features_noalloc(t, key_type=ahs.AHS_U32)
    assert f.n == 16 and f.span == 0 and f.nbins == 1 and f.entropy_bits == 0.0
