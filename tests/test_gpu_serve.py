"""Serving loop: continuous batching, admission by HBM budget, identity of
results alone and in a mix, latency statistics."""
import ctypes
import threading

import numpy as np
import pytest

import oracle
from gen import host as gen
from gpu_util import dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ahs():
    import paper_2506_20677_gb300 as m
    return m


def _serve(ahs, ctx, budget, inflight=64):
    cfg = ahs.ahs_serve_config_t(budget, inflight, 100)
    ahs.check(ahs.lib.ahs_serve_start(ctx.handle, ctypes.byref(cfg)), "serve_start")


def _submit(ahs, ctx, d_in, d_out, kt):
    req = ahs.ahs_request_t(d_in.data_ptr(), d_out.data_ptr(), d_in.numel(), kt)
    t = ctypes.c_uint64()
    rc = ahs.lib.ahs_serve_submit(ctx.handle, ctypes.byref(req), ctypes.byref(t))
    return rc, t.value


def _wait(ahs, ctx, ticket, timeout_ms=60000):
    res = ahs.ahs_result_t()
    rc = ahs.lib.ahs_serve_poll(ctx.handle, ticket, timeout_ms, ctypes.byref(res))
    return rc, res


def _oracle_sorted(a):
    return oracle.sort(a, profile=oracle.PAPER)[0]


def test_mix_equals_alone_and_oracle(ahs):
    import torch
    rng = np.random.default_rng(5)
    sizes = [1000, 17, 4096, 50_000, 300_000, 1 << 22, 5_000_000, 123_456, 2, 0, 70_000]
    arrays = []
    for i, n in enumerate(sizes):
        if i % 3 == 0:
            a = rng.integers(0, 4096, size=n, dtype=np.uint32)
        elif i % 3 == 1:
            a = rng.integers(0, 2**32, size=n, dtype=np.uint32)
        else:
            vals = rng.integers(0, 2**32, size=1024, dtype=np.uint32)
            a = vals[rng.integers(0, 1024, size=n)]
        arrays.append(a)
    # requests shaped like the served workload: config-4 distributions (a, b,
    # c, e of config 2), log-uniform sizes from 10^3 keys
    lengths = gen.log_uniform_lengths(8, 55, 1, 1000, 3_000_000)
    for j, L in enumerate(lengths):
        arrays.append(gen.config4_segment(900_000 + j, int(L), j % 4))
    with ahs.Context(0) as ctx:
        _serve(ahs, ctx, budget=8 << 30)
        # each request alone
        alone = []
        for a in arrays:
            d_in, d_out = dev(a), dev(np.zeros_like(a))
            rc, t = _submit(ahs, ctx, d_in, d_out, ahs.AHS_U32)
            assert rc == ahs.AHS_OK
            rc, res = _wait(ahs, ctx, t)
            assert rc == ahs.AHS_OK and res.status == ahs.AHS_OK
            alone.append(host(d_out, np.uint32))
        # all together, submitted from two threads while others run
        ins = [dev(a) for a in arrays]
        outs = [dev(np.zeros_like(a)) for a in arrays]
        tickets = [None] * len(arrays)

        def submitter(idx):
            for i in idx:
                rc, t = _submit(ahs, ctx, ins[i], outs[i], ahs.AHS_U32)
                assert rc == ahs.AHS_OK
                tickets[i] = t
        th = [threading.Thread(target=submitter, args=(list(range(k, len(arrays), 2)),)) for k in (0, 1)]
        for x in th:
            x.start()
        for x in th:
            x.join()
        for i, t in enumerate(tickets):
            rc, res = _wait(ahs, ctx, t)
            assert rc == ahs.AHS_OK and res.status == ahs.AHS_OK, i
            mixed = host(outs[i], np.uint32)
            assert np.array_equal(mixed, alone[i]), i
            assert np.array_equal(mixed, _oracle_sorted(arrays[i])), i
        st = ahs.ahs_serve_stats_t()
        ahs.check(ahs.lib.ahs_serve_stats(ctx.handle, ctypes.byref(st)), "stats")
        assert st.completed == 2 * sum(1 for a in arrays if len(a))
        assert 0 < st.p50_ms <= st.p99_ms
        assert st.peak_reserved_bytes <= 8 << 30
        assert st.batches >= 1
        ahs.check(ahs.lib.ahs_serve_stop(ctx.handle), "serve_stop")


def test_budget_refusal_and_admission_bound(ahs):
    rng = np.random.default_rng(6)
    with ahs.Context(0) as ctx:
        budget = 64 << 20
        _serve(ahs, ctx, budget=budget, inflight=4)
        big = dev(np.zeros(20_000_000, dtype=np.uint32))
        rc, _ = _submit(ahs, ctx, big, big, ahs.AHS_U32)
        assert rc == ahs.AHS_ERR_BUDGET        # could never fit
        arrays = [rng.integers(0, 2**32, size=2_000_000, dtype=np.uint32) for _ in range(12)]
        ins = [dev(a) for a in arrays]
        outs = [dev(np.zeros_like(a)) for a in arrays]
        tickets = [_submit(ahs, ctx, i, o, ahs.AHS_U32)[1] for i, o in zip(ins, outs)]
        for t, a, o in zip(tickets, arrays, outs):
            rc, res = _wait(ahs, ctx, t)
            assert rc == ahs.AHS_OK and res.status == ahs.AHS_OK
            assert np.array_equal(host(o, np.uint32), _oracle_sorted(a))
        st = ahs.ahs_serve_stats_t()
        ahs.check(ahs.lib.ahs_serve_stats(ctx.handle, ctypes.byref(st)), "stats")
        assert st.peak_reserved_bytes <= budget     # the ledger never exceeded the budget
        res = ahs.ahs_result_t()
        assert ahs.lib.ahs_serve_poll(ctx.handle, 10**9, 0, ctypes.byref(res)) == ahs.AHS_ERR_NOT_FOUND
        ahs.check(ahs.lib.ahs_serve_stop(ctx.handle), "serve_stop")
