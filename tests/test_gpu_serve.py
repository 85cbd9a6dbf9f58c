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


def test_generated_requests_against_oracle(ahs):
    """AHS_REQ_GENERATE: the library writes each request's keys on the device
    from (seed, id, kind); the same keys come from the host generator, and
    every result is the oracle's sort of them, alone and in the mix."""
    import torch
    seed = 5
    lengths = gen.log_uniform_lengths(12, 56, 1, 1000, 5_000_000)
    reqs = [(rid, int(L), rid % 4) for rid, L in enumerate(lengths)]
    reqs.append((99, 4_500_000, 3))           # large lane, nearly sorted kind
    with ahs.Context(0) as ctx:
        _serve(ahs, ctx, budget=16 << 30)
        outs = [torch.empty(L, dtype=torch.int32, device="cuda") for _, L, _ in reqs]
        tickets = []
        for (rid, L, kind), o in zip(reqs, outs):
            r = ahs.ahs_request_t()
            r.d_keys_out, r.n, r.type = o.data_ptr(), L, ahs.AHS_U32
            r.flags, r.gen_seed, r.gen_id, r.gen_kind = ahs.AHS_REQ_GENERATE, seed, rid, kind
            t = ctypes.c_uint64()
            ahs.check(ahs.lib.ahs_serve_submit(ctx.handle, ctypes.byref(r), ctypes.byref(t)), "submit")
            tickets.append(t.value)
        for (rid, L, kind), o, t in zip(reqs, outs, tickets):
            rc, res = _wait(ahs, ctx, t)
            assert rc == ahs.AHS_OK and res.status == ahs.AHS_OK, rid
            keys = gen.request_keys(seed, rid, kind, L)
            assert np.array_equal(host(o, np.uint32), _oracle_sorted(keys)), (rid, kind)
        # generation needs uint32 keys and no payload
        bad = ahs.ahs_request_t()
        bad.d_keys_out, bad.n, bad.type, bad.flags = outs[0].data_ptr(), 10, ahs.AHS_U64, 1
        t = ctypes.c_uint64()
        assert ahs.lib.ahs_serve_submit(ctx.handle, ctypes.byref(bad), ctypes.byref(t)) == \
            ahs.AHS_ERR_INVALID_ARG
        ahs.check(ahs.lib.ahs_serve_stop(ctx.handle), "serve_stop")


def test_payload_requests_stable_against_oracle(ahs):
    """Served requests with a uint32 payload come back in the unique stable
    order (the oracle's merge sort), in both lanes."""
    import torch
    rng = np.random.default_rng(9)
    sizes = [1000, 70_001, 300_000, 5_000_000, 2]
    arrays = [rng.integers(0, 5000 if i % 2 else 2**32, size=n, dtype=np.uint32)
              for i, n in enumerate(sizes)]
    with ahs.Context(0) as ctx:
        _serve(ahs, ctx, budget=8 << 30)
        bufs, tickets = [], []
        for a in arrays:
            v = np.arange(len(a), dtype=np.uint32)
            ki, ko, vi, vo = dev(a), dev(np.zeros_like(a)), dev(v), dev(np.zeros_like(v))
            r = ahs.ahs_request_t()
            r.d_keys_in, r.d_keys_out, r.n, r.type = ki.data_ptr(), ko.data_ptr(), len(a), ahs.AHS_U32
            r.d_vals_in, r.d_vals_out = vi.data_ptr(), vo.data_ptr()
            t = ctypes.c_uint64()
            ahs.check(ahs.lib.ahs_serve_submit(ctx.handle, ctypes.byref(r), ctypes.byref(t)), "submit")
            bufs.append((ki, ko, vi, vo, v))
            tickets.append(t.value)
        for a, (ki, ko, vi, vo, v), t in zip(arrays, bufs, tickets):
            rc, res = _wait(ahs, ctx, t)
            assert rc == ahs.AHS_OK and res.status == ahs.AHS_OK
            ek, ev = oracle.merge_sort(a, v)
            assert np.array_equal(host(ko, np.uint32), ek)
            assert np.array_equal(host(vo, np.uint32), ev)
        ahs.check(ahs.lib.ahs_serve_stop(ctx.handle), "serve_stop")
