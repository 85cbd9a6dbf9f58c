"""Failure detection without faulting the GPU: a bounded device wait that runs
out is reported as a status and leaves the context usable; an allocation
limit is reported as AHS_ERR_OOM."""
import numpy as np
import pytest

from gpu_util import dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ahs():
    import paper_2506_20677_gb300 as m
    return m


def test_lookback_timeout_reported_and_context_survives(ahs):
    # A payload keeps the radix path on its stable LSD passes, whose tiles
    # chain through the decoupled look-back that the debug flag starves.
    rng = np.random.default_rng(1)
    a = rng.integers(0, 2**32, size=1 << 20, dtype=np.uint32)
    v = np.arange(a.size, dtype=np.uint32)
    with ahs.Context(0, debug_flags=ahs.AHS_DEBUG_STALL_ONE_TILE) as bad:
        with pytest.raises(ahs.AhsError) as e:
            bad.sort(dev(a), dev(v), force=ahs.AHS_RADIX, key_type=ahs.AHS_U32)
        assert e.value.status == ahs.AHS_ERR_DEVICE_TIMEOUT
        # the same context keeps working on paths without look-back
        b = rng.integers(0, 1000, size=1 << 20, dtype=np.uint32)
        r = bad.sort(dev(b), force=ahs.AHS_COUNTING, key_type=ahs.AHS_U32)
        assert np.array_equal(host(r.keys, np.uint32), np.sort(b))
        r = bad.sort(dev(a), force=ahs.AHS_RADIX, key_type=ahs.AHS_U32)
        assert np.array_equal(host(r.keys, np.uint32), np.sort(a))
    with ahs.Context(0) as good:
        r = good.sort(dev(a), dev(v), force=ahs.AHS_RADIX, key_type=ahs.AHS_U32)
        order = np.argsort(a, kind="stable")
        assert np.array_equal(host(r.keys, np.uint32), a[order])
        assert np.array_equal(host(r.vals, np.uint32), v[order])


def test_workspace_limit_reports_oom(ahs):
    a = np.arange(1 << 20, dtype=np.uint32)[::-1].copy()
    with ahs.Context(0, workspace_limit=1 << 20) as small:
        with pytest.raises(ahs.AhsError) as e:
            small.sort(dev(a), key_type=ahs.AHS_U32)
        assert e.value.status == ahs.AHS_ERR_OOM
    with ahs.Context(0) as ok:
        r = ok.sort(dev(a), key_type=ahs.AHS_U32)
        assert np.array_equal(host(r.keys, np.uint32), np.sort(a))
