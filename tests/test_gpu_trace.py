"""Per-launch tracing (ahs_trace_enable / ahs_trace_collect) on the GPU."""
import numpy as np
import pytest

from gpu_util import dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ahs():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    import paper_2506_20677_gb300 as m
    return m


def test_trace_lists_every_launch_in_order(ahs):
    ctx = ahs.Context(0)
    try:
        rng = np.random.default_rng(3)
        a = rng.integers(0, 2**32, size=(1 << 20) + 3, dtype=np.uint32)
        t = dev(a)
        ctx.trace(True)
        r = ctx.sort(t, force=ahs.AHS_GENERAL, key_type=ahs.AHS_U32)
        ctx.trace(False)
        tr = ctx.trace_collect()
        assert r.strategy == ahs.AHS_GENERAL
        names = [e[0] for e in tr]
        assert names[:3] == ["features_minmax", "features_histogram", "features_entropy"]
        assert any(n.startswith("bucket_sort") for n in names)
        assert all(e[2] >= 0.0 for e in tr)
        starts = [e[3] for e in tr]
        assert starts[0] == 0.0
        # One stream: every launch starts after the previous one started.
        assert all(b >= a_ for a_, b in zip(starts, starts[1:]))
        # The keys the feature passes report are the input's.
        assert tr[0][1] == len(a)
        assert ctx.trace_collect() == []
    finally:
        ctx.close()
