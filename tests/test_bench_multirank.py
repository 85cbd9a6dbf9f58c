"""bench.py's multi-rank path (replicas, weak scaling) on CPU with gloo:
barrier, max-over-ranks timing and the whole-job value."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import sys
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    w, r, _ = bench.dist_setup()
    bench.barrier(w)
    local_ms = 100.0 + 50.0 * r           # rank 1 is slower
    m = bench.max_over_ranks(w, local_ms)
    v = bench.job_value(w, 1000, 10, m)
    bench.barrier(w)
    import torch.distributed as dist
    dist.destroy_process_group()
    q.put((r, w, m, v))


def test_two_rank_max_timing_and_weak_value():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    for r, w, m, v in out:
        assert w == 2 and m == 150.0                     # max over ranks
        assert abs(v - 2 * 1000 * 10 / 0.150 / 1e9) < 1e-12


def test_single_rank_value():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.max_over_ranks(1, 12.5) == 12.5
    assert bench.job_value(1, 2**28, 1, 1000.0) == 2**28 / 1e9
