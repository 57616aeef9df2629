"""bench.py's multi-rank host logic (replicas: max-over-ranks time, summed work) on two gloo
ranks on CPU."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    r, w, local = bench.dist_env()
    dist = bench.init_dist(w, "gloo")
    bench.barrier(dist)
    t = bench.max_over_ranks(dist, 1.0 + rank)          # per-rank elapsed seconds
    work = bench.sum_over_ranks(dist, 10.0 * (rank + 1))  # per-rank cell-updates
    out.put((r, t, work))
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_bench():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in res] == [0, 1]
    assert all(t == 2.0 for _, t, _ in res)               # the job's time is the slowest rank's
    assert all(w == 30.0 for _, _, w in res)              # value counts every rank's work


def test_single_process_has_no_collective():
    import bench
    assert bench.init_dist(1, "gloo") is None
    assert bench.max_over_ranks(None, 3.5) == 3.5
    assert bench.sum_over_ranks(None, 2.0) == 2.0
