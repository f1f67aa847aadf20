"""The N > 1 path of bench.py is replicas only: each rank solves its own copy
and rank 0 reports (total solves) / (max time over ranks). The rank plumbing
(gloo barrier + max reduction) runs here as two CPU processes."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist, r, ws, local = bench._dist()
    t = 10.0 + 5.0 * rank            # per-rank "time": rank 1 is slower
    m = bench._max_over_ranks(dist, t)
    bench._barrier(dist)
    q.put((rank, ws, m))
    dist.destroy_process_group()


def test_replicas_take_max_time_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    ps = [ctx.Process(target=_worker, args=(i, 2, port, q)) for i in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    assert out == [(0, 2, 15.0), (1, 2, 15.0)]


def _dying_worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), DPSR_PG_TIMEOUT_S="20")
    sys.path.insert(0, ROOT)
    import time

    import bench
    dist, r, ws, local = bench._dist()
    bench._barrier(dist)             # both ranks are up
    if rank == 1:
        os._exit(3)                  # dies between steps, with no collective in flight
    t0 = time.time()
    try:
        bench._max_over_ranks(dist, 1.0)
        q.put((rank, "no error", time.time() - t0))
    except Exception as exc:         # the survivor learns of it from its next collective
        q.put((rank, type(exc).__name__, time.time() - t0))


def test_rank_failure_ends_the_next_collective():
    """A rank that exits between steps makes the other rank's next collective
    fail within the process group's timeout instead of hanging."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 30500 + os.getpid() % 1000
    ps = [ctx.Process(target=_dying_worker, args=(i, 2, port, q)) for i in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
    assert ps[1].exitcode == 3
    assert ps[0].exitcode == 0
    rank, what, dt = q.get(timeout=10)
    assert rank == 0 and what != "no error" and dt < 60.0, (what, dt)
