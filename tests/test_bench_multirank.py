"""The multi-rank timing logic of bench.py (barrier, max over ranks, the
whole-job value) on two CPU processes over gloo."""
import os
import sys

import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(world),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import bench
    ws, r, _ = bench.dist_setup()
    bench.barrier(ws)
    ms = 10.0 * (r + 1)          # rank-dependent "step time"
    worst = bench.max_over_ranks(ms, ws)
    T = 1000
    value = T * ws / (worst * 1e-3)  # whole-job sub-intervals/s, as the bench computes it
    q.put((r, ws, worst, value))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_rank_max_and_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2, 2]
    assert all(r[2] == 20.0 for r in res)          # the slower rank's time on every rank
    assert all(abs(r[3] - 2 * 1000 / 0.020) < 1e-6 for r in res)
