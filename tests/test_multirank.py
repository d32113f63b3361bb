"""Multi-GPU host logic on CPU (gloo, world size 2): the benchmark's whole-job
aggregation over ranks (units summed, slowest rank's time) and the per-rank
workloads of a weak-scaling run (independent solves, no data exchange)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    rate, units, secs = bench.reduce_job(100.0 * (rank + 1), 1.0 + rank, dist)
    wl = bench._workload(rank)
    q.put((rank, rate, units, secs, float(wl["obs"].sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_and_independent_workloads():
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
    for rank, rate, units, secs, _ in res:
        assert units == pytest.approx(300.0)     # summed over ranks
        assert secs == pytest.approx(2.0)        # slowest rank
        assert rate == pytest.approx(150.0)
    assert res[0][4] != res[1][4]                # each rank solves its own scene


def test_single_process_reduce_is_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_job(50.0, 2.0) == (25.0, 50.0, 2.0)
