"""Multi-GPU host logic on CPU (gloo): the benchmark's whole-job aggregation
over ranks (units summed, slowest rank's time), the per-rank workloads of a
weak-scaling run (independent solves, no data exchange), and one solve
partitioned by samples (each rank's contiguous tile range, the all-gather of
the tile partials, every rank merging all tiles in tile order) with the
library's tile calls replaced by a stand-in that marks each tile."""
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


class _FakeNative:
    """Stands in for the library's tile calls on CPU: tile t of the solve
    holds the value t in every entry, so the merge's input shows whether
    every tile arrived once and in tile order."""

    def __init__(self, n_tiles, tile_floats):
        self.n_tiles, self.tile_floats = n_tiles, tile_floats
        self.merged = None

    def tile_layout(self, ctx, inst):
        return self.n_tiles, self.tile_floats

    def solve_tiles(self, ctx, inst, tile0, n_tiles, tiles_out, stream):
        import torch
        tiles_out[:n_tiles] = torch.arange(tile0, tile0 + n_tiles, dtype=torch.float32)[:, None]

    def merge_tiles(self, ctx, inst, tiles, stream):
        self.merged = tiles.clone()


class _FakeSolver:
    ctx = None


def _sharded_worker(rank, world, port, n_tiles, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2508_05773_gb300.sharded import solve_sharded
    nat = _FakeNative(n_tiles, 5)
    inst = dict(x0=torch.zeros(7, dtype=torch.float64))
    first, count = solve_sharded(_FakeSolver(), inst, native=nat)
    q.put((rank, first, count, nat.merged.numpy().tolist()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,n_tiles", [(2, 7), (3, 2), (2, 128)])
def test_sample_partition_gathers_every_tile_in_order(world, n_tiles):
    # one solve's tiles split over `world` gloo ranks (uneven splits and a
    # rank without tiles included): every rank merges all tiles, each once,
    # in tile order -- the order a single launch merges them in
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sharded_worker, args=(r, world, port, n_tiles, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    expect = np.repeat(np.arange(n_tiles, dtype=np.float32)[:, None], 5, axis=1)
    covered = []
    for rank, first, count, merged in res:
        np.testing.assert_array_equal(np.asarray(merged, np.float32), expect)
        covered.extend(range(first, first + count))
    assert covered == list(range(n_tiles))


def test_rank_tiles_partition():
    import sys
    sys.path.insert(0, ROOT)
    from paper_2508_05773_gb300.sharded import rank_tiles
    for n in (1, 2, 7, 128, 129):
        for w in (1, 2, 3, 8):
            parts = [rank_tiles(n, w, r) for r in range(w)]
            assert sum(c for _, c in parts) == n
            pos = 0
            for first, count in parts:
                assert first == pos and count >= 0
                pos += count
            assert max(c for _, c in parts) - min(c for _, c in parts) <= 1
