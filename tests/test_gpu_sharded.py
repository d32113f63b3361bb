"""One solve partitioned by samples (the multi-GPU path of one solve), with
the ranks emulated one after another on one GPU (they never wait on each
other): each "rank" rolls out its contiguous tile range into its own buffer
(brmppi_solve_tiles), the buffers are concatenated in rank order (what the
all-gather does), and the merge (brmppi_merge_tiles) must reproduce the
single-launch solve bit for bit: U*, optimal trajectory, warm start,
status, and every sample's cost pair and applied inputs."""
import numpy as np
import pytest

from paper_2508_05773_gb300 import scenarios as sc
from tests.gpu_solve import device_tensors, host_outputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from paper_2508_05773_gb300 import build as native_build
    native_build.build()
    import paper_2508_05773_gb300
    paper_2508_05773_gb300.load()
    return paper_2508_05773_gb300


def _case(name):
    if name == "config2":
        return sc.config2()
    if name == "moving":
        return sc.with_moving(sc.small_random(61, S=1000, H=24, n_obs=5), 7)
    return sc.small_random(62, S=777, H=19, n_obs=6)


@pytest.mark.parametrize("name", ["config2", "ragged", "moving"])
@pytest.mark.parametrize("ranks", [2, 3, 5])
def test_partitioned_solve_equals_single_launch(pkg, name, ranks):
    import torch
    dev = torch.device("cuda:0")
    c = _case(name)
    n_obs = int(c["obs"].shape[0])
    s = pkg.Solver(c["params"], max_obstacles=max(n_obs, 1), max_path_pts=max(2, c["path"].shape[0]))
    try:
        one = device_tensors(c, dev)
        one["U_next"] = torch.empty_like(one["U_out"])
        s.solve_device_ex(one)
        torch.cuda.synchronize()
        ref = host_outputs(one)
        assert ref["status"] == 0

        part = device_tensors(c, dev)
        part["U_next"] = torch.empty_like(part["U_out"])
        n_tiles, tile_floats = pkg.brmppi_tile_layout(s.ctx, part)
        bufs = []
        for r in range(ranks):
            first, count = pkg.rank_tiles(n_tiles, ranks, r)
            buf = torch.empty((max(count, 1), tile_floats), device=dev)
            if count:
                assert pkg.brmppi_solve_tiles(s.ctx, part, first, count, buf) == 0
            bufs.append(buf[:count])
        tiles = torch.cat(bufs).contiguous()
        assert tiles.shape[0] == n_tiles
        assert pkg.brmppi_merge_tiles(s.ctx, part, tiles) == 0
        torch.cuda.synchronize()
        got = host_outputs(part)
        for k in ("U", "traj", "U_next", "J", "J_lo", "u_hist"):
            assert np.array_equal(got[k], ref[k]), k
        assert got["status"] == 0
        # a merge without every tile is refused
        assert pkg.brmppi_merge_tiles(s.ctx, part, tiles[:-1].contiguous()) == pkg.BRMPPI_EINVAL
    finally:
        s.close()


def test_partitioned_solve_reports_input_errors(pkg):
    # a non-finite state seen by the tile launches surfaces in the merge's status
    import torch
    dev = torch.device("cuda:0")
    c = sc.small_random(63, S=300, H=10, n_obs=2)
    x0 = np.array(c["x0"])
    x0[3] = np.nan
    s = pkg.Solver(c["params"], max_obstacles=2, max_path_pts=512)
    try:
        part = device_tensors(c, dev, x0=x0)
        n_tiles, tile_floats = pkg.brmppi_tile_layout(s.ctx, part)
        tiles = torch.empty((n_tiles, tile_floats), device=dev)
        assert pkg.brmppi_solve_tiles(s.ctx, part, 0, n_tiles, tiles) == 0
        assert pkg.brmppi_merge_tiles(s.ctx, part, tiles) == 0
        torch.cuda.synchronize()
        assert int(part["status"].item()) == pkg.BRMPPI_ENONFINITE
        # the context's next solve starts from clean error bits
        ok = device_tensors(c, dev)
        s.solve_device_ex(ok)
        torch.cuda.synchronize()
        assert int(ok["status"].item()) == 0
    finally:
        s.close()
