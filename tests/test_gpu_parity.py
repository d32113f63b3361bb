"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs, element by element (U*, optimal trajectory, every
sample's cost), at sizes that span several blocks and a ragged tail, for
every kernel variant, plus the edge cases of the solve."""
import numpy as np
import pytest

import oracle
from paper_2508_05773_gb300 import scenarios as sc
from tests.gpu_solve import device_solve, device_tensors, host_outputs
from tests.parity import assert_solve_matches, err_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from paper_2508_05773_gb300 import build as native_build
    native_build.build()
    import paper_2508_05773_gb300
    paper_2508_05773_gb300.load()
    return paper_2508_05773_gb300


def _oracle(c, **over):
    p = sc.as_float32(dict(c["params"], **over))
    return p, oracle.solve(p, c["x0"], c["U_nom"], c["obs"], c["path"], c["ds"], c["seed"],
                           c["counter"], want_uhist=True)


def _gpu(pkg, c, tps=0, threads=0, max_obs=None, **over):
    p = dict(c["params"], **over)
    n_obs = c["obs"].shape[0]
    s = pkg.Solver(p, max_obstacles=max(n_obs, 1) if max_obs is None else max_obs,
                   max_path_pts=max(2, c["path"].shape[0]), threads_per_sample=tps,
                   block_threads=threads)
    try:
        return device_solve(s, c)
    finally:
        s.close()


@pytest.mark.parametrize("make", [sc.config1, sc.config1b])
def test_config1_matches_oracle(pkg, make):
    c = make()
    p, ref = _oracle(c)
    out = _gpu(pkg, c)
    assert_solve_matches(out, ref, p, make.__name__, strict=True)


@pytest.mark.parametrize("tps", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("threads", [64, 96, 256])
def test_every_variant_matches_oracle(pkg, tps, threads):
    # 5 obstacles -> 9 normals per step -> 3 Philox blocks: teams of 1..32
    # lanes cover them with 1..3 blocks per lane; S = 300 leaves a ragged
    # last block for every shape.
    c = sc.small_random(11, S=300, H=16, n_obs=5)
    p, ref = _oracle(c)
    out = _gpu(pkg, c, tps=tps, threads=threads)
    assert_solve_matches(out, ref, p, f"tps={tps} threads={threads}")


@pytest.mark.parametrize("tps", [2, 4, 8, 16])
@pytest.mark.parametrize("n_obs", [0, 7, 13, 21, 29, 45, 70, 100])
def test_blocks_per_lane_grid(pkg, tps, n_obs):
    # 1 + n_obs constraints -> ceil((4 + n_obs) / 4) Philox blocks per step:
    # with 2..16 lanes per sample this walks every blocks-per-lane variant
    # (1, 2, 3, 4 and the producer-warp / lane-staged split) that a team
    # width offers; S = 96 leaves a ragged last tile at 128 threads.
    P = (4 + n_obs + 3) // 4
    if P > (2 if tps == 16 else 4) * tps:
        pytest.skip("no variant with that many blocks per lane")
    c = sc.small_random(300 + n_obs, S=96, H=8, n_obs=n_obs)
    p, ref = _oracle(c)
    out = _gpu(pkg, c, tps=tps, threads=128)
    assert_solve_matches(out, ref, p, f"tps={tps} n_obs={n_obs}")


@pytest.mark.parametrize("seed", range(8))
def test_fuzz_small_cases(pkg, seed):
    rng = np.random.default_rng(100 + seed)
    S = int(rng.integers(1, 400))
    H = int(rng.integers(1, 40))
    n_obs = int(rng.integers(0, 13))
    c = sc.small_random(200 + seed, S=S, H=H, n_obs=n_obs, reverse=bool(seed % 2))
    p, ref = _oracle(c)
    out = _gpu(pkg, c)
    assert_solve_matches(out, ref, p, f"S={S} H={H} n_obs={n_obs}")


@pytest.mark.parametrize("jerk", [False, True])
@pytest.mark.parametrize("where,S,n_pts", [("shared memory", 300, None), ("tile partials", 1024, 3),
                                           ("serial", 64, 3)])
def test_trajectory_scratch_paths(pkg, where, S, n_pts, jerk):
    """The merge's optimal trajectory keeps its per-step values in the CTA's
    table regions when they hold 8 (H+1) floats, else in the consumed tile
    partials, else runs one serial thread.  A short path and no obstacles
    (4 lanes x 128 threads: 32 samples per tile, H = 40) shrink the tables
    below 8 (H+1) floats; S picks between partials (32 tiles) and serial
    (2 tiles)."""
    c = sc.small_random(41, S=S, H=40, n_obs=0 if n_pts else 4)
    if n_pts:
        c["path"] = c["path"][:n_pts].copy()
    if jerk:
        c = sc.jerk_model(c, a0=0.3, seed=5)
    p, ref = _oracle(c)
    if jerk:  # the trajectory output holds the 7 kinematic states
        ref = dict(ref, traj=ref["traj"][:, :7])
    out = _gpu(pkg, c, tps=4, threads=128)
    assert_solve_matches(out, ref, p, f"{where} jerk={jerk}")


def test_standard_mppi_flag(pkg):
    c = sc.config1b(S=200, H=25)
    p, ref = _oracle(c, flags=sc.FLAG_PROJ_NONE)
    out = _gpu(pkg, c, flags=sc.FLAG_PROJ_NONE)
    assert_solve_matches(out, ref, p, "PROJ_NONE")


def test_config2_tick0_matches_oracle(pkg):
    c = sc.config2()
    p, ref = _oracle(c)
    out = _gpu(pkg, c)
    assert_solve_matches(out, ref, p, "config2", strict=True)


def test_many_obstacles_wide_teams(pkg):
    c = sc.small_random(5, S=512, H=20, n_obs=64)
    p, ref = _oracle(c)
    out = _gpu(pkg, c, max_obs=64)
    assert_solve_matches(out, ref, p, "64 obstacles")


def test_zero_noise_all_samples_equal(pkg):
    c = sc.small_random(6, S=130, H=12, n_obs=3)
    over = dict(sigma=(0.0, 0.0, 0.0), sigma_alpha=0.0)
    p, ref = _oracle(c, **over)
    out = _gpu(pkg, c, **over)
    assert np.all(out["J"] == out["J"][0])
    assert_solve_matches(out, ref, p, "zero noise")


def test_edge_sizes(pkg):
    for S, H in [(1, 1), (1, 7), (2, 1), (33, 3)]:
        c = sc.small_random(7, S=S, H=H, n_obs=2)
        p, ref = _oracle(c)
        out = _gpu(pkg, c)
        assert_solve_matches(out, ref, p, f"S={S} H={H}")


def test_deterministic_bits(pkg):
    c = sc.small_random(8, S=777, H=15, n_obs=4)
    a = _gpu(pkg, c)
    b = _gpu(pkg, c)
    assert np.array_equal(a["U"], b["U"]) and np.array_equal(a["J"], b["J"])
    assert np.array_equal(a["traj"], b["traj"])


def test_invalid_inputs_rejected(pkg):
    c = sc.small_random(9, S=16, H=5, n_obs=2)
    s = pkg.Solver(c["params"], max_obstacles=4, max_path_pts=512)
    try:
        bad = c["obs"].copy()
        bad[0, 5] = 4.0
        st, *_ = pkg.brmppi_solve(s.ctx, c["x0"], c["U_nom"], bad, c["path"], c["ds"], 0, 0, 5)
        assert st == pkg.BRMPPI_EINVAL
        x0 = c["x0"].copy()
        x0[2] = np.nan
        st, *_ = pkg.brmppi_solve(s.ctx, x0, c["U_nom"], c["obs"], c["path"], c["ds"], 0, 0, 5)
        assert st == pkg.BRMPPI_ENONFINITE
        st, *_ = pkg.brmppi_solve(s.ctx, c["x0"], c["U_nom"], np.zeros((5, 6), np.float32),
                                  c["path"], c["ds"], 0, 0, 5)
        assert st == pkg.BRMPPI_EINVAL  # more obstacles than the capacity
        sharp = c["path"].copy()
        sharp[len(sharp) // 2:, 2] += 1.0  # a 1 rad heading jump between two rows
        st, *_ = pkg.brmppi_solve(s.ctx, c["x0"], c["U_nom"], c["obs"], sharp, c["ds"], 0, 0, 5)
        assert st == pkg.BRMPPI_EINVAL
        # the context still works after rejected calls
        out = s.solve(c["x0"], c["U_nom"], c["obs"], c["path"], c["ds"], c["seed"], c["counter"])
        assert out["status"] == 0
    finally:
        s.close()


def test_device_path_turn_rejected_by_the_kernel(pkg):
    # device buffers are not checked on the host: the kernel flags a path
    # whose consecutive headings differ by more than pi/4 and reports EINVAL
    import torch
    c = sc.small_random(11, S=64, H=8, n_obs=2)
    s = pkg.Solver(c["params"], max_obstacles=4, max_path_pts=512)
    try:
        dev = torch.device("cuda:0")
        t = lambda a, dt=torch.float32: torch.tensor(np.asarray(a), dtype=dt, device=dev)
        U = torch.empty((8, 3), device=dev)
        st = torch.full((1,), 99, dtype=torch.int32, device=dev)
        sharp = c["path"].copy()
        sharp[5:, 2] -= 0.8
        rc = s.solve_device(t(c["x0"], torch.float64), t(c["U_nom"]), t(c["obs"]), t(sharp),
                            c["ds"], c["seed"], c["counter"], U, None, None, None, st)
        assert rc == 0
        torch.cuda.synchronize()
        assert int(st.item()) == pkg.BRMPPI_EINVAL
        # the next solve on the same context starts from clean error bits
        rc = s.solve_device(t(c["x0"], torch.float64), t(c["U_nom"]), t(c["obs"]), t(c["path"]),
                            c["ds"], c["seed"], c["counter"], U, None, None, None, st)
        torch.cuda.synchronize()
        assert rc == 0 and int(st.item()) == 0
    finally:
        s.close()


def test_device_entry_point_matches_host(pkg):
    import torch
    c = sc.small_random(10, S=500, H=20, n_obs=6)
    s = pkg.Solver(c["params"], max_obstacles=8, max_path_pts=1024)
    try:
        host = s.solve(c["x0"], c["U_nom"], c["obs"], c["path"], c["ds"], c["seed"], c["counter"],
                       want_traj=True, want_J=True)
        ex = device_solve(s, c)
        for k in ("U", "traj", "J"):
            assert np.array_equal(ex[k], host[k]), k
        dev = torch.device("cuda:0")
        t = lambda a, dt=torch.float32: torch.tensor(np.asarray(a), dtype=dt, device=dev)
        U = torch.empty((20, 3), device=dev)
        tr = torch.empty((21, 7), device=dev)
        J = torch.empty(500, device=dev)
        Un = torch.empty((20, 3), device=dev)
        st = torch.full((1,), 99, dtype=torch.int32, device=dev)
        rc = s.solve_device(t(c["x0"], torch.float64), t(c["U_nom"]), t(c["obs"]), t(c["path"]),
                            c["ds"], c["seed"], c["counter"], U, tr, J, Un, st)
        assert rc == 0
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        assert np.array_equal(U.cpu().numpy(), host["U"])
        assert np.array_equal(tr.cpu().numpy(), host["traj"])
        assert np.array_equal(J.cpu().numpy(), host["J"])
        Uh = host["U"]
        np.testing.assert_array_equal(Un.cpu().numpy(), np.vstack([Uh[1:], Uh[-1:]]))
    finally:
        s.close()


def test_stored_trajectories_match_oracle(pkg):
    import torch
    dev = torch.device("cuda:0")
    c = sc.small_random(12, S=300, H=16, n_obs=5)
    p = sc.as_float32(c["params"])
    ref = oracle.solve(p, c["x0"], c["U_nom"], c["obs"], c["path"], c["ds"], c["seed"], c["counter"],
                       want_uhist=True, want_states=True)
    s = pkg.Solver(c["params"], max_obstacles=8, max_path_pts=1024)
    try:
        a = device_tensors(c, dev, states=True)
        b = device_tensors(c, dev, states=False, inputs=False)
        s.solve_device_ex(a)
        s.solve_device_ex(b)
        torch.cuda.synchronize()
        assert int(a["status"].item()) == 0
        states = a["states_out"].cpu().numpy()
        assert err_state(states, ref["states"]) <= 1e-4
        # storing the states and inputs changes nothing else
        for k in ("U_out", "traj_out", "J_out"):
            assert np.array_equal(a[k].cpu().numpy(), b[k].cpu().numpy()), k
        assert_solve_matches(host_outputs(a), ref, p, "stored-trajectory variant")
        # a smaller solve through the same context (S, H below the capacity)
        c2 = sc.small_random(13, S=77, H=9, n_obs=3)
        d = device_tensors(c2, dev, states=True)
        s.solve_device_ex(d)
        torch.cuda.synchronize()
        p2 = sc.as_float32(c2["params"])
        ref2 = oracle.solve(p2, c2["x0"], c2["U_nom"], c2["obs"], c2["path"], c2["ds"], c2["seed"],
                            c2["counter"], want_uhist=True, want_states=True)
        assert err_state(d["states_out"].cpu().numpy(), ref2["states"]) <= 1e-4
        assert_solve_matches(host_outputs(d), ref2, p2, "smaller solve")
    finally:
        s.close()
