"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs, element by element (U*, optimal trajectory, every
sample's cost), at sizes that span several blocks and a ragged tail, for
every kernel variant, plus the edge cases of the solve."""
import numpy as np
import pytest

import oracle
from paper_2508_05773_gb300 import scenarios as sc
from tests.parity import EPS_J, assert_solve_matches, err_j, err_state, err_u

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
        return s.solve(c["x0"], c["U_nom"], c["obs"], c["path"], c["ds"], c["seed"], c["counter"],
                       want_traj=True, want_J=True)
    finally:
        s.close()


@pytest.mark.parametrize("make", [sc.config1, sc.config1b])
def test_config1_matches_oracle(pkg, make):
    c = make()
    p, ref = _oracle(c)
    out = _gpu(pkg, c)
    assert_solve_matches(out, ref, p, make.__name__)


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


def test_standard_mppi_flag(pkg):
    c = sc.config1b(S=200, H=25)
    p, ref = _oracle(c, flags=sc.FLAG_PROJ_NONE)
    out = _gpu(pkg, c, flags=sc.FLAG_PROJ_NONE)
    assert_solve_matches(out, ref, p, "PROJ_NONE")


def test_config2_tick0_matches_oracle(pkg):
    c = sc.config2()
    p, ref = _oracle(c)
    out = _gpu(pkg, c)
    assert_solve_matches(out, ref, p, "config2")


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
        # the context still works after rejected calls
        out = s.solve(c["x0"], c["U_nom"], c["obs"], c["path"], c["ds"], c["seed"], c["counter"])
        assert out["status"] == 0
    finally:
        s.close()


def test_device_entry_point_matches_host(pkg):
    import torch
    c = sc.small_random(10, S=500, H=20, n_obs=6)
    host = _gpu(pkg, c)
    s = pkg.Solver(c["params"], max_obstacles=8, max_path_pts=1024)
    try:
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


@pytest.mark.slow
def test_config5_full_size_sampled(pkg):
    # Full-size stress solve: every sample's cost from the GPU; the oracle
    # recomputes a spread of samples one by one.  U* is checked by its
    # properties (bounds; convex combination of applied inputs).
    c = sc.config5()
    p = sc.as_float32(c["params"])
    out = _gpu(pkg, c, max_obs=64)
    assert np.all(np.isfinite(out["J"]))
    for s in [0, 1, 4097, 31337, 65535]:
        one = oracle.rollout_sample(p, c["x0"], c["U_nom"], c["obs"], c["path"], c["ds"], c["seed"],
                                    c["counter"], s)
        assert abs(out["J"][s] - one["J"]) / abs(one["J"]) <= EPS_J, s
    U = out["U"]
    assert np.all(U >= np.array(p["z_lo"]) - 1e-6) and np.all(U <= np.array(p["z_hi"]) + 1e-6)
    tr = out["traj"]
    assert np.all(np.isfinite(tr)) and np.array_equal(tr[0, [4, 5]], c["x0"][[4, 5]].astype(np.float32))
