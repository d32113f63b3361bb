"""GPU parity of the optional terms against the FP64 oracle, through the C
ABI: the hitch-angle stabilizer (Sec. IV-D), moving and e = 4 obstacles
(Sec. IV-C), the collision cost of the comparison method (Sec. V) and the
barrier-rate buffer cost (Sec. IV-A), on the plain, batched and serving
paths."""
import numpy as np
import pytest

import oracle
from paper_2508_05773_gb300 import scenarios as sc
from tests import test_oracle_stabilizer as tz
from tests.parity import assert_solve_matches, buffer_conditioning, stab_tolerance
from tests.gpu_solve import add_cost_outputs, device_solve, host_outputs
from tests.served import served_costs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from paper_2508_05773_gb300 import build as native_build
    native_build.build()
    import paper_2508_05773_gb300
    paper_2508_05773_gb300.load()
    return paper_2508_05773_gb300


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


def _oracle(c, **over):
    p = sc.as_float32(dict(c["params"], **over))
    return p, oracle.solve(p, c["x0"], c["U_nom"], c["obs"], c["path"], c["ds"], c["seed"],
                           c["counter"], want_uhist=True)


def _gpu(pkg, c, tps=0, threads=0, **over):
    p = dict(c["params"], **over)
    n_obs = c["obs"].shape[0]
    s = pkg.Solver(p, max_obstacles=max(n_obs, 1), max_path_pts=max(2, c["path"].shape[0]),
                   threads_per_sample=tps, block_threads=threads)
    try:
        return device_solve(s, c)
    finally:
        s.close()


# ------------------------------------------------------------ stabilizer
def _stab_cases(p, rng, n):
    """Active (feasible and infeasible) cases near the hitch limit and
    random states far from it."""
    xs, us = [], []
    for x, u in tz._active_cases(p, n // 3, int(rng.integers(1 << 30))):
        xs.append(x)
        us.append(u)
    for x, u in tz._active_cases(p, n // 6, int(rng.integers(1 << 30)), feasible=False):
        xs.append(x)
        us.append(u)
    while len(xs) < n:
        th1 = rng.uniform(-3, 3)
        xs.append((rng.uniform(-50, 50), rng.uniform(-50, 50), th1, th1 + rng.uniform(-0.6, 0.6),
                   rng.uniform(-2, 2), rng.uniform(-0.5, 0.5), rng.uniform(0, 30)))
        us.append((rng.uniform(-3, 3), rng.uniform(-1, 1), rng.uniform(0, 3)))
    return np.asarray(xs, np.float64), np.asarray(us, np.float32)


@pytest.mark.parametrize("seed", range(3))
def test_stabilizer_matches_oracle(pkg, torch, seed):
    rng = np.random.default_rng(seed)
    pd = sc.params(alpha_stab=float(rng.uniform(0.2, 1.0)),
                   q_stab=(float(rng.uniform(0.3, 3.0)), float(rng.uniform(0.3, 3.0))))
    p = sc.as_float32(pd)
    X, U = _stab_cases(p, rng, 3000)
    s = pkg.Solver(pd)
    try:
        xd = torch.from_numpy(X).cuda()
        ud = torch.from_numpy(U).cuda()
        out = torch.zeros((len(X), 4), dtype=torch.float32, device="cuda")
        s.hitch_stabilize_device(xd, ud, out)
        torch.cuda.synchronize()
        G = out.cpu().numpy().astype(np.float64)
    finally:
        s.close()
    n_inf = 0
    for i in range(len(X)):
        st, o, slack = oracle.hitch_stabilize(p, X[i], U[i].astype(np.float64))
        Au, h, br = oracle.hitch_row(p, X[i])
        tol, eps_rhs = stab_tolerance(p, X[i], Au[:2], o)
        assert G[i, 2] == np.float32(U[i, 2]), i  # nu passes through
        assert abs(G[i, 3] - slack) <= 4 * eps_rhs + float(np.abs(Au[:2]) @ tol), (i, G[i, 3], slack)
        if st == 1 and slack < -4 * eps_rhs:
            n_inf += 1
            np.testing.assert_array_equal(G[i, :2], o[:2].astype(np.float32), err_msg=str(i))
            continue
        d = np.abs(G[i, :2] - o[:2])
        assert np.all(d <= tol), (i, G[i], o, tol)
    assert n_inf >= 100


def test_stabilizer_inside_the_solve(pkg, torch):
    """u_safe_out of a solve is the stabilizer applied to (x0, U*[0])."""
    c = sc.config1b(S=512, H=30)
    x0 = np.array(c["x0"])
    x0[3] = x0[2] + 0.95  # hitch near its limit (1.0 at v = -1)
    x0[5] = 0.4
    pd = dict(c["params"], alpha_stab=0.4)
    s = pkg.Solver(pd, max_obstacles=1, max_path_pts=c["path"].shape[0])
    try:
        t = lambda a, dt=torch.float32: torch.as_tensor(np.asarray(a), dtype=dt, device="cuda")
        H = c["params"]["H"]
        inst = dict(x0=t(x0, torch.float64), U_nom=t(c["U_nom"]), obs=t(c["obs"]), path=t(c["path"]),
                    ds=c["ds"], S=512, seed=c["seed"], counter=0,
                    U_out=torch.zeros((H, 3), device="cuda"),
                    u_safe_out=torch.zeros(4, device="cuda"))
        s.solve_device_ex(inst)
        alone = torch.zeros((1, 4), device="cuda")
        s.hitch_stabilize_device(inst["x0"].reshape(1, 7), inst["U_out"][0].reshape(1, 3).contiguous(),
                                 alone)
        torch.cuda.synchronize()
        U = inst["U_out"].cpu().numpy()
        from_solve = inst["u_safe_out"].cpu().numpy().astype(np.float64)
        sep = alone.cpu().numpy()[0].astype(np.float64)
    finally:
        s.close()
    p = sc.as_float32(pd)
    st, o, slack = oracle.hitch_stabilize(p, x0, U[0].astype(np.float64))
    Au, h, br = oracle.hitch_row(p, x0)
    tol, eps_rhs = stab_tolerance(p, x0, Au[:2], o)
    assert np.all(np.abs(from_solve[:2] - o[:2]) <= tol), (from_solve, o)
    assert np.all(np.abs(sep[:2] - o[:2]) <= tol), (sep, o)
    assert from_solve[2] == U[0, 2]
    assert abs(from_solve[3] - slack) <= 4 * eps_rhs + float(np.abs(Au[:2]) @ tol)


# ------------------------------------------------- moving and e = 4 obstacles
@pytest.mark.parametrize("tps", [0, 1, 2, 4, 8])
@pytest.mark.parametrize("seed", range(3))
def test_moving_and_superellipse_obstacles(pkg, tps, seed):
    c = sc.with_moving(sc.small_random(300 + seed, S=300, H=20, n_obs=5), seed)
    assert set(c["obs"][:, 5]) <= {2.0, 4.0}
    p, ref = _oracle(c)
    out = _gpu(pkg, c, tps=tps)
    assert_solve_matches(out, ref, p, f"moving tps={tps} seed={seed}")


def test_crossing_scene(pkg):
    c = sc.crossing(S=1024, H=40)
    p, ref = _oracle(c)
    out = _gpu(pkg, c)
    assert_solve_matches(out, ref, p, "crossing")


def test_exponent_four_needs_the_flag(pkg):
    c = sc.with_moving(sc.small_random(7, S=64, H=8, n_obs=3), 1, e4_frac=1.0)
    rows6 = np.ascontiguousarray(c["obs"][:, :6])
    s = pkg.Solver(dict(c["params"], flags=0), max_obstacles=3, max_path_pts=c["path"].shape[0])
    try:
        st, *_ = pkg.brmppi_solve(s.ctx, c["x0"], c["U_nom"], rows6, c["path"], c["ds"], 1, 0, 8)
        assert st == pkg.BRMPPI_EINVAL
    finally:
        s.close()


# ------------------------------------------------------------ collision cost
def _on_path(c, n):
    """The case with its obstacles moved onto the path ahead (rollouts
    penetrate them without the projection)."""
    o = np.array(c["obs"])
    idx = np.linspace(3, min(len(c["path"]) - 1, 40), n).astype(int)
    o[:n, 0:2] = c["path"][idx, 0:2]
    out = dict(c)
    out["obs"] = o.astype(np.float32)
    return out


@pytest.mark.parametrize("tps", [0, 1, 4])
def test_mppi_collision_cost(pkg, tps):
    c = _on_path(sc.small_random(41, S=400, H=24, n_obs=4), 4)
    flags = sc.FLAG_PROJ_NONE | sc.FLAG_COLLISION_COST
    p, ref = _oracle(c, flags=flags, q_coll=200.0)
    base = oracle.solve(dict(p, flags=sc.FLAG_PROJ_NONE), c["x0"], c["U_nom"], c["obs"], c["path"],
                        c["ds"], c["seed"], c["counter"])
    assert np.max(ref["J"] - base["J"]) > 1.0, "case must penetrate obstacles"
    out = _gpu(pkg, c, tps=tps, flags=flags, q_coll=200.0)
    assert_solve_matches(out, ref, p, f"collision tps={tps}")


def test_collision_cost_with_moving_obstacles(pkg):
    c = sc.with_moving(_on_path(sc.small_random(43, S=256, H=20, n_obs=3), 3), 2, e4_frac=0.3)
    flags = sc.FLAG_PROJ_NONE | sc.FLAG_COLLISION_COST | sc.FLAG_OBS8
    p, ref = _oracle(c, flags=flags)
    out = _gpu(pkg, c, flags=flags)
    assert_solve_matches(out, ref, p, "collision+moving")


# --------------------------------------------------------------- buffer cost
@pytest.mark.parametrize("tps", [0, 1, 2, 8])
def test_alpha_buffer_cost(pkg, tps):
    c = sc.small_random(51, S=300, H=20, n_obs=6)
    over = dict(flags=sc.FLAG_ALPHA_BUFFER, q_abuf=5.0, h_buf=2.0)
    p, ref = _oracle(c, **over)
    plain = oracle.solve(dict(p, flags=0), c["x0"], c["U_nom"], c["obs"], c["path"], c["ds"],
                         c["seed"], c["counter"])
    assert np.max(ref["J"] - plain["J"]) > 0.1, "case must reach the buffer zone"
    out = _gpu(pkg, c, tps=tps, **over)
    assert_solve_matches(out, ref, p, f"buffer tps={tps}")


def test_all_terms_together(pkg):
    c = sc.with_moving(sc.small_random(61, S=333, H=25, n_obs=7), 3)
    over = dict(flags=sc.FLAG_OBS8 | sc.FLAG_ALPHA_BUFFER | sc.FLAG_COLLISION_COST, q_abuf=3.0,
                h_buf=1.0, q_coll=50.0)
    p, ref = _oracle(c, **over)
    out = _gpu(pkg, c, **over)
    assert_solve_matches(out, ref, p, "all terms")


# ------------------------------------------------------ batched and served
def test_batch_with_moving_obstacles(pkg, torch):
    rng = np.random.default_rng(8)
    cases = [sc.with_moving(sc.small_random(int(rng.integers(1 << 30)), S=int(rng.integers(50, 400)),
                                            H=int(rng.integers(5, 30)), n_obs=int(rng.integers(0, 9))),
                            int(rng.integers(1 << 30))) for _ in range(12)]
    pd = dict(sc.params(S=400, H=30), flags=sc.FLAG_OBS8)
    s = pkg.Solver(pd, max_obstacles=8, max_path_pts=512, max_batch=16)
    try:
        t = lambda a, dt=torch.float32: torch.as_tensor(np.asarray(a), dtype=dt, device="cuda")
        insts = []
        for c in cases:
            H = c["params"]["H"]
            insts.append(dict(x0=t(c["x0"], torch.float64), U_nom=t(c["U_nom"]),
                              obs=t(c["obs"]) if len(c["obs"]) else None, path=t(c["path"]),
                              ds=c["ds"], S=c["params"]["S"], seed=c["seed"], counter=c["counter"],
                              U_out=torch.zeros((H, 3), device="cuda"),
                              traj_out=torch.zeros((H + 1, 7), device="cuda"),
                              J_out=torch.zeros(c["params"]["S"], device="cuda"),
                              u_safe_out=torch.zeros(4, device="cuda") if len(insts) % 2 else None))
            add_cost_outputs(insts[-1], c["params"]["S"], H)
        s.solve_batch(insts)
        torch.cuda.synchronize()
        for k, (c, q) in enumerate(zip(cases, insts)):
            p, ref = _oracle(c)
            out = host_outputs(q)
            U = out["U"]
            assert_solve_matches(out, ref, p, f"batch instance {k}")
            if q["u_safe_out"] is not None:
                # the stabilizer on (x0, U*[0]) after the batch
                st, o, slack = oracle.hitch_stabilize(p, c["x0"], U[0].astype(np.float64))
                Au, h, br = oracle.hitch_row(p, c["x0"])
                tol, eps_rhs = stab_tolerance(p, c["x0"], Au[:2], o)
                g = q["u_safe_out"].cpu().numpy().astype(np.float64)
                assert np.all(np.abs(g[:2] - o[:2]) <= tol), (k, g, o)
                assert g[2] == U[0, 2]
    finally:
        s.close()


def test_served_moving_obstacles(pkg):
    c = sc.with_moving(sc.small_random(71, S=256, H=16, n_obs=4), 9)
    pd = c["params"]
    s = pkg.Solver(pd, max_obstacles=8, max_path_pts=512, max_vehicles=2, max_batch=1)
    try:
        s.register(0, c["path"], c["ds"], c["U_nom"], c["seed"])
        st, t = s.submit(0, c["x0"], c["obs"])
        assert st == 0
        import time
        t0 = time.time()
        while True:
            st, U, traj, lat = s.poll(t, True)
            if st != pkg.BRMPPI_EAGAIN:
                break
            assert time.time() - t0 < 30
            time.sleep(1e-4)
        assert st == 0
        p = sc.as_float32(pd)
        ref = oracle.solve(p, c["x0"], c["U_nom"], c["obs"], c["path"], c["ds"], c["seed"], 0,
                           want_uhist=True)
        sv = served_costs(s, c, c["U_nom"], c["seed"], 0, U)
        assert_solve_matches(dict(U=U, traj=traj, **sv), ref, p, "served moving")
    finally:
        s.close()


# ------------------------------------------------------------ footprint discs
def _discs(c, **kw):
    out = dict(c)
    out["params"] = dict(c["params"], **sc.FIVE_DISCS, **kw)
    return out


@pytest.mark.parametrize("tps", [0, 1, 2, 4, 8])
def test_footprint_discs(pkg, tps):
    c = _discs(sc.small_random(81, S=300, H=20, n_obs=4), r_inflate=0.3)
    p, ref = _oracle(c)
    out = _gpu(pkg, c, tps=tps)
    assert_solve_matches(out, ref, p, f"discs tps={tps}")


@pytest.mark.parametrize("flags", [sc.FLAG_OBS8, sc.FLAG_ALPHA_BUFFER, sc.FLAG_COLLISION_COST])
def test_discs_with_one_optional_term(pkg, flags):
    c = _discs(sc.with_moving(sc.small_random(83, S=257, H=18, n_obs=5), 4), flags=flags, q_abuf=3.0,
               h_buf=1.0)
    if not flags & sc.FLAG_OBS8:  # rows of 6: parked ellipses
        c["obs"] = np.ascontiguousarray(
            np.hstack([c["obs"][:, :5], np.full((len(c["obs"]), 1), 2.0, np.float32)]))
    p, ref = _oracle(c)
    out = _gpu(pkg, c)
    extra = buffer_conditioning(p, c) if flags & sc.FLAG_ALPHA_BUFFER else None
    assert_solve_matches(out, ref, p, f"discs + flags {flags}", j_extra=extra)


def test_discs_with_every_optional_term(pkg):
    c = _discs(sc.with_moving(sc.small_random(83, S=257, H=18, n_obs=5), 4),
               flags=sc.FLAG_OBS8 | sc.FLAG_ALPHA_BUFFER | sc.FLAG_COLLISION_COST, q_abuf=3.0, h_buf=1.0)
    p, ref = _oracle(c)
    out = _gpu(pkg, c)
    assert_solve_matches(out, ref, p, "discs + all terms", j_extra=buffer_conditioning(p, c))


def test_mppi_collision_cost_with_discs(pkg):
    c = _discs(_on_path(sc.small_random(85, S=300, H=20, n_obs=3), 3),
               flags=sc.FLAG_PROJ_NONE | sc.FLAG_COLLISION_COST)
    p, ref = _oracle(c)
    out = _gpu(pkg, c)
    assert_solve_matches(out, ref, p, "collision + discs")


def test_batch_and_serving_with_discs(pkg, torch):
    rng = np.random.default_rng(86)
    cases = [_discs(sc.small_random(int(rng.integers(1 << 30)), S=int(rng.integers(50, 300)), H=16,
                                    n_obs=int(rng.integers(0, 6)))) for _ in range(8)]
    pd = dict(sc.params(S=300, H=16), **sc.FIVE_DISCS)
    s = pkg.Solver(pd, max_obstacles=6, max_path_pts=512, max_batch=8, max_vehicles=2)
    try:
        t = lambda a, dt=torch.float32: torch.as_tensor(np.asarray(a), dtype=dt, device="cuda")
        insts = [dict(x0=t(c["x0"], torch.float64), U_nom=t(c["U_nom"]),
                      obs=t(c["obs"]) if len(c["obs"]) else None, path=t(c["path"]), ds=c["ds"],
                      S=c["params"]["S"], seed=c["seed"], counter=c["counter"],
                      U_out=torch.zeros((16, 3), device="cuda"),
                      traj_out=torch.zeros((17, 7), device="cuda"),
                      J_out=torch.zeros(c["params"]["S"], device="cuda")) for c in cases]
        for c, q in zip(cases, insts):
            add_cost_outputs(q, c["params"]["S"], 16)
        s.solve_batch(insts)
        torch.cuda.synchronize()
        for k, (c, q) in enumerate(zip(cases, insts)):
            p, ref = _oracle(c)
            assert_solve_matches(host_outputs(q), ref, p, f"disc batch {k}")
        # serving: one vehicle, one request
        c = _discs(sc.small_random(87, S=300, H=16, n_obs=4))
        s.register(0, c["path"], c["ds"], c["U_nom"], c["seed"])
        st, tk = s.submit(0, c["x0"], c["obs"])
        assert st == 0
        import time
        t0 = time.time()
        while True:
            st, U, traj, lat = s.poll(tk, True)
            if st != pkg.BRMPPI_EAGAIN:
                break
            assert time.time() - t0 < 30
            time.sleep(1e-4)
        assert st == 0
        p = sc.as_float32(c["params"])
        ref = oracle.solve(p, c["x0"], c["U_nom"], c["obs"], c["path"], c["ds"], c["seed"], 0,
                           want_uhist=True)
        sv = served_costs(s, c, c["U_nom"], c["seed"], 0, U)
        assert_solve_matches(dict(U=U, traj=traj, **sv), ref, p, "served discs")
    finally:
        s.close()


# ------------------------------------------------------------ third-order rows
@pytest.mark.parametrize("tps", [0, 1, 4, 8])
def test_third_order_rows(pkg, tps):
    c = sc.small_random(91, S=300, H=20, n_obs=5)
    p, ref = _oracle(c, flags=sc.FLAG_THIRD_ORDER)
    out = _gpu(pkg, c, tps=tps, flags=sc.FLAG_THIRD_ORDER)
    assert_solve_matches(out, ref, p, f"third order tps={tps}")


def test_third_order_with_moving_superellipses(pkg):
    c = sc.with_moving(sc.small_random(93, S=300, H=20, n_obs=6), 5)
    flags = sc.FLAG_OBS8 | sc.FLAG_THIRD_ORDER
    p, ref = _oracle(c, flags=flags)
    out = _gpu(pkg, c, flags=flags)
    assert_solve_matches(out, ref, p, "third order + moving")


# ------------------------------------------------------------ jerk-input model
def _ref7(ref):
    out = dict(ref)
    out["traj"] = ref["traj"][:, :7]  # the GPU outputs keep 7 state columns
    return out


@pytest.mark.parametrize("tps", [0, 1, 4, 8])
def test_jerk_model(pkg, tps):
    c = sc.jerk_model(sc.small_random(101, S=300, H=20, n_obs=5), a0=0.3, seed=1)
    p, ref = _oracle(c)
    out = _gpu(pkg, c, tps=tps)
    assert_solve_matches(out, _ref7(ref), p, f"jerk tps={tps}")


def test_jerk_model_third_order_and_moving(pkg):
    c = sc.jerk_model(sc.with_moving(sc.small_random(103, S=300, H=20, n_obs=5), 2), a0=-0.4, seed=2)
    flags = c["params"]["flags"] | sc.FLAG_THIRD_ORDER
    p, ref = _oracle(c, flags=flags)
    out = _gpu(pkg, c, flags=flags)
    assert_solve_matches(out, _ref7(ref), p, "jerk third order + moving")


def test_jerk_model_stabilizer(pkg, torch):
    pd = sc.params(flags=sc.FLAG_JERK, alpha_stab=0.6)
    p = sc.as_float32(pd)
    rng = np.random.default_rng(7)
    X, U = _stab_cases(sc.as_float32(sc.params(alpha_stab=0.6)), rng, 600)
    X = np.hstack([X, rng.uniform(-1.0, 1.0, (len(X), 1))])  # acceleration state
    s = pkg.Solver(pd)
    try:
        out = torch.zeros((len(X), 4), dtype=torch.float32, device="cuda")
        s.hitch_stabilize_device(torch.from_numpy(X).cuda(), torch.from_numpy(U).cuda(), out)
        torch.cuda.synchronize()
        G = out.cpu().numpy().astype(np.float64)
    finally:
        s.close()
    for i in range(len(X)):
        st, o, slack = oracle.hitch_stabilize(p, X[i], U[i].astype(np.float64))
        Au, h, br = oracle.jerk_hitch_row(p, X[i])
        tol, eps_rhs = stab_tolerance(p, X[i], Au[:2], o)
        eps_rhs += 8 * 2.0 ** -23 * abs(X[i][7] * 0.05)  # the folded a-term
        assert abs(G[i, 3] - slack) <= 4 * eps_rhs + float(np.abs(Au[:2]) @ tol) + 1e-6, (i, G[i], slack)
        if st == 1 and slack < -4 * eps_rhs - 1e-6:
            np.testing.assert_array_equal(G[i, :2], o[:2].astype(np.float32), err_msg=str(i))
            continue
        assert np.all(np.abs(G[i, :2] - o[:2]) <= tol + 1e-5), (i, G[i], o, tol)


def test_jerk_model_batch(pkg, torch):
    rng = np.random.default_rng(104)
    cases = [sc.jerk_model(sc.small_random(int(rng.integers(1 << 30)), S=int(rng.integers(50, 300)), H=16,
                                           n_obs=int(rng.integers(0, 6))), a0=float(rng.uniform(-1, 1)),
                           seed=k) for k in range(6)]
    pd = cases[0]["params"] | dict(S=300, H=16)
    s = pkg.Solver(pd, max_obstacles=6, max_path_pts=512, max_batch=8)
    try:
        t = lambda a, dt=torch.float32: torch.as_tensor(np.asarray(a), dtype=dt, device="cuda")
        insts = [dict(x0=t(c["x0"], torch.float64), U_nom=t(c["U_nom"]),
                      obs=t(c["obs"]) if len(c["obs"]) else None, path=t(c["path"]), ds=c["ds"],
                      S=c["params"]["S"], seed=c["seed"], counter=c["counter"],
                      U_out=torch.zeros((16, 3), device="cuda"), traj_out=torch.zeros((17, 7), device="cuda"),
                      J_out=torch.zeros(c["params"]["S"], device="cuda")) for c in cases]
        for c, q in zip(cases, insts):
            add_cost_outputs(q, c["params"]["S"], 16)
        s.solve_batch(insts)
        torch.cuda.synchronize()
        for k, (c, q) in enumerate(zip(cases, insts)):
            p, ref = _oracle(c)
            assert_solve_matches(host_outputs(q), _ref7(ref), p, f"jerk batch {k}")
    finally:
        s.close()


# ------------------------------------------------- three blocks per lane
@pytest.mark.parametrize("moving", [False, True])
@pytest.mark.parametrize("tps,n_obs", [(4, 30), (8, 64)])
def test_three_blocks_per_lane_variants(pkg, tps, n_obs, moving):
    """Teams of 4 (8) lanes drawing 9..12 (17..24) Philox blocks per step
    run the variants with three blocks per lane, in both kernel families
    (moving and e = 4 rows select the extended one)."""
    c = sc.small_random(131 + n_obs, S=200, H=12, n_obs=n_obs)
    if moving:
        c = sc.with_moving(c, seed=7)
    p, ref = _oracle(c)
    out = _gpu(pkg, c, tps=tps, threads=128)
    assert_solve_matches(out, ref, p, f"tps={tps} n_obs={n_obs} moving={moving}")
