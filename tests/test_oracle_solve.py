"""Solve-level pins of the oracle (Sec. II-B MPPI with the BR-MPPI rollout of
Sec. IV-A): zero-noise rollouts equal a deterministic integration written
here, the equality rows hold for every projected z with the realised rate,
applied inputs respect their bounds, equal costs give the mean of the
samples, and the update is the softmin-weighted mean of applied inputs."""
import math

import numpy as np
import pytest

import oracle
from paper_2508_05773_gb300 import scenarios as sc


def _euler(p, x0, U):
    """Independent explicit Euler of the kinematics (Sec. III-A)."""
    x = np.array(x0, dtype=np.float64)
    out = [x.copy()]
    k = p["lh"] / p["l1"]
    for a, om, nu in U:
        px, py, th1, th2, v, dl, psi = x
        t = math.tan(dl)
        x = np.array([px + p["Ts"] * v * math.cos(th1), py + p["Ts"] * v * math.sin(th1),
                      th1 + p["Ts"] * v * t / p["l1"],
                      th2 + p["Ts"] * v / p["l2"] * (math.sin(th1 - th2) - k * math.cos(th1 - th2) * t),
                      v + p["Ts"] * a, dl + p["Ts"] * om, psi + p["Ts"] * nu])
        out.append(x.copy())
    return np.array(out)


def _run(c, **over):
    p = sc.as_float32(dict(c["params"], **over))
    return p, oracle.solve(p, c["x0"], c["U_nom"], c["obs"], c["path"], c["ds"], c["seed"],
                           c["counter"], want_uhist=True, want_states=True)


def test_zero_noise_standard_mppi_is_plain_euler():
    c = sc.small_random(3, S=16, H=10)
    p, r = _run(c, sigma=(0.0, 0.0, 0.0), sigma_alpha=0.0, flags=sc.FLAG_PROJ_NONE)
    assert r["status"] == 0
    U = np.clip(c["U_nom"].astype(np.float64), p["z_lo"], p["z_hi"])
    np.testing.assert_allclose(r["U"], U, rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(r["traj"], _euler(p, c["x0"], U), rtol=1e-13, atol=1e-13)
    for s in range(16):
        np.testing.assert_allclose(r["states"][s], _euler(p, c["x0"], U), rtol=1e-13, atol=1e-13)


def test_zero_noise_brmppi_rollouts_identical():
    c = sc.small_random(4, S=8, H=12)
    p, r = _run(c, sigma=(0.0, 0.0, 0.0), sigma_alpha=0.0)
    assert np.all(r["J"] == r["J"][0])
    assert np.all(r["u_hist"] == r["u_hist"][0])
    np.testing.assert_allclose(r["U"], r["u_hist"][0], rtol=1e-14, atol=1e-15)
    # the optimal trajectory is the integration of U*, which reproduces the
    # rollout's own states
    np.testing.assert_allclose(r["traj"], _euler(p, c["x0"], r["U"]), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(r["states"][0], r["traj"], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_equality_rows_hold_and_bounds(seed):
    c = sc.small_random(seed, S=4, H=15, n_obs=3)
    p = sc.as_float32(c["params"])
    obs = c["obs"].astype(np.float64)
    n_obs = obs.shape[0]
    clipped = 0
    for s in range(4):
        r = oracle.rollout_sample(p, c["x0"], c["U_nom"], obs, c["path"], c["ds"], c["seed"],
                                  c["counter"], s)
        assert r["status"] == 0
        for tau in range(p["H"]):
            x = r["states"][tau]
            zs = r["z_star"][tau]
            al = r["alpha"][tau]
            for i in range(1 + n_obs):
                Au, h, br = (oracle.hitch_row(p, x) if i == 0 else oracle.obstacle_row(p, obs[i - 1], x))
                ht = math.copysign(max(abs(h), p["h_floor"]), h if h != 0 else 1.0)
                lhs = float(np.dot(Au, zs[:3])) + ht * zs[3 + i]
                rhs = -al[i] * h + br
                assert abs(lhs - rhs) <= 1e-9 * max(1.0, abs(rhs))
                # realised barrier-rate: the Taylor increment equals
                # -(alpha + u_alpha) h  (up to the floor on h)
                if abs(h) > p["h_floor"]:
                    inc = float(np.dot(Au, zs[:3])) - br
                    np.testing.assert_allclose(inc, -(al[i] + zs[3 + i]) * h, rtol=1e-9, atol=1e-12)
                # barrier rate update
                np.testing.assert_allclose(r["alpha"][tau + 1][i], al[i] + zs[3 + i], rtol=1e-15)
            u = r["u"][tau]
            assert np.all(u >= np.array(p["z_lo"])) and np.all(u <= np.array(p["z_hi"]))
            inside = np.all(zs[:3] >= np.array(p["z_lo"])) and np.all(zs[:3] <= np.array(p["z_hi"]))
            if inside:
                assert np.array_equal(u, zs[:3])
            else:
                clipped += 1
            # sampled input respects its bounds before projection
            zd = r["z_des"][tau]
            assert np.all(zd[:3] >= np.array(p["z_lo"])) and np.all(zd[:3] <= np.array(p["z_hi"]))
            assert np.all(zd[3:] >= p["ua_lo"]) and np.all(zd[3:] <= p["ua_hi"])
    assert clipped < 4 * p["H"]


def test_post_projection_clip():
    # A costly barrier rate (large w_alpha) makes the projection move the
    # physical inputs, often out of the box: the applied input is then the
    # clipped z*, within bounds, and equals z* wherever z* is inside.
    c = sc.config1b(S=4, H=40)
    p = sc.as_float32(dict(c["params"], w_alpha=1e4))
    lo, hi = np.array(p["z_lo"]), np.array(p["z_hi"])
    n_out = 0
    for s in range(4):
        r = oracle.rollout_sample(p, c["x0"], c["U_nom"], c["obs"], c["path"], c["ds"], c["seed"],
                                  c["counter"], s)
        zs = r["z_star"][:, :3]
        np.testing.assert_array_equal(r["u"], np.clip(zs, lo, hi))
        n_out += int(np.sum((zs < lo) | (zs > hi)))
    assert n_out > 0


def test_update_is_weighted_mean_of_applied_inputs():
    c = sc.config1(S=64, H=20)
    p, r = _run(c)
    st, g = oracle.softmin(r["J"], p["lambda"])
    np.testing.assert_allclose(r["U"], np.einsum("s,shj->hj", g, r["u_hist"]), rtol=1e-12,
                               atol=1e-14)
    # "mean perturbation" form of the same update
    du = r["u_hist"] - c["U_nom"][None].astype(np.float64)
    np.testing.assert_allclose(r["U"], c["U_nom"] + np.einsum("s,shj->hj", g, du), atol=1e-12)


def test_equal_costs_give_mean_of_samples():
    c = sc.config1(S=32, H=10)
    p, r = _run(c, **{"lambda": 1e12})
    np.testing.assert_allclose(r["U"], r["u_hist"].mean(axis=0), rtol=1e-9, atol=1e-12)


def test_rollout_sample_matches_solve_and_is_deterministic():
    c = sc.small_random(7, S=6, H=9)
    p, r = _run(c)
    for s in (0, 5):
        one = oracle.rollout_sample(p, c["x0"], c["U_nom"], c["obs"], c["path"], c["ds"], c["seed"],
                                    c["counter"], s)
        np.testing.assert_array_equal(one["states"], r["states"][s])
        np.testing.assert_array_equal(one["u"], r["u_hist"][s])
        assert one["J"] == r["J"][s]
    p2, r2 = _run(c)
    np.testing.assert_array_equal(r2["U"], r["U"])
    c3 = dict(c, counter=c["counter"] + 1)
    p3, r3 = _run(c3)
    assert not np.array_equal(r3["U"], r["U"])


def test_cost_accumulates_stage_costs_after_each_step():
    c = sc.small_random(9, S=2, H=8)
    p = sc.as_float32(c["params"])
    one = oracle.rollout_sample(p, c["x0"], c["U_nom"], c["obs"], c["path"], c["ds"], c["seed"],
                                c["counter"], 1)
    J = sum(oracle.stage_cost(p, one["states"][k + 1], one["u"][k], c["path"], c["ds"])
            for k in range(p["H"]))
    np.testing.assert_allclose(one["J"], J, rtol=1e-14)


def test_invalid_inputs():
    c = sc.small_random(1, S=4, H=5)
    p = sc.as_float32(c["params"])
    bad = c["obs"].copy()
    bad[0, 5] = 3.0  # odd exponent
    r = oracle.solve(p, c["x0"], c["U_nom"], bad, c["path"], c["ds"], c["seed"], c["counter"])
    assert r["status"] == oracle.ORC_EINVAL
    r = oracle.solve(p, c["x0"], c["U_nom"], c["obs"], c["path"][:1], c["ds"], c["seed"], c["counter"])
    assert r["status"] == oracle.ORC_EINVAL


def test_no_obstacles_only_hitch():
    c = sc.small_random(2, S=8, H=6, n_obs=0)
    p, r = _run(c)
    assert r["status"] == 0
    assert np.all(np.isfinite(r["U"]))


def test_sample_ranges_and_update_reassemble_the_solve():
    # A solve spread over sample ranges (one per worker process) and joined
    # by the update gives the full solve's costs, inputs and U* bit for bit.
    c = sc.small_random(12, S=37, H=9, n_obs=3)
    p, ref = _run(c)
    args = (p, c["x0"], c["U_nom"], c["obs"], c["path"], c["ds"], c["seed"], c["counter"])
    parts = [oracle.rollouts(*args, s0, s1) for s0, s1 in ((0, 5), (5, 6), (6, 37))]
    assert all(r["status"] == 0 for r in parts)
    J = np.concatenate([r["J"] for r in parts])
    uh = np.concatenate([r["u_hist"] for r in parts])
    st, U, g = oracle.update(J, uh, p["lambda"], c["U_nom"])
    assert st == 0
    assert np.array_equal(J, ref["J"]) and np.array_equal(uh, ref["u_hist"]) and np.array_equal(U, ref["U"])
    # the update is the weighted mean of the applied inputs with the softmin
    # weights (non-negative, summing to 1), written out here
    w = np.exp(-(J - J.min()) / p["lambda"])
    np.testing.assert_allclose(g, w / w.sum(), rtol=1e-13)
    np.testing.assert_allclose(U, np.einsum("s,shj->hj", w / w.sum(), uh), rtol=1e-12, atol=1e-15)


def test_update_without_finite_costs_returns_the_nominal():
    U_nom = np.arange(12, dtype=np.float64).reshape(4, 3)
    st, U, g = oracle.update(np.array([np.inf, np.nan]), np.ones((2, 4, 3)), 1.0, U_nom)
    assert st == oracle.ORC_ENONFINITE
    assert np.array_equal(U, U_nom) and np.all(g == 0)
