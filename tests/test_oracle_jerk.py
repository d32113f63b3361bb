"""Pins of the oracle's jerk-input model (the paper's form of the
kinematics, Sec. III-A: the longitudinal acceleration a is a state driven by
the jerk; inputs (jerk, steer rate, progress rate)).

* the Euler step against the discrete closed form of constant jerk, and
  against the acceleration model driven by the state's a;
* every row against a fine RK4 of the 8-state field (O(Ts^3) miss at second
  order, O(Ts^4) with third-order obstacle rows);
* the rows against the acceleration model's (separately pinned) rows: with
  a held, the jerk row's constant is the acceleration row's constant plus
  a times its a-coefficient, its steer-rate column is the same, and its
  jerk column is zero for obstacles at second order (relative degree 3),
  -kappa Ts^2/2 for the hitch, and Ts/3 times the second-order
  a-coefficient for third-order obstacle rows.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2508_05773_gb300 import scenarios as sc

BASE = sc.params(flags=sc.FLAG_JERK)


def _field8(p, x, u):
    px, py, th1, th2, v, delta, psi, a = x
    j, om, nu = u
    k = p["lh"] / p["l1"]
    t = math.tan(delta)
    return np.array([v * math.cos(th1), v * math.sin(th1), v * t / p["l1"],
                     v / p["l2"] * (math.sin(th1 - th2) - k * math.cos(th1 - th2) * t),
                     a, om, nu, j])


def _flow8(p, x0, u, T, n=2000):
    x = np.array(x0, dtype=np.float64)
    h = T / n
    for _ in range(n):
        k1 = _field8(p, x, u)
        k2 = _field8(p, x + 0.5 * h * k1, u)
        k3 = _field8(p, x + 0.5 * h * k2, u)
        k4 = _field8(p, x + h * k3, u)
        x = x + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    return x


STATES = [(0.5, 0.2, 0.4, 0.3, 1.2, 0.25, 0.0, 0.7),
          (0.0, 0.0, math.pi, math.pi - 0.3, -1.0, -0.3, 0.0, -0.5),
          (1.0, -1.0, 0.0, 0.6, 2.0, 0.1, 0.0, 1.5)]
OBS = [(3.0, 1.0, 1.0, 0.6, 0.3, 2.0, 0.0, 0.0), (-2.0, 2.5, 1.5, 0.6, 2.2, 4.0, 0.5, -0.4)]
U = (0.8, -0.5, 1.0)


def test_constant_jerk_closed_form():
    p = sc.params(flags=sc.FLAG_JERK, Ts=0.1)
    x = np.array([0.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.3])
    j = 0.5
    for k in range(1, 30):
        x = oracle.jerk_step(p, x, (j, 0.0, 0.0))
        Ts = p["Ts"]
        np.testing.assert_allclose(x[7], 0.3 + k * Ts * j, rtol=1e-13)
        np.testing.assert_allclose(x[4], 1.0 + k * Ts * 0.3 + Ts * Ts * j * k * (k - 1) / 2, rtol=1e-13)
    assert x[1] == 0.0 and x[2] == 0.0 and x[3] == 0.0


@pytest.mark.parametrize("x", STATES)
def test_step_is_the_acceleration_model_driven_by_the_state(x):
    xn = oracle.jerk_step(BASE, x, (0.9, -0.2, 1.5))
    xa = oracle.dynamics_step(sc.params(), x[:7], (x[7], -0.2, 1.5))
    np.testing.assert_array_equal(xn[:7], xa)
    np.testing.assert_allclose(xn[7], x[7] + BASE["Ts"] * 0.9, rtol=1e-15)


def _miss(kind, p, x0, obs=None, t0=0.0):
    if kind == "hitch":
        Au, h, br = oracle.jerk_hitch_row(p, x0)
        h1 = oracle.hitch_h(p, _flow8(p, x0, U, p["Ts"])[:7])
    else:
        Au, h, br = oracle.jerk_obstacle_row(p, obs, x0, t0)
        h1 = oracle.obstacle_h_at(p, obs, _flow8(p, x0, U, p["Ts"])[:7], t0 + p["Ts"])
    return (h1 - h) - (float(np.dot(Au, U)) - br)


@pytest.mark.parametrize("x0", STATES)
def test_hitch_row_is_second_order_taylor(x0):
    ms = [_miss("hitch", sc.params(flags=sc.FLAG_JERK, Ts=T), x0) for T in (0.04, 0.02, 0.01)]
    assert abs(ms[0]) / abs(ms[1]) > 5.5 and abs(ms[1]) / abs(ms[2]) > 5.5, ms


@pytest.mark.parametrize("x0", STATES)
@pytest.mark.parametrize("obs", OBS)
@pytest.mark.parametrize("third", [False, True])
def test_obstacle_row_taylor_order(x0, obs, third):
    flags = sc.FLAG_JERK | (sc.FLAG_THIRD_ORDER if third else 0)
    ms = [_miss("obs", sc.params(flags=flags, Ts=T), x0, obs, 0.3) for T in (0.04, 0.02, 0.01)]
    lo = 11.0 if third else 5.5
    assert abs(ms[0]) / abs(ms[1]) > lo and abs(ms[1]) / abs(ms[2]) > lo, ms


@pytest.mark.parametrize("x", STATES)
def test_rows_match_the_acceleration_model(x):
    pa, pj = sc.params(), BASE
    a = x[7]
    A, h, br = oracle.jerk_hitch_row(pj, x)
    Aa, ha, bra = oracle.hitch_row(pa, x[:7])
    assert h == ha
    np.testing.assert_allclose(A[0], -pa["kappa"] * 0.5 * pa["Ts"] ** 2, rtol=1e-12)
    np.testing.assert_allclose(A[1], Aa[1], rtol=1e-12, atol=1e-18)
    np.testing.assert_allclose(br, bra - a * Aa[0], rtol=1e-11, atol=1e-15)
    for obs in OBS:
        A, h, br = oracle.jerk_obstacle_row(pj, obs, x, 0.4)
        Aa, ha, bra = oracle.obstacle_row_at(pa, obs, x[:7], 0.4)
        np.testing.assert_allclose(h, ha, rtol=1e-14)
        assert A[0] == 0.0 and A[1] == 0.0 and A[2] == 0.0  # relative degree 3
        np.testing.assert_allclose(br, bra - a * Aa[0], rtol=1e-11, atol=1e-15)
        # third order: steer rate as in the acceleration model, jerk column
        # Ts/3 times the second-order a-coefficient
        p3j = sc.params(flags=sc.FLAG_JERK | sc.FLAG_THIRD_ORDER)
        p3a = sc.params(flags=sc.FLAG_THIRD_ORDER)
        A3, _, br3 = oracle.jerk_obstacle_row(p3j, obs, x, 0.4)
        A3a, _, br3a = oracle.obstacle_row3(p3a, obs, x[:7], 0.4)
        np.testing.assert_allclose(A3[1], A3a[1], rtol=1e-11, atol=1e-18)
        np.testing.assert_allclose(A3[0], pa["Ts"] / 3.0 * Aa[0], rtol=1e-11, atol=1e-18)
        np.testing.assert_allclose(br3, br3a - a * A3a[0], rtol=1e-10, atol=1e-14)


def test_rollout_rows_and_zero_noise_integration():
    c = sc.jerk_model(sc.small_random(31, S=4, H=10, n_obs=3), a0=0.4, seed=3)
    p = sc.as_float32(dict(c["params"], S=4, H=10))
    r = oracle.rollout_sample(p, c["x0"], c["U_nom"], c["obs"], c["path"], c["ds"], c["seed"], 0, 1)
    assert r["status"] == 0 and r["states"].shape == (11, 8)
    for k in range(p["H"]):
        x, zs = r["states"][k], r["z_star"][k]
        Au, h, br = oracle.jerk_hitch_row(p, x)
        ht = math.copysign(max(abs(h), p["h_floor"]), h if h != 0 else 1.0)
        np.testing.assert_allclose(float(np.dot(Au, zs[:3])) + ht * zs[3], -r["alpha"][k, 0] * h + br,
                                   rtol=1e-9, atol=1e-9)
        for o in range(3):
            Au, h, br = oracle.jerk_obstacle_row(p, c["obs"][o], x, k * p["Ts"])
            ht = math.copysign(max(abs(h), p["h_floor"]), h if h != 0 else 1.0)
            lhs = float(np.dot(Au, zs[:3])) + ht * zs[4 + o]
            np.testing.assert_allclose(lhs, -r["alpha"][k, 1 + o] * h + br, rtol=1e-9, atol=1e-9)
    # zero noise: every rollout is the integration of its applied inputs
    p0 = dict(p, sigma=(0.0, 0.0, 0.0), sigma_alpha=0.0)
    r0 = oracle.rollout_sample(p0, c["x0"], c["U_nom"], c["obs"], c["path"], c["ds"], c["seed"], 0, 0)
    np.testing.assert_allclose(oracle.jerk_integrate(p0, c["x0"], r0["u"]), r0["states"], rtol=1e-12,
                               atol=1e-12)


def test_jerk_model_refuses_offset_discs():
    c = sc.jerk_model(sc.small_random(31, S=4, H=6, n_obs=2))
    p = sc.as_float32(dict(c["params"], S=4, H=6, **sc.FIVE_DISCS))
    r = oracle.rollout_sample(p, c["x0"], c["U_nom"], c["obs"], c["path"], c["ds"], c["seed"], 0, 0)
    assert r["status"] == -1
