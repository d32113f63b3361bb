"""Pins of the oracle's barrier functions and barrier-rate rows
(Sec. IV-C Eq. barrier_function / barrier_function_approx, Sec. IV-D
Eq. hitch_angle_barrier, Sec. IV-A Eq. cbf_equality).

The rows claim  L_f h + L_g h u = Ts hdot + Ts^2/2 hddot  along the
continuous vector field with the input held.  The test integrates that
vector field with a fine RK4 of its own and checks that the row's prediction
misses the true change of h by O(Ts^3): halving Ts divides the miss by ~8.
A dropped term, a wrong sign or a transposed rotation breaks the ratio.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2508_05773_gb300 import scenarios as sc

BASE = sc.params()


def _field(p, x, u):
    px, py, th1, th2, v, delta, psi = x
    a, om, nu = u
    k = p["lh"] / p["l1"]
    t = math.tan(delta)
    return np.array([
        v * math.cos(th1), v * math.sin(th1), v * t / p["l1"],
        v / p["l2"] * (math.sin(th1 - th2) - k * math.cos(th1 - th2) * t),
        a, om, nu])


def _flow(p, x0, u, T, n=2000):
    x = np.array(x0, dtype=np.float64)
    h = T / n
    for _ in range(n):
        k1 = _field(p, x, u)
        k2 = _field(p, x + 0.5 * h * k1, u)
        k3 = _field(p, x + 0.5 * h * k2, u)
        k4 = _field(p, x + h * k3, u)
        x = x + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    return x


def _miss(kind, p, x0, u, obs=None):
    if kind == "obs":
        Au, h, br = oracle.obstacle_row(p, obs, x0)
        h1 = oracle.obstacle_h(p, obs, _flow(p, x0, u, p["Ts"]))
    else:
        Au, h, br = oracle.hitch_row(p, x0)
        h1 = oracle.hitch_h(p, _flow(p, x0, u, p["Ts"]))
    predicted = float(np.dot(Au, u)) - br
    return (h1 - h) - predicted


OBSTACLES = [
    (3.0, 1.0, 1.0, 0.6, 0.3, 2.0),
    (-2.0, 2.5, 1.5, 0.4, 2.2, 2.0),
    (2.0, -1.0, 0.8, 0.8, 0.0, 4.0),   # even exponent 4 (super-ellipse)
]
STATES = [
    (0.5, 0.2, 0.4, 0.3, 1.2, 0.25, 0.0),
    (0.0, 0.0, math.pi, math.pi - 0.1, -1.0, -0.3, 0.0),
]
INPUTS = [(0.8, -0.4, 1.0), (-1.5, 0.5, 0.0)]


@pytest.mark.parametrize("obs", OBSTACLES)
@pytest.mark.parametrize("x0", STATES)
@pytest.mark.parametrize("u", INPUTS)
def test_obstacle_row_is_second_order_taylor(obs, x0, u):
    m1 = _miss("obs", sc.params(Ts=0.2), x0, u, obs)
    m2 = _miss("obs", sc.params(Ts=0.1), x0, u, obs)
    m3 = _miss("obs", sc.params(Ts=0.05), x0, u, obs)
    assert abs(m2) < 0.2 * abs(m1) + 1e-13
    r = m2 / m3
    assert 5.5 < r < 11.0, (m1, m2, m3)


@pytest.mark.parametrize("x0", [
    (0.0, 0.0, 0.5, 0.7, 1.1, 0.2, 0.0),       # Delta > 0
    (0.0, 0.0, 3.0, 2.6, -1.0, -0.35, 0.0),    # Delta < 0, reversing
    (0.0, 0.0, 1.0, 1.3, -0.7, 0.4, 0.0),
])
@pytest.mark.parametrize("u", INPUTS)
def test_hitch_row_is_second_order_taylor(x0, u):
    m1 = _miss("hitch", sc.params(Ts=0.2), x0, u)
    m2 = _miss("hitch", sc.params(Ts=0.1), x0, u)
    m3 = _miss("hitch", sc.params(Ts=0.05), x0, u)
    r = m2 / m3
    assert 5.5 < r < 11.0, (m1, m2, m3)


def test_obstacle_barrier_values():
    p = BASE
    obs = (1.0, 2.0, 2.0, 1.0, 0.0, 2.0)
    assert oracle.obstacle_h(p, obs, (1.0, 2.0, 0, 0, 0, 0, 0)) == -1.0   # centre
    np.testing.assert_allclose(oracle.obstacle_h(p, obs, (3.0, 2.0, 0, 0, 0, 0, 0)), 0.0, atol=1e-15)
    np.testing.assert_allclose(oracle.obstacle_h(p, obs, (1.0, 3.0, 0, 0, 0, 0, 0)), 0.0, atol=1e-15)
    # rotation by pi/2 swaps the axes
    obs_r = (1.0, 2.0, 2.0, 1.0, math.pi / 2, 2.0)
    np.testing.assert_allclose(oracle.obstacle_h(p, obs_r, (1.0, 4.0, 0, 0, 0, 0, 0)), 0.0, atol=1e-12)
    # footprint inflation: semi-axes grow by r
    p2 = sc.params(r_inflate=0.5)
    np.testing.assert_allclose(oracle.obstacle_h(p2, obs, (3.5, 2.0, 0, 0, 0, 0, 0)), 0.0, atol=1e-15)
    # odd or fractional exponents are rejected
    assert math.isnan(oracle.obstacle_h(p, (0, 0, 1, 1, 0, 3.0), (0, 0, 0, 0, 0, 0, 0)))
    assert math.isnan(oracle.obstacle_h(p, (0, 0, 1, 1, 0, 2.5), (0, 0, 0, 0, 0, 0, 0)))


def test_circle_rows_invariant_to_heading():
    x0 = STATES[0]
    rows = [oracle.obstacle_row(BASE, (2.0, 1.0, 0.9, 0.9, th, 2.0), x0) for th in (0.0, 0.7, 2.5)]
    for Au, h, br in rows[1:]:
        np.testing.assert_allclose(Au, rows[0][0], rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(h, rows[0][1], rtol=1e-12)
        np.testing.assert_allclose(br, rows[0][2], rtol=1e-12)


def test_obstacle_row_inputs():
    # steer rate and progress rate do not enter an obstacle row at second
    # order; a stationary vehicle has no hdot and only the accel term
    Au, h, br = oracle.obstacle_row(BASE, OBSTACLES[0], (0.0, 0.0, 0.3, 0.3, 0.0, 0.2, 0.0))
    assert Au[1] == 0.0 and Au[2] == 0.0
    assert br == 0.0


def test_hitch_barrier_values():
    p = BASE
    x = (0, 0, 1.0, 1.2, 2.0, 0, 0)
    np.testing.assert_allclose(oracle.hitch_h(p, x), 0.9 - 0.1 * 2.0 - 0.2, atol=1e-15)
    x = (0, 0, 1.2, 1.0, -1.0, 0, 0)
    np.testing.assert_allclose(oracle.hitch_h(p, x), 0.9 + 0.1 - 0.2, atol=1e-15)
    # hitch row: progress never enters; at v = 0, delta = 0, phi = 0 the only
    # accel effect is the speed-dependent threshold, -Ts kappa, and the
    # steer rate has no effect at second order.
    Au, h, br = oracle.hitch_row(p, (0, 0, 0.4, 0.4, 0.0, 0.0, 0))
    assert Au[2] == 0.0
    np.testing.assert_allclose(Au[0], -p["Ts"] * p["kappa"], atol=1e-15)
    np.testing.assert_allclose(Au[1], 0.0, atol=1e-15)
    np.testing.assert_allclose(br, 0.0, atol=1e-15)
