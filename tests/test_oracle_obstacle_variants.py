"""Pins of the oracle's obstacle variants: moving super-ellipses (predicted
pedestrians, Sec. IV-C), the collision cost of the comparison method
(standard MPPI + collision penalty, Sec. V) and the barrier-rate buffer cost
(Sec. IV-A).

Moving rows claim  L_f h + L_g h u = Ts hdot + Ts^2/2 hddot  for the barrier
of the RELATIVE position p - c(t), c(t) = c + t v.  As for the static rows,
a fine RK4 of the vehicle with the obstacle moving checks that the row misses
the true change of h by O(Ts^3).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2508_05773_gb300 import scenarios as sc
from tests import test_oracle_barriers as tb

MOVING = [
    (3.0, 1.0, 0.4, 0.4, 0.0, 2.0, -0.8, 0.3),    # pedestrian circle
    (-2.0, 2.5, 1.5, 0.6, 2.2, 4.0, 0.5, -0.4),   # super-ellipse, e = 4
    (2.0, -1.0, 0.8, 0.5, 0.7, 2.0, 1.2, 1.1),
]


def _miss_moving(p, obs, x0, u, t0):
    Au, h, br = oracle.obstacle_row_at(p, obs, x0, t0)
    x1 = tb._flow(p, x0, u, p["Ts"])
    h1 = oracle.obstacle_h_at(p, obs, x1, t0 + p["Ts"])
    return (h1 - h) - (float(np.dot(Au, u)) - br)


@pytest.mark.parametrize("obs", MOVING)
@pytest.mark.parametrize("x0", tb.STATES)
@pytest.mark.parametrize("t0", [0.0, 0.35])
def test_moving_row_is_second_order_taylor(obs, x0, t0):
    u = tb.INPUTS[0]
    m = [_miss_moving(sc.params(Ts=T), obs, x0, u, t0) for T in (0.2, 0.1, 0.05)]
    assert abs(m[1]) < 0.2 * abs(m[0]) + 1e-13
    r = m[1] / m[2]
    assert 5.5 < r < 11.0, m


def test_zero_velocity_rows_equal_static_rows():
    p = sc.params(r_inflate=0.2)
    for obs in tb.OBSTACLES:
        for x in tb.STATES:
            Au6, h6, b6 = oracle.obstacle_row(p, obs, x)
            Au8, h8, b8 = oracle.obstacle_row_at(p, tuple(obs) + (0.0, 0.0), x, 1.7)
            np.testing.assert_array_equal(Au6, Au8)
            assert h6 == h8 and b6 == b8


def test_centre_moves_with_time():
    p = sc.params()
    obs = (1.0, 2.0, 2.0, 1.0, 0.0, 2.0, 0.5, -1.0)
    for t in (0.0, 0.4, 2.0):
        c = (1.0 + 0.5 * t, 2.0 - 1.0 * t)
        assert oracle.obstacle_h_at(p, obs, (c[0], c[1], 0, 0, 0, 0, 0), t) == -1.0
        np.testing.assert_allclose(
            oracle.obstacle_h_at(p, obs, (c[0] + 2.0, c[1], 0, 0, 0, 0, 0), t), 0.0, atol=1e-14)
    # e = 4 level set: (x/a)^4 + (y/b)^4 = 1 at (a 2^-1/4, b 2^-1/4)
    obs4 = (0.0, 0.0, 2.0, 1.0, 0.0, 4.0, 0.0, 0.0)
    k = 2.0 ** -0.25
    np.testing.assert_allclose(oracle.obstacle_h_at(p, obs4, (2 * k, k, 0, 0, 0, 0, 0), 0.0), 0.0,
                               atol=1e-14)


def test_comoving_vehicle_sees_a_frozen_obstacle():
    """A vehicle driving straight at the obstacle's own velocity keeps its
    relative position: hdot = 0 and hddot = 0 at a = 0 (b_rest = 0), and
    the accel coefficient is that of a static obstacle seen from rest."""
    p = sc.params()
    th = 0.6
    v = 1.3
    obs = (2.0, 1.0, 1.2, 0.7, 0.4, 2.0, v * math.cos(th), v * math.sin(th))
    x = (0.3, -0.5, th, th, v, 0.0, 0.0)
    Au, h, br = oracle.obstacle_row_at(p, obs, x, 0.8)
    assert abs(br) < 1e-15
    x_rest = (0.3, -0.5, th, th, 0.0, 0.0, 0.0)
    frozen = (obs[0] + 0.8 * obs[6], obs[1] + 0.8 * obs[7]) + obs[2:6]
    Au_s, h_s, br_s = oracle.obstacle_row_at(p, frozen, x_rest, 0.0)
    np.testing.assert_allclose(Au, Au_s, rtol=1e-13)
    np.testing.assert_allclose(h, h_s, rtol=1e-13)
    assert br_s == 0.0


def test_collision_cost_values():
    p = sc.params(q_coll=50.0)
    obs = np.array([(0.0, 0.0, 2.0, 1.0, 0.0, 2.0), (0.5, 0.0, 1.0, 1.0, 0.0, 2.0)])
    assert oracle.collision_cost(p, obs, (10.0, 0, 0, 0, 0, 0, 0)) == 0.0
    # centre of the first (h = -1), inside the second at h = 0.25 - 1
    np.testing.assert_allclose(oracle.collision_cost(p, obs, (0.0, 0, 0, 0, 0, 0, 0)),
                               50.0 * (1.0 + 0.75), rtol=1e-15)
    # on a boundary: no charge
    assert oracle.collision_cost(p, obs[:1], (2.0, 0, 0, 0, 0, 0, 0)) == 0.0
    # moving obstacle: charged where its centre is at time t
    pm = sc.params(q_coll=50.0, flags=sc.FLAG_OBS8)
    om = np.array([(0.0, 0.0, 2.0, 1.0, 0.0, 2.0, 1.0, 0.0)])
    assert oracle.collision_cost(pm, om, (3.0, 0, 0, 0, 0, 0, 0), 3.0) == 50.0
    assert oracle.collision_cost(pm, om, (3.0, 0, 0, 0, 0, 0, 0), 0.0) == 0.0


def test_alpha_buffer_cost_values():
    p = sc.params(q_abuf=4.0, h_buf=0.5)
    # weight 1 at h <= 0, 1/2 at h_buf/2, 0 from h_buf on; only positive rates
    h = np.array([-0.3, 0.0, 0.25, 0.5, 2.0, 0.1, 0.4])
    a = np.array([0.5, 0.5, 0.5, 0.5, 0.5, -0.7, 0.3])
    want = 4.0 * (0.25 + 0.25 + 0.5 * 0.25 + 0.0 + 0.0 + 0.0 + 0.2 * 0.09)
    np.testing.assert_allclose(oracle.alpha_buffer_cost(p, h, a), want, rtol=1e-15)


def _case(flags, seed=3, **kw):
    c = sc.small_random(seed, S=8, H=10, n_obs=3)
    p = sc.as_float32(sc.params(S=8, H=10, flags=flags, **kw))
    return c, p


def test_collision_cost_enters_after_each_step():
    """J(MPPI + collision) - J(MPPI) = sum over steps of the penalty at the
    state after the step, at that step's time."""
    flags = sc.FLAG_PROJ_NONE | sc.FLAG_OBS8
    c, p0 = _case(flags)
    obs8 = np.hstack([c["obs"], np.tile([[0.4, -0.2]], (len(c["obs"]), 1))])
    # obstacles moved onto the path so that rollouts hit them
    obs8[:, 0:2] = c["path"][[5, 8, 12], 0:2]
    p1 = dict(p0, flags=flags | sc.FLAG_COLLISION_COST)
    r0 = oracle.solve(p0, c["x0"], c["U_nom"], obs8, c["path"], c["ds"], c["seed"], 0,
                      want_states=True)
    r1 = oracle.solve(p1, c["x0"], c["U_nom"], obs8, c["path"], c["ds"], c["seed"], 0)
    extra = np.array([sum(oracle.collision_cost(p1, obs8, r0["states"][s, k + 1], (k + 1) * p1["Ts"])
                          for k in range(p1["H"])) for s in range(p1["S"])])
    assert extra.max() > 0.0, "case must penetrate an obstacle"
    np.testing.assert_allclose(r1["J"] - r0["J"], extra, rtol=1e-12, atol=1e-9)


def test_alpha_buffer_cost_enters_with_updated_rates():
    """J(buffer) - J(plain) = sum over steps of the buffer cost of the rows'
    h at the step's state and the rates alpha_tau the rows were built with."""
    c, p0 = _case(0, seed=5)
    p1 = dict(p0, flags=sc.FLAG_ALPHA_BUFFER, h_buf=1e3)
    n = len(c["obs"])
    extra = []
    for s in range(p0["S"]):
        r0 = oracle.rollout_sample(p0, c["x0"], c["U_nom"], c["obs"], c["path"], c["ds"],
                                   c["seed"], 0, s)
        r1 = oracle.rollout_sample(p1, c["x0"], c["U_nom"], c["obs"], c["path"], c["ds"],
                                   c["seed"], 0, s)
        # the buffer cost changes no input, state or rate: only J
        np.testing.assert_array_equal(r0["states"], r1["states"])
        e = 0.0
        for k in range(p0["H"]):
            h = [oracle.obstacle_h(p1, c["obs"][o], r0["states"][k]) for o in range(n)]
            e += oracle.alpha_buffer_cost(p1, h, r0["alpha"][k, 1:])
        extra.append(r1["J"] - r0["J"])
        np.testing.assert_allclose(r1["J"] - r0["J"], e, rtol=1e-12, atol=1e-12)
    assert max(extra) > 0.0


def test_moving_rows_used_at_step_time():
    """With moving obstacles the rollout's rows are those of the obstacle
    at time tau Ts: the projected input satisfies them."""
    flags = sc.FLAG_OBS8
    c, p = _case(flags, seed=9)
    obs8 = np.hstack([c["obs"], np.tile([[0.6, 0.3]], (len(c["obs"]), 1))])
    r = oracle.rollout_sample(p, c["x0"], c["U_nom"], obs8, c["path"], c["ds"], c["seed"], 0, 2)
    assert r["status"] == 0
    for k in range(p["H"]):
        x = r["states"][k]
        zs = r["z_star"][k]
        for o in range(len(obs8)):
            Au, h, br = oracle.obstacle_row_at(p, obs8[o], x, k * p["Ts"])
            ht = math.copysign(max(abs(h), p["h_floor"]), h if h != 0 else 1.0)
            lhs = float(np.dot(Au, zs[:3])) + ht * zs[4 + o]
            rhs = -r["alpha"][k, 1 + o] * h + br
            np.testing.assert_allclose(lhs, rhs, rtol=1e-9, atol=1e-9)
