"""Pins of the oracle's third-order obstacle rows (the expansion of
Eq. barrier_function_approx carried to Ts^3, which brings the steer rate
into obstacle rows).

A fine RK4 of the vehicle (and of a moving obstacle) checks that the row
misses the true change of h by O(Ts^4): halving Ts divides the miss by ~16
(a dropped or mis-weighted third-order term leaves O(Ts^3), ratio ~8).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2508_05773_gb300 import scenarios as sc
from tests import test_oracle_barriers as tb

OBS = [(3.0, 1.0, 1.0, 0.6, 0.3, 2.0, 0.0, 0.0),
       (-2.0, 2.5, 1.5, 0.6, 2.2, 4.0, 0.5, -0.4),
       (2.0, -1.0, 0.8, 0.5, 0.7, 4.0, 1.2, 1.1)]
STATES = [tb.STATES[0], (0.0, 0.0, math.pi, math.pi - 0.3, -1.0, -0.3, 0.0),
          (0.5, -0.5, 1.0, 0.8, 2.5, 0.4, 0.0)]


def _miss3(p, obs, x0, u, t0):
    Au, h, br = oracle.obstacle_row3(p, obs, x0, t0)
    h1 = oracle.obstacle_h_at(p, obs, tb._flow(p, x0, u, p["Ts"]), t0 + p["Ts"])
    return (h1 - h) - (float(np.dot(Au, u)) - br)


@pytest.mark.parametrize("obs", OBS)
@pytest.mark.parametrize("x0", STATES)
def test_third_order_row_misses_by_ts4(obs, x0):
    u = (0.8, -0.5, 1.0)
    ms = [_miss3(sc.params(Ts=T), obs, x0, u, 0.3) for T in (0.08, 0.04, 0.02)]
    assert abs(ms[0]) / abs(ms[1]) > 11.0 and abs(ms[1]) / abs(ms[2]) > 11.0, ms


@pytest.mark.parametrize("obs", OBS)
def test_third_order_extends_the_second_order_row(obs):
    """row3 - row2 is the Ts^3 / 6 term: it scales as Ts^3."""
    x = STATES[2]
    d = []
    for T in (0.1, 0.05):
        p = sc.params(Ts=T)
        A3, h3, b3 = oracle.obstacle_row3(p, obs, x, 0.2)
        A2, h2, b2 = oracle.obstacle_row_at(p, obs, x, 0.2)
        np.testing.assert_allclose(h3, h2, rtol=1e-14)
        d.append(np.concatenate([A3 - A2, [b3 - b2]]))
    r = np.abs(d[0]) / np.maximum(np.abs(d[1]), 1e-300)
    big = np.abs(d[0]) > 1e-12
    np.testing.assert_allclose(r[big], 8.0, rtol=1e-9)


def test_steer_rate_enters_at_third_order():
    p = sc.params()
    obs = OBS[0]
    A, _, _ = oracle.obstacle_row3(p, obs, STATES[2])
    assert abs(A[1]) > 1e-9 and A[2] == 0.0
    # omega enters through v th1ddot: none at standstill
    A0, _, _ = oracle.obstacle_row3(p, obs, (0.5, -0.5, 1.0, 0.8, 0.0, 0.4, 0.0))
    assert A0[1] == 0.0


def test_rollout_uses_third_order_rows():
    c = sc.small_random(21, S=4, H=8, n_obs=3)
    p = sc.as_float32(sc.params(S=4, H=8, flags=sc.FLAG_THIRD_ORDER))
    r = oracle.rollout_sample(p, c["x0"], c["U_nom"], c["obs"], c["path"], c["ds"], c["seed"], 0, 1)
    assert r["status"] == 0
    for k in range(p["H"]):
        x, zs = r["states"][k], r["z_star"][k]
        for o in range(3):
            Au, h, br = oracle.obstacle_row3(p, c["obs"][o], x, k * p["Ts"])
            ht = math.copysign(max(abs(h), p["h_floor"]), h if h != 0 else 1.0)
            lhs = float(np.dot(Au, zs[:3])) + ht * zs[4 + o]
            np.testing.assert_allclose(lhs, -r["alpha"][k, 1 + o] * h + br, rtol=1e-9, atol=1e-9)


def test_third_order_refuses_offset_discs():
    c = sc.small_random(21, S=4, H=8, n_obs=2)
    p = sc.as_float32(sc.params(S=4, H=8, flags=sc.FLAG_THIRD_ORDER, **sc.FIVE_DISCS))
    r = oracle.rollout_sample(p, c["x0"], c["U_nom"], c["obs"], c["path"], c["ds"], c["seed"], 0, 0)
    assert r["status"] == -1  # ORC_EINVAL
