"""Pins of the oracle's footprint discs (Sec. IV-C: the tractor-trailer body
covered by discs whose radius inflates the obstacles).

Disc positions are pinned to the kinematics they ride on: the tractor's rear
axle and the trailer's axle move without lateral slip (the non-holonomic
constraints the trailer-angle equation of Sec. III-A encodes), and the hitch
point is the same point seen from either body.  Disc rows are pinned like
the single-point rows: a fine RK4 of the vehicle checks that the row misses
the true change of h at the disc by O(Ts^3), now with the steer rate in the
input (offset discs feel it through the heading accelerations).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2508_05773_gb300 import scenarios as sc
from tests import test_oracle_barriers as tb


def _p(**kw):
    return sc.params(**dict(sc.FIVE_DISCS, **kw))


def _flow_path(p, x0, u, T, n):
    """States along the exact flow at n+1 equally spaced times."""
    xs = [np.array(x0, np.float64)]
    for _ in range(n):
        xs.append(tb._flow(p, xs[-1], u, T / n, n=20))
    return xs


@pytest.mark.parametrize("x0", [(0.0, 0.0, 0.3, 0.1, 1.2, 0.2, 0.0),
                                (1.0, -2.0, 3.0, 2.6, -1.0, -0.35, 0.0)])
def test_axles_do_not_slip(x0):
    p = _p()
    u = (0.4, 0.3, 1.0)
    T, n = 0.002, 2
    xs = _flow_path(p, x0, u, T, n)
    for m, on_trailer in ((0, False), (3, True)):  # tractor rear axle, trailer axle
        pos = [oracle.disc_position(p, m, x) for x in xs]
        vel = (pos[2] - pos[0]) / T  # central difference at the middle state
        th = xs[1][3] if on_trailer else xs[1][2]
        lateral = -math.sin(th) * vel[0] + math.cos(th) * vel[1]
        assert abs(lateral) < 1e-7 * max(1.0, float(np.linalg.norm(vel))), (m, lateral)
        along = math.cos(th) * vel[0] + math.sin(th) * vel[1]
        assert abs(along) > 0.1


def test_hitch_point_seen_from_both_bodies():
    p = sc.params(n_discs=2, disc_trailer_mask=0b10,
                  disc_off=(-0.5, 8.0, 0, 0, 0, 0, 0, 0))  # -lh on the tractor, l2 on the trailer
    for x in [(0.0, 0.0, 0.3, 1.0, 1.0, 0.2, 0.0), (3.0, 1.0, -2.0, -1.1, -1.0, 0.0, 0.0)]:
        np.testing.assert_allclose(oracle.disc_position(p, 0, x), oracle.disc_position(p, 1, x),
                                   atol=1e-13)
    # the default single disc is the tractor's rear axle
    x = (1.5, -0.5, 0.7, 0.2, 1.0, 0.1, 0.0)
    np.testing.assert_array_equal(oracle.disc_position(sc.params(), 0, x), [1.5, -0.5])


def _miss(p, obs, m, x0, u, t0=0.0):
    Au, h, br = oracle.disc_row(p, obs, m, x0, t0)
    h1 = oracle.disc_h(p, obs, m, tb._flow(p, x0, u, p["Ts"]), t0 + p["Ts"])
    return (h1 - h) - (float(np.dot(Au, u)) - br)


OBS = [(3.0, 1.0, 1.0, 0.6, 0.3, 2.0, 0.0, 0.0),
       (-2.0, 2.5, 1.5, 0.6, 2.2, 4.0, 0.5, -0.4),
       (-6.0, -1.0, 0.5, 0.5, 0.0, 2.0, 1.0, 0.8)]


# fast articulation (3 m/s, hitch angle 0.8 rad): the trailer's heading
# rate, and with it its discs' centripetal terms, are large
FAST_FOLD = (0.0, 0.0, 0.5, -0.3, 3.0, 0.1, 0.0)


@pytest.mark.parametrize("m", range(5))
@pytest.mark.parametrize("obs", OBS)
@pytest.mark.parametrize("x0", [tb.STATES[0], (0.0, 0.0, math.pi, math.pi - 0.3, -1.0, -0.3, 0.0),
                                FAST_FOLD])
def test_disc_row_is_second_order_taylor(m, obs, x0):
    u = (0.8, -0.5, 1.0)  # steer rate on: offset discs feel it at second order
    ms = [_miss(_p(Ts=T), obs, m, x0, u, 0.2) for T in (0.04, 0.02, 0.01)]
    # the miss is O(Ts^3) (ratio ~8 per halving; higher where its
    # third-order term happens to vanish); a wrong term leaves O(Ts^2) (~4)
    assert abs(ms[0]) / abs(ms[1]) > 5.5 and abs(ms[1]) / abs(ms[2]) > 5.5, ms


def test_single_rear_axle_disc_is_the_point_row():
    p = sc.params(r_inflate=0.3)
    for obs in tb.OBSTACLES:
        for x in tb.STATES:
            Au, h, br = oracle.obstacle_row_at(p, obs, x, 0.0)
            Ad, hd, bd = oracle.disc_row(p, obs, 0, x, 0.0)
            np.testing.assert_allclose(Ad, Au, rtol=1e-13, atol=1e-16)
            np.testing.assert_allclose(hd, h, rtol=1e-13, atol=1e-15)
            np.testing.assert_allclose(bd, br, rtol=1e-12, atol=1e-15)


def test_steer_rate_enters_offset_discs_only():
    p = _p()
    x = (0.0, 0.0, 0.3, 0.1, 1.2, 0.2, 0.0)
    obs = OBS[0]
    assert oracle.disc_row(p, obs, 0, x)[0][1] == 0.0       # rear axle
    assert abs(oracle.disc_row(p, obs, 2, x)[0][1]) > 1e-6  # tractor front
    assert abs(oracle.disc_row(p, obs, 3, x)[0][1]) > 1e-6  # trailer axle
    for m in range(5):
        assert oracle.disc_row(p, obs, m, x)[0][2] == 0.0   # progress never


def test_rollout_rows_cover_every_obstacle_and_disc():
    c = sc.small_random(13, S=4, H=8, n_obs=3)
    p = sc.as_float32(_p(S=4, H=8))
    r = oracle.rollout_sample(p, c["x0"], c["U_nom"], c["obs"], c["path"], c["ds"], c["seed"], 0, 1)
    assert r["status"] == 0
    nd = p["n_discs"]
    assert r["alpha"].shape == (9, 1 + 3 * nd)
    for k in range(p["H"]):
        x, zs = r["states"][k], r["z_star"][k]
        for o in range(3):
            for m in range(nd):
                i = 1 + o * nd + m
                Au, h, br = oracle.disc_row(p, c["obs"][o], m, x, k * p["Ts"])
                ht = math.copysign(max(abs(h), p["h_floor"]), h if h != 0 else 1.0)
                lhs = float(np.dot(Au, zs[:3])) + ht * zs[3 + i]
                np.testing.assert_allclose(lhs, -r["alpha"][k, i] * h + br, rtol=1e-9, atol=1e-9)


def test_collision_cost_counts_every_disc():
    p = _p(q_coll=10.0)
    x = (0.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0)  # straight along +x
    # a circle around the tractor's mid disc (x = 2) only
    obs = np.array([(2.0, 0.0, 0.5, 0.5, 0.0, 2.0)])
    np.testing.assert_allclose(oracle.collision_cost(p, obs, x), 10.0, rtol=1e-15)
    # a long ellipse over the whole tractor: three discs inside
    obs = np.array([(2.0, 0.0, 3.0, 0.5, 0.0, 2.0)])
    want = 10.0 * sum(1.0 - (d - 2.0) ** 2 / 9.0 for d in (0.0, 2.0, 4.0))
    np.testing.assert_allclose(oracle.collision_cost(p, obs, x), want, rtol=1e-14)
