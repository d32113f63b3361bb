"""Pins of the oracle's tractor-trailer kinematics (Sec. III-A,
Eq. tt_discrete_kinematics) against closed forms of special cases."""
import math

import numpy as np
import pytest

import oracle
from paper_2508_05773_gb300 import scenarios as sc

P = sc.params()


def _roll(x0, U):
    return oracle.integrate(P, x0, np.asarray(U, dtype=np.float64))


def test_straight_line_constant_speed():
    # delta = 0, a = 0: the rear axle moves on a line, headings constant
    x0 = (1.0, -2.0, 0.7, 0.7, 1.3, 0.0, 0.0)
    K = 40
    traj = _roll(x0, np.zeros((K, 3)))
    k = np.arange(K + 1)
    np.testing.assert_allclose(traj[:, 0], 1.0 + k * P["Ts"] * 1.3 * math.cos(0.7), rtol=0, atol=1e-12)
    np.testing.assert_allclose(traj[:, 1], -2.0 + k * P["Ts"] * 1.3 * math.sin(0.7), rtol=0, atol=1e-12)
    assert np.all(traj[:, 2] == 0.7) and np.all(traj[:, 3] == 0.7)


def test_constant_accel_and_steer_rate_and_progress():
    x0 = (0.0, 0.0, 0.0, 0.0, -1.0, 0.05, 2.0)
    K = 25
    U = np.tile([0.4, -0.2, 1.7], (K, 1))
    traj = _roll(x0, U)
    k = np.arange(K + 1)
    np.testing.assert_allclose(traj[:, 4], -1.0 + k * P["Ts"] * 0.4, atol=1e-12)
    np.testing.assert_allclose(traj[:, 5], 0.05 - k * P["Ts"] * 0.2, atol=1e-12)
    np.testing.assert_allclose(traj[:, 6], 2.0 + k * P["Ts"] * 1.7, atol=1e-12)


def test_constant_steer_angle_dirichlet_sums():
    # a = omega = 0, delta fixed: th1 grows linearly by D = Ts v tan(delta)/l1,
    # and px, py are Dirichlet-kernel sums of cos/sin(th1_0 + j D).
    v, delta, th = -1.0, 0.2, 0.3
    x0 = (0.5, 0.25, th, th, v, delta, 0.0)
    K = 60
    traj = _roll(x0, np.zeros((K, 3)))
    D = P["Ts"] * v * math.tan(delta) / P["l1"]
    for kk in (1, 7, 33, 60):
        np.testing.assert_allclose(traj[kk, 2], th + kk * D, atol=1e-12)
        S = math.sin(kk * D / 2) / math.sin(D / 2)
        mid = th + (kk - 1) * D / 2
        np.testing.assert_allclose(traj[kk, 0], 0.5 + P["Ts"] * v * S * math.cos(mid), atol=1e-11)
        np.testing.assert_allclose(traj[kk, 1], 0.25 + P["Ts"] * v * S * math.sin(mid), atol=1e-11)


@pytest.mark.parametrize("v", [-1.0, 1.0])
def test_hitch_angle_recurrence_and_jackknife(v):
    # delta = 0: th1 is constant and phi = th1 - th2 follows
    # phi_{k+1} = phi_k - Ts (v / l2) sin(phi_k); linearised growth factor
    # 1 - Ts v / l2 (> 1 when reversing: the jackknife instability).
    phi0 = 0.3
    x0 = (0.0, 0.0, 1.0, 1.0 - phi0, v, 0.0, 0.0)
    K = 50
    traj = _roll(x0, np.zeros((K, 3)))
    phi = phi0
    for k in range(1, K + 1):
        phi = phi - P["Ts"] * (v / P["l2"]) * math.sin(phi)
        np.testing.assert_allclose(traj[k, 2] - traj[k, 3], phi, atol=1e-12)
    # small-angle growth
    eps = 1e-7
    x0 = (0.0, 0.0, 0.0, -eps, v, 0.0, 0.0)
    traj = _roll(x0, np.zeros((K, 3)))
    ratio = (traj[K, 2] - traj[K, 3]) / eps
    np.testing.assert_allclose(ratio, (1.0 - P["Ts"] * v / P["l2"]) ** K, rtol=1e-6)
    if v < 0:
        assert ratio > 1.0
    else:
        assert ratio < 1.0


def test_trailer_steering_coupling_term():
    # phi = 0, delta != 0: th2 moves only through the hitch-offset term
    # -(lh/l1) cos(phi) tan(delta) v / l2.
    v, delta = 1.0, 0.3
    x0 = (0.0, 0.0, 0.0, 0.0, v, delta, 0.0)
    xn = oracle.dynamics_step(P, x0, (0.0, 0.0, 0.0))
    np.testing.assert_allclose(xn[3], -P["Ts"] * v / P["l2"] * (P["lh"] / P["l1"]) * math.tan(delta),
                               atol=1e-15)
    np.testing.assert_allclose(xn[2], P["Ts"] * v * math.tan(delta) / P["l1"], atol=1e-15)


def test_steady_state_trailer_angle_on_circle():
    # Forward on a constant steer: the articulation converges to the steady
    # state where th1dot = th2dot, i.e. sin(phi) - k cos(phi) t = l2 t / l1.
    v, delta = 1.0, 0.15
    x0 = (0.0, 0.0, 0.0, 0.0, v, delta, 0.0)
    traj = _roll(x0, np.zeros((4000, 3)))
    phi = traj[-1, 2] - traj[-1, 3]
    t = math.tan(delta)
    k = P["lh"] / P["l1"]
    np.testing.assert_allclose(math.sin(phi) - k * math.cos(phi) * t, P["l2"] * t / P["l1"],
                               atol=1e-9)
