"""Pins of the oracle's hitch-angle stabilizer (Sec. IV-D, Eq. hitch_angle_qp).

The stabilizer is a QP in (a, omega): the input nearest the BR-MPPI reference
in the Q_h norm, inside the input box, whose hitch barrier increment meets
the discrete CBF condition  g . u + c0 >= -alpha_stab h  (the rollout's
second-order hitch row; sign of Eq. cbf_equality).  The oracle solves it by
bisection on the KKT multiplier.  These tests pin it to things other than
that method: the closed form when no bound is active, a brute-force grid
over the box, scipy's SLSQP, the corner that maximises the increment when
nothing is feasible, and the closed-loop property the condition exists for
(the hitch angle stays inside its velocity-dependent limit).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2508_05773_gb300 import scenarios as sc
from tests import test_oracle_barriers as tb


def _row(p, x):
    Au, h, br = oracle.hitch_row(p, x)
    g = np.array(Au[:2])
    rhs = -p["alpha_stab"] * h + br  # need g . u >= rhs
    return g, rhs, h


def _cost(p, u, u_ref):
    q = np.array(p["q_stab"])
    d = np.asarray(u[:2]) - np.asarray(u_ref[:2])
    return float(np.sum(q * d * d))


def _active_cases(p, n, seed, feasible=True):
    """Random reversing states a few hundredths of a radian inside the
    hitch limit with the trailer folding, and references whose box
    projection breaks the condition (feasible: some input in the box meets
    it)."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        v = float(rng.uniform(-2.0, -0.3))
        sgn = 1.0 if rng.random() < 0.5 else -1.0
        th1 = float(rng.uniform(-math.pi, math.pi))
        lim = p["dtheta_max"] - p["kappa"] * v
        Delta = sgn * (lim - float(rng.uniform(0.0, 0.03)))
        delta = sgn * float(rng.uniform(0.0, 0.5))
        x = (0.0, 0.0, th1, th1 + Delta, v, delta, 0.0)
        u_ref = (float(rng.uniform(-2.5, 2.5)), float(rng.uniform(-0.8, 0.8)), 1.0)
        g, rhs, _ = _row(p, x)
        uc = np.clip(u_ref[:2], p["z_lo"][:2], p["z_hi"][:2])
        if g @ uc >= rhs:
            continue
        corners = [g @ np.array((a, w)) for a in (p["z_lo"][0], p["z_hi"][0])
                   for w in (p["z_lo"][1], p["z_hi"][1])]
        if (max(corners) >= rhs) == feasible:
            out.append((x, u_ref))
    return out


def test_admissible_reference_is_unchanged():
    p = sc.params()
    x = (0.0, 0.0, 0.3, 0.3, -1.0, 0.0, 0.0)  # straight, far from the limit
    u_ref = (0.4, -0.1, 2.2)
    st, u, slack = oracle.hitch_stabilize(p, x, u_ref)
    assert st == 0 and slack >= 0.0
    np.testing.assert_array_equal(u, u_ref)
    # outside the box: only the box projection (constraint inactive)
    st, u, slack = oracle.hitch_stabilize(p, x, (5.0, -3.0, 1.0))
    assert st == 0
    np.testing.assert_array_equal(u, (2.0, -0.6, 1.0))


@pytest.mark.parametrize("seed", range(4))
def test_closed_form_without_active_bounds(seed):
    p = sc.params(z_lo=(-1e3, -1e3, 0.0), z_hi=(1e3, 1e3, 3.0), q_stab=(2.0, 0.5))
    for x, u_ref in _active_cases(p, 3, seed):
        g, rhs, h = _row(p, x)
        u0 = np.array(u_ref[:2])
        qi = 1.0 / np.array(p["q_stab"])
        mu = (rhs - g @ u0) / (g @ (qi * g))
        want = u0 + mu * qi * g
        st, u, slack = oracle.hitch_stabilize(p, x, (u0[0], u0[1], 0.7))
        assert st == 0
        np.testing.assert_allclose(u[:2], want, rtol=1e-12, atol=1e-12)
        assert u[2] == 0.7
        assert abs(slack) < 1e-12


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_grid(seed):
    rng = np.random.default_rng(seed)
    p = sc.params(q_stab=tuple(rng.uniform(0.2, 3.0, 2)), alpha_stab=float(rng.uniform(0.1, 1.0)))
    A = np.linspace(p["z_lo"][0], p["z_hi"][0], 801)
    W = np.linspace(p["z_lo"][1], p["z_hi"][1], 801)
    aa, ww = np.meshgrid(A, W, indexing="ij")
    q = p["q_stab"]
    for x, u_ref in _active_cases(p, 2, 50 + seed):
        g, rhs, _ = _row(p, x)
        st, u, slack = oracle.hitch_stabilize(p, x, u_ref)
        feas = g[0] * aa + g[1] * ww >= rhs
        assert st == 0 and slack >= -1e-12
        assert u[0] >= p["z_lo"][0] and u[0] <= p["z_hi"][0]
        assert u[1] >= p["z_lo"][1] and u[1] <= p["z_hi"][1]
        if not feas.any():
            continue  # feasible set thinner than the grid
        c = q[0] * (aa - u_ref[0]) ** 2 + q[1] * (ww - u_ref[1]) ** 2
        best = c[feas].min()
        mine = _cost(p, u, u_ref)
        assert mine <= best + 1e-9
        # the grid's best feasible point lies within one cell of the
        # optimum: its cost exceeds the optimum's by at most
        # |grad c| * cell + max(q) * cell^2
        cell = math.hypot(A[1] - A[0], W[1] - W[0])
        grad = 2.0 * max(q) * float(np.linalg.norm(np.asarray(u[:2]) - np.asarray(u_ref[:2])))
        assert best - mine <= grad * cell + max(q) * cell * cell + 1e-12


@pytest.mark.parametrize("seed", range(4))
def test_scipy_slsqp_agrees(seed):
    opt = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(100 + seed)
    p = sc.params(q_stab=tuple(rng.uniform(0.2, 3.0, 2)))
    q = np.array(p["q_stab"])
    for x, u_ref in _active_cases(p, 2, 200 + seed):
        u0 = np.array(u_ref[:2])
        g, rhs, _ = _row(p, x)
        res = opt.minimize(lambda u: float(np.sum(q * (u - u0) ** 2)),
                           x0=np.clip(u0, p["z_lo"][:2], p["z_hi"][:2]),
                           jac=lambda u: 2 * q * (u - u0), method="SLSQP",
                           bounds=list(zip(p["z_lo"][:2], p["z_hi"][:2])),
                           constraints=[dict(type="ineq", fun=lambda u: g @ u - rhs,
                                             jac=lambda u: g)],
                           options=dict(ftol=1e-15, maxiter=500))
        st, u, _ = oracle.hitch_stabilize(p, x, u_ref)
        assert res.success and st == 0
        np.testing.assert_allclose(u[:2], res.x, atol=1e-6)


def test_infeasible_returns_increment_maximiser():
    p = sc.params()
    for x, u_ref in _active_cases(p, 4, 7, feasible=False):
        g, rhs, h = _row(p, x)
        corners = [(a, w) for a in (p["z_lo"][0], p["z_hi"][0]) for w in (p["z_lo"][1], p["z_hi"][1])]
        best = max(corners, key=lambda c: g @ np.array(c))
        st, u, slack = oracle.hitch_stabilize(p, x, u_ref)
        assert st == 1
        np.testing.assert_array_equal(u[:2], best)
        np.testing.assert_allclose(slack, g @ np.array(best) - rhs, rtol=1e-12)
        assert slack < 0


@pytest.mark.parametrize("alpha", [0.3, 0.5, 1.0])
def test_keeps_hitch_inside_its_limit_in_closed_loop(alpha):
    """Reversing at -1 m/s while a steering loop holds delta = 0.4 folds
    the trailer (the jackknife the stabilizer exists for).  With the
    stabilizer between that reference and the plant (exact flow, input held
    for Ts), every step where the condition is feasible has
    h_{k+1} >= (1 - alpha) h_k up to the O(Ts^3) Taylor error, so the
    barrier stays non-negative while the stabilizer has the authority."""
    p = sc.params(Ts=0.05, alpha_stab=alpha)

    def u_ref(x):
        return (float(np.clip(2.0 * (-1.0 - x[4]), -2, 2)),
                float(np.clip(3.0 * (0.4 - x[5]), -0.6, 0.6)), 0.0)

    x = np.array([0.0, 0.0, 0.0, 0.0, -1.0, 0.0, 0.0])
    free = x.copy()
    steps = 0
    for _ in range(300):
        st, u, _ = oracle.hitch_stabilize(p, x, u_ref(x))
        if st:
            break
        h0 = oracle.hitch_h(p, x)
        x = tb._flow(p, x, u, p["Ts"], n=10)
        h1 = oracle.hitch_h(p, x)
        assert h1 >= (1.0 - alpha) * h0 - 1e-4
        assert h1 > -1e-4
        free = tb._flow(p, free, u_ref(free), p["Ts"], n=10)
        steps += 1
    assert steps >= 100
    assert oracle.hitch_h(p, free) < 0.0, "the unstabilised reference must jackknife"
