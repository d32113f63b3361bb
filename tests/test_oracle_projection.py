"""Pins of the oracle's soft-bound projection (Sec. IV-A, Eq. softproj and
its closed form Eq. closed-form_projection).

z* minimises ||z - z_des||_W^2 + rho/2 (||z - z_lo||^2 + ||z_hi - z||^2)
subject to A z = b.  Pinned by: the KKT conditions, the textbook orthogonal
projection (rho = 0, W = I) via numpy's pseudo-inverse, the unconstrained
minimiser (no rows), the one-row closed form, a brute-force grid over the
null space of A, and scipy's SLSQP on the same objective.  A numpy
restatement of the Woodbury (diagonal + rank-2) form used on the GPU is
checked against the dense closed form as well.
"""
import math

import numpy as np
import pytest
from scipy import optimize

import oracle

RNG = np.random.default_rng(1234)


def _objective(z, z_des, w, rho, lo, hi):
    return (np.sum(w * (z - z_des) ** 2)
            + 0.5 * rho * (np.sum((z - lo) ** 2) + np.sum((hi - z) ** 2)))


def _random_problem(d, nc, rng):
    A = rng.normal(size=(nc, d))
    b = rng.normal(size=nc)
    w = rng.uniform(0.5, 2.0, size=d)
    lo = -rng.uniform(0.5, 2.0, size=d)
    hi = rng.uniform(0.5, 2.0, size=d)
    z_des = rng.normal(size=d)
    rho = float(rng.uniform(0.0, 0.5))
    return A, b, w, rho, lo, hi, z_des


@pytest.mark.parametrize("d,nc", [(4, 1), (5, 2), (7, 3), (12, 9), (20, 17)])
def test_kkt(d, nc):
    for trial in range(5):
        A, b, w, rho, lo, hi, z_des = _random_problem(d, nc, RNG)
        st, z = oracle.project(A, b, w, rho, lo, hi, z_des)
        assert st == 0
        # primal feasibility
        np.testing.assert_allclose(A @ z, b, rtol=1e-12, atol=1e-12 * max(1.0, np.abs(b).max()))
        # stationarity: grad of objective = M z - p  lies in range(A^T)
        M = w + rho
        p = w * z_des + 0.5 * rho * (hi + lo)
        g = 2.0 * (M * z - p)
        lam, *_ = np.linalg.lstsq(A.T, g, rcond=None)
        np.testing.assert_allclose(A.T @ lam, g, atol=1e-10 * max(1.0, np.abs(g).max()))


def test_textbook_orthogonal_projection():
    for d, nc in [(3, 1), (6, 2), (10, 4)]:
        A, b, _, _, lo, hi, z_des = _random_problem(d, nc, RNG)
        st, z = oracle.project(A, b, np.ones(d), 0.0, lo, hi, z_des)
        ref = z_des - np.linalg.pinv(A) @ (A @ z_des - b)
        np.testing.assert_allclose(z, ref, rtol=1e-11, atol=1e-12)


def test_no_rows_is_unconstrained_minimiser():
    d = 5
    _, _, w, rho, lo, hi, z_des = _random_problem(d, 1, RNG)
    st, z = oracle.project(np.zeros((0, d)), np.zeros(0), w, rho, lo, hi, z_des)
    assert st == 0
    np.testing.assert_allclose(z, (w * z_des + 0.5 * rho * (hi + lo)) / (w + rho), rtol=1e-14)


def test_single_row_scalar_form():
    d = 4
    A, b, w, rho, lo, hi, z_des = _random_problem(d, 1, RNG)
    a = A[0]
    M = w + rho
    p = w * z_des + 0.5 * rho * (hi + lo)
    lam = (np.sum(a * p / M) - b[0]) / np.sum(a * a / M)
    st, z = oracle.project(A, b, w, rho, lo, hi, z_des)
    np.testing.assert_allclose(z, (p - lam * a) / M, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("d,nc", [(3, 1), (4, 2), (4, 1)])
def test_brute_force_grid_over_null_space(d, nc):
    rng = np.random.default_rng(d * 10 + nc)
    for trial in range(3):
        A, b, w, rho, lo, hi, z_des = _random_problem(d, nc, rng)
        st, z = oracle.project(A, b, w, rho, lo, hi, z_des)
        z_p = np.linalg.pinv(A) @ b
        _, _, Vt = np.linalg.svd(A)
        N = Vt[nc:].T  # null-space basis, d x (d - nc)
        k = N.shape[1]
        assert k <= 3
        centre = np.zeros(k)
        half = 4.0
        for level in range(8):
            axes = [np.linspace(c - half, c + half, 41) for c in centre]
            grid = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, k)
            Z = z_p[None, :] + grid @ N.T
            f = (np.sum(w * (Z - z_des) ** 2, axis=1)
                 + 0.5 * rho * (np.sum((Z - lo) ** 2, axis=1) + np.sum((hi - Z) ** 2, axis=1)))
            centre = grid[np.argmin(f)]
            half /= 8.0
        z_grid = z_p + N @ centre
        np.testing.assert_allclose(z, z_grid, atol=1e-6)


def test_scipy_slsqp_agrees():
    rng = np.random.default_rng(99)
    for d, nc in [(5, 2), (8, 4)]:
        A, b, w, rho, lo, hi, z_des = _random_problem(d, nc, rng)
        st, z = oracle.project(A, b, w, rho, lo, hi, z_des)
        res = optimize.minimize(_objective, z_des, args=(z_des, w, rho, lo, hi), method="SLSQP",
                                constraints=[{"type": "eq", "fun": lambda zz: A @ zz - b,
                                              "jac": lambda zz: A}],
                                options={"ftol": 1e-14, "maxiter": 500})
        assert res.success
        np.testing.assert_allclose(z, res.x, atol=1e-6)
        assert _objective(z, z_des, w, rho, lo, hi) <= res.fun + 1e-9


def _woodbury(A_u, h_t, b, w, rho, lo, hi, z_des):
    """Diagonal-plus-rank-2 restatement: A = [A_u | diag(h_t)], columns
    (a, omega) of A_u only; returns z*."""
    M = w + rho
    p = w * z_des + 0.5 * rho * (hi + lo)
    m_u = M[:2]
    m_a = M[3:]
    D = h_t ** 2 / m_a
    r = A_u[:, 0] * p[0] / m_u[0] + A_u[:, 1] * p[1] / m_u[1] + h_t * p[3:] / m_a - b
    S2 = np.diag(m_u) + (A_u[:, :2].T / D) @ A_u[:, :2]
    g = (A_u[:, :2].T / D) @ r
    y = np.linalg.solve(S2, g)
    lam = (r - A_u[:, :2] @ y) / D
    z = np.empty_like(z_des)
    z[:2] = p[:2] / m_u - y
    z[2] = p[2] / M[2]
    z[3:] = (p[3:] - h_t * lam) / m_a
    return z


@pytest.mark.parametrize("nc", [1, 2, 9, 65])
def test_woodbury_form_matches_dense(nc):
    rng = np.random.default_rng(nc)
    d = 3 + nc
    for trial in range(4):
        A_u = np.zeros((nc, 3))
        A_u[:, 0] = rng.normal(size=nc) * 1e-2
        A_u[0, 1] = rng.normal() * 1e-3
        h_t = rng.uniform(0.05, 3.0, size=nc) * rng.choice((-1.0, 1.0), size=nc)
        if trial == 3:
            h_t[0] = 1e-6  # floored barrier value
        A = np.zeros((nc, d))
        A[:, :3] = A_u
        A[np.arange(nc), 3 + np.arange(nc)] = h_t
        b = rng.normal(size=nc)
        w = np.ones(d)
        lo = np.r_[-2.0, -0.6, 0.0, -0.5 * np.ones(nc)]
        hi = np.r_[2.0, 0.6, 3.0, 0.5 * np.ones(nc)]
        z_des = rng.normal(size=d)
        st, z = oracle.project(A, b, w, 0.01, lo, hi, z_des)
        zw = _woodbury(A_u, h_t, b, w, 0.01, lo, hi, z_des)
        # identical algebra; the residual is the conditioning of the small
        # accel column (entries ~1e-2 against unit alpha columns)
        np.testing.assert_allclose(zw, z, rtol=1e-6, atol=1e-9)
