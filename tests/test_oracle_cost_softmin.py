"""Pins of the oracle's path lookup, contouring cost (Sec. IV-B,
Eq. cost_function_contour / contour_lag_errors) and MPPI weights
(Sec. II-B)."""
import math

import numpy as np
import pytest

import oracle
from paper_2508_05773_gb300 import scenarios as sc

ZERO_R = sc.params(R=(0.0, 0.0, 0.0))


def _straight(theta, n=101, ds=0.1):
    s = np.arange(n) * ds
    return np.stack([s * math.cos(theta), s * math.sin(theta), np.full(n, theta)], axis=1)


def test_path_lookup_interpolation_and_clamp():
    path = np.array([[0.0, 0.0, 0.0], [1.0, 2.0, 0.5], [3.0, 2.0, 1.5]])
    ds = 0.5
    assert oracle.path_lookup(path, ds, 0.0) == (0.0, 0.0, 0.0)
    np.testing.assert_allclose(oracle.path_lookup(path, ds, 0.25), (0.5, 1.0, 0.25))
    np.testing.assert_allclose(oracle.path_lookup(path, ds, 0.5), (1.0, 2.0, 0.5))
    np.testing.assert_allclose(oracle.path_lookup(path, ds, 0.875), (2.5, 2.0, 1.25))
    np.testing.assert_allclose(oracle.path_lookup(path, ds, 7.0), (3.0, 2.0, 1.5))   # clamped
    np.testing.assert_allclose(oracle.path_lookup(path, ds, -1.0), (0.0, 0.0, 0.0))  # clamped


@pytest.mark.parametrize("theta", [0.0, 0.8, math.pi, -2.0])
def test_cost_on_path_is_zero_and_offsets_are_quadratic(theta):
    path = _straight(theta)
    psi = 3.0
    base = np.array([psi * math.cos(theta), psi * math.sin(theta), theta, theta, 1.0, 0.0, psi])
    u = (0.0, 0.0, 3.0)  # nu = nu_bar
    assert abs(oracle.stage_cost(ZERO_R, base, u, path, 0.1)) < 1e-20
    d = 0.37
    # lateral offset (left normal) -> contouring error only
    x = base.copy()
    x[0] -= d * math.sin(theta)
    x[1] += d * math.cos(theta)
    np.testing.assert_allclose(oracle.stage_cost(ZERO_R, x, u, path, 0.1), 10.0 * d * d, rtol=1e-12)
    # longitudinal offset -> lag error only
    x = base.copy()
    x[0] += d * math.cos(theta)
    x[1] += d * math.sin(theta)
    np.testing.assert_allclose(oracle.stage_cost(ZERO_R, x, u, path, 0.1), 10.0 * d * d, rtol=1e-12)
    # heading offsets of tractor and trailer
    x = base.copy()
    x[2] += 0.2
    x[3] -= 0.1
    np.testing.assert_allclose(oracle.stage_cost(ZERO_R, x, u, path, 0.1), 5.0 * (0.04 + 0.01),
                               rtol=1e-12)
    # heading errors are wrapped: a full turn costs nothing
    x = base.copy()
    x[2] += 2 * math.pi
    x[3] -= 4 * math.pi
    assert abs(oracle.stage_cost(ZERO_R, x, u, path, 0.1)) < 1e-20


def test_cost_effort_and_progress_terms():
    p = sc.params()
    path = _straight(0.0)
    x = np.array([1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 1.0])
    u = (0.5, -0.3, 1.2)
    want = 0.1 * 0.25 + 0.1 * 0.09 + 0.01 * 1.44 + 1.0 * (3.0 - 1.2) ** 2
    np.testing.assert_allclose(oracle.stage_cost(p, x, u, path, 0.1), want, rtol=1e-14)


def test_softmin_basic_properties():
    rng = np.random.default_rng(5)
    J = rng.uniform(100, 130, size=300)
    st, g = oracle.softmin(J, 1.0)
    assert st == 0
    assert np.all(g >= 0)
    np.testing.assert_allclose(g.sum(), 1.0, atol=1e-12)
    # invariant to a common shift
    st, g2 = oracle.softmin(J + 1e4, 1.0)
    np.testing.assert_allclose(g2, g, rtol=1e-9, atol=1e-300)


def test_softmin_closed_forms():
    st, g = oracle.softmin(np.full(17, 3.0), 0.7)
    np.testing.assert_allclose(g, np.full(17, 1 / 17), rtol=1e-15)
    lam = 0.8
    st, g = oracle.softmin(np.array([5.0, 5.0 + lam * math.log(2.0)]), lam)
    np.testing.assert_allclose(g, [2 / 3, 1 / 3], rtol=1e-14)
    J = np.array([4.0, 1.0, 3.0, 2.0])
    st, g = oracle.softmin(J, 1e-3)
    np.testing.assert_allclose(g, [0, 1, 0, 0], atol=1e-300)
    st, g = oracle.softmin(J, 1e9)
    np.testing.assert_allclose(g, np.full(4, 0.25), rtol=1e-8)


def test_softmin_nonfinite():
    st, g = oracle.softmin(np.array([1.0, np.inf, np.nan, 2.0]), 1.0)
    assert st == 0
    np.testing.assert_allclose(g, [1 / (1 + math.exp(-1)), 0, 0, math.exp(-1) / (1 + math.exp(-1))])
    st, g = oracle.softmin(np.array([np.inf, np.nan]), 1.0)
    assert st == oracle.ORC_ENONFINITE
