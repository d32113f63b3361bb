"""Tolerances of the GPU-vs-oracle comparison (FP32 CUDA path against the
FP64 oracle), 1e-4 relative as the solve's accuracy target:

* states and trajectories: |g - o| / max(|o|, 1)            <= 1e-4
* U*: |g - o| / max(|o|, 0.01 (z_hi - z_lo))                <= 1e-4
* per-sample costs J (diagnostic): |g - o| / |o|            <= 1e-5
"""
import numpy as np

TOL_STATE = 1e-4
TOL_U = 1e-4
TOL_J = 1e-5


def err_state(g, o):
    g = np.asarray(g, np.float64)
    o = np.asarray(o, np.float64)
    return float(np.max(np.abs(g - o) / np.maximum(np.abs(o), 1.0))) if o.size else 0.0


def err_u(g, o, p):
    span = np.asarray(p["z_hi"], np.float64) - np.asarray(p["z_lo"], np.float64)
    g = np.asarray(g, np.float64).reshape(-1, 3)
    o = np.asarray(o, np.float64).reshape(-1, 3)
    return float(np.max(np.abs(g - o) / np.maximum(np.abs(o), 0.01 * span)))


def err_j(g, o):
    g = np.asarray(g, np.float64)
    o = np.asarray(o, np.float64)
    return float(np.max(np.abs(g - o) / np.abs(o)))


def assert_solve_matches(out, ref, p, label="", check_J=True):
    eu = err_u(out["U"], ref["U"], p)
    ex = err_state(out["traj"], ref["traj"]) if out.get("traj") is not None else 0.0
    ej = err_j(out["J"], ref["J"]) if (check_J and out.get("J") is not None) else 0.0
    assert eu <= TOL_U, f"{label} U* rel err {eu:.3e}"
    assert ex <= TOL_STATE, f"{label} trajectory rel err {ex:.3e}"
    assert ej <= TOL_J, f"{label} J rel err {ej:.3e}"
    return eu, ex, ej
