"""Closed-loop harness: the simulated vehicle of a receding-horizon run.

The plant is the tractor-trailer kinematics (Sec. III-A,
Eq. tt_discrete_kinematics, acceleration input, progress psi driven by nu)
integrated in FP64 on the host, advanced by the first input of each solve;
the nominal sequence is warm-started by a one-step shift with the last
input repeated (Sec. II-B, receding horizon).  It is the environment around
the solver, not part of the solve.
"""
from __future__ import annotations

import math

import numpy as np


def step(p: dict, x, u) -> np.ndarray:
    px, py, th1, th2, v, dl, psi = np.asarray(x, dtype=np.float64).tolist()
    a, om, nu = np.asarray(u, dtype=np.float64).tolist()[:3]
    Ts, l1, l2 = float(p["Ts"]), float(p["l1"]), float(p["l2"])
    t = math.tan(dl)
    k = float(p["lh"]) / l1
    phi = th1 - th2
    Tv = Ts * v
    return np.array([
        px + Tv * math.cos(th1),
        py + Tv * math.sin(th1),
        th1 + Tv * t / l1,
        th2 + Tv / l2 * (math.sin(phi) - k * math.cos(phi) * t),
        v + Ts * a,
        dl + Ts * om,
        psi + Ts * nu,
    ], dtype=np.float64)


def shift(U) -> np.ndarray:
    U = np.asarray(U)
    out = np.empty_like(U)
    out[:-1] = U[1:]
    out[-1] = U[-1]
    return out
