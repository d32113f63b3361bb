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
    px, py, th1, th2, v, dl, psi = (float(a) for a in x)
    a, om, nu = (float(b) for b in u)
    Ts = float(p["Ts"])
    t = math.tan(dl)
    k = float(p["lh"]) / float(p["l1"])
    return np.array([
        px + Ts * v * math.cos(th1),
        py + Ts * v * math.sin(th1),
        th1 + Ts * v * t / float(p["l1"]),
        th2 + Ts * v / float(p["l2"]) * (math.sin(th1 - th2) - k * math.cos(th1 - th2) * t),
        v + Ts * a,
        dl + Ts * om,
        psi + Ts * nu,
    ], dtype=np.float64)


def shift(U) -> np.ndarray:
    U = np.asarray(U)
    return np.concatenate([U[1:], U[-1:]], axis=0)
