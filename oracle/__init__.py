"""FP64 CPU oracle for one BR-MPPI solve (ctypes binding of ``brmppi_oracle.c``).

TEST INFRASTRUCTURE ONLY: the slow, plain restatement of the method that the
CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it; the product package
never does.  It shares no code with the CUDA library; both receive the same
inputs from the seeded generators.

Parameters are passed as a plain dict with the field names of the C struct
``orc_params``.  Floating inputs are taken as given (callers that compare
with the FP32 CUDA path round them to binary32 first, so that both sides see
identical numbers).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "brmppi_oracle.c")
_HDR = os.path.join(_HERE, "brmppi_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")

ORC_OK = 0
ORC_EINVAL = -1
ORC_ENONFINITE = -5
ORC_PROJ_NONE = 1

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (plain C11, libm)."""
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(p) > os.path.getmtime(_LIB) for p in (_SRC, _HDR))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c11", "-D_DEFAULT_SOURCE", "-O2", "-fPIC", "-shared",
               "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("S", ctypes.c_int32), ("H", ctypes.c_int32), ("flags", ctypes.c_int32),
        ("Ts", ctypes.c_double), ("lambda_", ctypes.c_double),
        ("l1", ctypes.c_double), ("lh", ctypes.c_double), ("l2", ctypes.c_double),
        ("dtheta_max", ctypes.c_double), ("kappa", ctypes.c_double),
        ("r_inflate", ctypes.c_double),
        ("Qc", ctypes.c_double), ("Ql", ctypes.c_double), ("Qth", ctypes.c_double),
        ("R", ctypes.c_double * 3), ("mu", ctypes.c_double), ("nu_bar", ctypes.c_double),
        ("z_lo", ctypes.c_double * 3), ("z_hi", ctypes.c_double * 3),
        ("sigma", ctypes.c_double * 3),
        ("alpha0", ctypes.c_double), ("sigma_alpha", ctypes.c_double),
        ("ua_lo", ctypes.c_double), ("ua_hi", ctypes.c_double),
        ("w_u", ctypes.c_double * 3), ("w_alpha", ctypes.c_double),
        ("rho", ctypes.c_double), ("h_floor", ctypes.c_double),
        ("q_coll", ctypes.c_double),
        ("alpha_stab", ctypes.c_double), ("q_stab", ctypes.c_double * 2),
        ("q_abuf", ctypes.c_double), ("h_buf", ctypes.c_double),
        ("n_discs", ctypes.c_int32), ("disc_trailer_mask", ctypes.c_int32),
        ("disc_off", ctypes.c_double * 8),
    ]

_INT_FIELDS = ("S", "H", "flags", "n_discs", "disc_trailer_mask")

PROJ_NONE = 1
COLLISION_COST = 2
OBS8 = 4
ALPHA_BUFFER = 8
THIRD_ORDER = 16
JERK = 32


def state_dim(p: dict) -> int:
    """Entries of a state under the flags of p (8 for the jerk model)."""
    return 8 if int(p["flags"]) & JERK else 7


def obs_stride(p: dict) -> int:
    """Doubles per obstacle row under the flags of p."""
    return 8 if int(p["flags"]) & OBS8 else 6


_DP = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER(_Params)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            sig = {
                "orc_philox4x32_10": (None, [u32p, u32p, u32p]),
                "orc_normals": (None, [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                       ctypes.c_uint32, ctypes.c_int, _DP]),
                "orc_dynamics_step": (None, [P, _DP, _DP, _DP]),
                "orc_obstacle_h": (ctypes.c_double, [P, _DP, _DP]),
                "orc_obstacle_row": (None, [P, _DP, _DP, _DP, _DP, _DP]),
                "orc_hitch_h": (ctypes.c_double, [P, _DP]),
                "orc_hitch_row": (None, [P, _DP, _DP, _DP, _DP]),
                "orc_project": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _DP, _DP, _DP,
                                               ctypes.c_double, _DP, _DP, _DP, _DP]),
                "orc_path_lookup": (None, [_DP, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                           _DP, _DP, _DP]),
                "orc_stage_cost": (ctypes.c_double, [P, _DP, _DP, _DP, ctypes.c_int,
                                                     ctypes.c_double]),
                "orc_softmin": (ctypes.c_int, [ctypes.c_int, _DP, ctypes.c_double, _DP]),
                "orc_rollout_sample": (ctypes.c_int, [P, _DP, _DP, _DP, ctypes.c_int, _DP,
                                                      ctypes.c_int, ctypes.c_double,
                                                      ctypes.c_uint64, ctypes.c_uint64,
                                                      ctypes.c_uint32, _DP, _DP, _DP, _DP,
                                                      _DP, _DP]),
                "orc_solve": (ctypes.c_int, [P, _DP, _DP, _DP, ctypes.c_int, _DP, ctypes.c_int,
                                             ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64,
                                             _DP, _DP, _DP, _DP, _DP]),
                "orc_integrate": (None, [P, _DP, _DP, ctypes.c_int, _DP]),
                "orc_noise_table": (None, [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, u32p, _DP]),
                "orc_update": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _DP, _DP, ctypes.c_double,
                                              _DP, _DP, _DP]),
                "orc_rollout_range": (ctypes.c_int, [P, _DP, _DP, _DP, ctypes.c_int, _DP, ctypes.c_int,
                                                     ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64,
                                                     ctypes.c_uint32, ctypes.c_uint32, _DP, _DP, _DP]),
                "orc_obstacle_h_at": (ctypes.c_double, [P, _DP, ctypes.c_int, ctypes.c_double,
                                                        _DP]),
                "orc_obstacle_row_at": (None, [P, _DP, ctypes.c_int, ctypes.c_double, _DP, _DP,
                                               _DP, _DP]),
                "orc_collision_cost": (ctypes.c_double, [P, _DP, ctypes.c_int, ctypes.c_int,
                                                         ctypes.c_double, _DP]),
                "orc_alpha_buffer_cost": (ctypes.c_double, [P, ctypes.c_int, _DP, _DP]),
                "orc_hitch_stabilize": (ctypes.c_int, [P, _DP, _DP, _DP, _DP]),
                "orc_obstacle_row3": (None, [P, _DP, ctypes.c_int, ctypes.c_double, _DP, _DP, _DP,
                                             _DP]),
                "orc_jerk_step": (None, [P, _DP, _DP, _DP]),
                "orc_jerk_integrate": (None, [P, _DP, _DP, ctypes.c_int, _DP]),
                "orc_jerk_hitch_row": (None, [P, _DP, _DP, _DP, _DP]),
                "orc_jerk_obstacle_row": (None, [P, _DP, ctypes.c_int, ctypes.c_double, _DP, _DP,
                                                 _DP, _DP]),
                "orc_disc_position": (None, [P, ctypes.c_int, _DP, _DP]),
                "orc_disc_h": (ctypes.c_double, [P, _DP, ctypes.c_int, ctypes.c_double,
                                                 ctypes.c_int, _DP]),
                "orc_disc_row": (None, [P, _DP, ctypes.c_int, ctypes.c_double, ctypes.c_int, _DP,
                                        _DP, _DP, _DP]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


class using_library:
    """Context manager: route every wrapper in this module through another
    build of the oracle (the mutation tests compile planted mistakes into
    copies of the source and check that the pins catch them)."""

    def __init__(self, path: str):
        self.path = path
        self.saved = None

    def __enter__(self):
        global _lib
        _load()
        with _lock:
            self.saved = _lib
            _lib = None
        # load the alternative build with the same prototypes
        lib = ctypes.CDLL(self.path)
        for name in ("orc_philox4x32_10", "orc_normals", "orc_dynamics_step", "orc_obstacle_h",
                     "orc_obstacle_row", "orc_hitch_h", "orc_hitch_row", "orc_project",
                     "orc_path_lookup", "orc_stage_cost", "orc_softmin", "orc_rollout_sample",
                     "orc_solve", "orc_integrate", "orc_obstacle_h_at", "orc_obstacle_row_at",
                     "orc_collision_cost", "orc_alpha_buffer_cost", "orc_hitch_stabilize",
                     "orc_disc_position", "orc_disc_h", "orc_disc_row", "orc_obstacle_row3",
                     "orc_jerk_step", "orc_jerk_integrate", "orc_jerk_hitch_row",
                     "orc_jerk_obstacle_row"):
            src = getattr(self.saved, name)
            dst = getattr(lib, name)
            dst.restype = src.restype
            dst.argtypes = src.argtypes
        with _lock:
            _lib = lib
        return lib

    def __exit__(self, *exc):
        global _lib
        with _lock:
            _lib = self.saved
        return False


def compile_variant(source_text: str, out_dir: str, name: str = "variant") -> str:
    """Compile a (modified) copy of the oracle source into out_dir."""
    c_path = os.path.join(out_dir, name + ".c")
    so_path = os.path.join(out_dir, name + ".so")
    with open(c_path, "w") as f:
        f.write(source_text)
    import shutil
    shutil.copy(_HDR, os.path.join(out_dir, os.path.basename(_HDR)))
    subprocess.run(["gcc", "-std=c11", "-D_DEFAULT_SOURCE", "-O1", "-fPIC", "-shared",
                    "-fno-fast-math", "-ffp-contract=off", "-o", so_path, c_path, "-lm"],
                   check=True)
    return so_path


def source() -> str:
    with open(_SRC) as f:
        return f.read()


def _params(p: dict, S: int | None = None, H: int | None = None) -> _Params:
    out = _Params()
    for name, _ in _Params._fields_:
        key = "lambda" if name == "lambda_" else name
        val = p[key]
        if name == "S" and S is not None:
            val = S
        if name == "H" and H is not None:
            val = H
        attr = getattr(out, name)
        if isinstance(attr, ctypes.Array):
            for i, v in enumerate(val):
                attr[i] = float(v)
        elif name in _INT_FIELDS:
            setattr(out, name, int(val))
        else:
            setattr(out, name, float(val))
    return out


def _d(a, n=None):
    arr = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None:
        assert arr.size == n, (arr.size, n)
    return arr


def _ptr(arr):
    if arr is None:
        return None
    return arr.ctypes.data_as(_DP)


# ----------------------------------------------------------------------------
def philox4x32_10(ctr, key) -> np.ndarray:
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    lib.orc_philox4x32_10(c.ctypes.data_as(u32p), k.ctypes.data_as(u32p), out.ctypes.data_as(u32p))
    return out


def normals(seed: int, counter: int, s: int, tau: int, d: int) -> np.ndarray:
    lib = _load()
    out = np.zeros(d, dtype=np.float64)
    lib.orc_normals(seed, counter, s, tau, d, _ptr(out))
    return out


def dynamics_step(p: dict, x, u) -> np.ndarray:
    lib = _load()
    P = _params(p)
    xn = np.zeros(7)
    lib.orc_dynamics_step(ctypes.byref(P), _ptr(_d(x, 7)), _ptr(_d(u, 3)), _ptr(xn))
    return xn


def integrate(p: dict, x0, U) -> np.ndarray:
    lib = _load()
    U = _d(U)
    H = U.size // 3
    traj = np.zeros((H + 1, 7))
    P = _params(p)
    lib.orc_integrate(ctypes.byref(P), _ptr(_d(x0, 7)), _ptr(U), H, _ptr(traj))
    return traj


def obstacle_h(p: dict, obs, x) -> float:
    lib = _load()
    P = _params(p)
    return lib.orc_obstacle_h(ctypes.byref(P), _ptr(_d(obs, 6)), _ptr(_d(x, 7)))


def obstacle_row(p: dict, obs, x):
    """Returns (A_u[3], h, b_rest) with b = -alpha*h + b_rest."""
    lib = _load()
    P = _params(p)
    Au = np.zeros(3)
    h = ctypes.c_double()
    br = ctypes.c_double()
    lib.orc_obstacle_row(ctypes.byref(P), _ptr(_d(obs, 6)), _ptr(_d(x, 7)), _ptr(Au),
                         ctypes.byref(h), ctypes.byref(br))
    return Au, h.value, br.value


def obstacle_h_at(p: dict, obs, x, t: float) -> float:
    """h of one obstacle row (6 or 8 entries) at time t."""
    lib = _load()
    o = _d(obs)
    return lib.orc_obstacle_h_at(ctypes.byref(_params(p)), _ptr(o), o.size, float(t),
                                 _ptr(_d(x, 7)))


def obstacle_row_at(p: dict, obs, x, t: float):
    """Row of one obstacle (6 or 8 entries) at time t: (A_u[3], h, b_rest)."""
    lib = _load()
    o = _d(obs)
    Au = np.zeros(3)
    h = ctypes.c_double()
    br = ctypes.c_double()
    lib.orc_obstacle_row_at(ctypes.byref(_params(p)), _ptr(o), o.size, float(t), _ptr(_d(x, 7)),
                            _ptr(Au), ctypes.byref(h), ctypes.byref(br))
    return Au, h.value, br.value


def collision_cost(p: dict, obs, x, t: float = 0.0) -> float:
    lib = _load()
    stride = obs_stride(p)
    o = _d(obs).reshape(-1, stride)
    return lib.orc_collision_cost(ctypes.byref(_params(p)), _ptr(o) if o.size else None, stride,
                                  o.shape[0], float(t), _ptr(_d(x, 7)))


def alpha_buffer_cost(p: dict, h, alpha) -> float:
    lib = _load()
    h = _d(h)
    return lib.orc_alpha_buffer_cost(ctypes.byref(_params(p)), h.size, _ptr(h),
                                     _ptr(_d(alpha, h.size)))


def jerk_step(p: dict, x, u) -> np.ndarray:
    lib = _load()
    xn = np.zeros(8)
    lib.orc_jerk_step(ctypes.byref(_params(p)), _ptr(_d(x, 8)), _ptr(_d(u, 3)), _ptr(xn))
    return xn


def jerk_integrate(p: dict, x0, U) -> np.ndarray:
    lib = _load()
    U = _d(U)
    H = U.size // 3
    traj = np.zeros((H + 1, 8))
    lib.orc_jerk_integrate(ctypes.byref(_params(p)), _ptr(_d(x0, 8)), _ptr(U), H, _ptr(traj))
    return traj


def jerk_hitch_row(p: dict, x):
    lib = _load()
    Au = np.zeros(3)
    h = ctypes.c_double()
    br = ctypes.c_double()
    lib.orc_jerk_hitch_row(ctypes.byref(_params(p)), _ptr(_d(x, 8)), _ptr(Au), ctypes.byref(h),
                           ctypes.byref(br))
    return Au, h.value, br.value


def jerk_obstacle_row(p: dict, obs, x, t: float = 0.0):
    lib = _load()
    o = _d(obs)
    Au = np.zeros(3)
    h = ctypes.c_double()
    br = ctypes.c_double()
    lib.orc_jerk_obstacle_row(ctypes.byref(_params(p)), _ptr(o), o.size, float(t), _ptr(_d(x, 8)),
                              _ptr(Au), ctypes.byref(h), ctypes.byref(br))
    return Au, h.value, br.value


def obstacle_row3(p: dict, obs, x, t: float = 0.0):
    """Third-order row of one obstacle (6 or 8 entries): (A_u[3], h, b_rest)."""
    lib = _load()
    o = _d(obs)
    Au = np.zeros(3)
    h = ctypes.c_double()
    br = ctypes.c_double()
    lib.orc_obstacle_row3(ctypes.byref(_params(p)), _ptr(o), o.size, float(t), _ptr(_d(x, 7)),
                          _ptr(Au), ctypes.byref(h), ctypes.byref(br))
    return Au, h.value, br.value


def disc_position(p: dict, m: int, x):
    lib = _load()
    pos = np.zeros(2)
    lib.orc_disc_position(ctypes.byref(_params(p)), int(m), _ptr(_d(x, 7)), _ptr(pos))
    return pos


def disc_h(p: dict, obs, m: int, x, t: float = 0.0) -> float:
    lib = _load()
    o = _d(obs)
    return lib.orc_disc_h(ctypes.byref(_params(p)), _ptr(o), o.size, float(t), int(m),
                          _ptr(_d(x, 7)))


def disc_row(p: dict, obs, m: int, x, t: float = 0.0):
    """Row of one obstacle (6 or 8 entries) seen from disc m: (A_u[3], h, b_rest)."""
    lib = _load()
    o = _d(obs)
    Au = np.zeros(3)
    h = ctypes.c_double()
    br = ctypes.c_double()
    lib.orc_disc_row(ctypes.byref(_params(p)), _ptr(o), o.size, float(t), int(m), _ptr(_d(x, 7)),
                     _ptr(Au), ctypes.byref(h), ctypes.byref(br))
    return Au, h.value, br.value


def hitch_stabilize(p: dict, x, u_ref):
    """Returns (infeasible, u[3], slack)."""
    lib = _load()
    u = np.zeros(3)
    sl = ctypes.c_double()
    st = lib.orc_hitch_stabilize(ctypes.byref(_params(p)), _ptr(_d(x, state_dim(p))), _ptr(_d(u_ref, 3)),
                                 _ptr(u), ctypes.byref(sl))
    return st, u, sl.value


def hitch_h(p: dict, x) -> float:
    lib = _load()
    P = _params(p)
    return lib.orc_hitch_h(ctypes.byref(P), _ptr(_d(x, 7)))


def hitch_row(p: dict, x):
    lib = _load()
    P = _params(p)
    Au = np.zeros(3)
    h = ctypes.c_double()
    br = ctypes.c_double()
    lib.orc_hitch_row(ctypes.byref(P), _ptr(_d(x, 7)), _ptr(Au), ctypes.byref(h),
                      ctypes.byref(br))
    return Au, h.value, br.value


def project(A, b, w, rho, z_lo, z_hi, z_des):
    """Dense closed-form soft projection. Returns (status, z_star)."""
    lib = _load()
    z_des = _d(z_des)
    d = z_des.size
    A = _d(A).reshape(-1)
    nc = A.size // d if d else 0
    b = _d(b, nc)
    z = np.zeros(d)
    st = lib.orc_project(d, nc, _ptr(A) if nc else None, _ptr(b) if nc else None,
                         _ptr(_d(w, d)), float(rho), _ptr(_d(z_lo, d)), _ptr(_d(z_hi, d)),
                         _ptr(z_des), _ptr(z))
    return st, z


def path_lookup(path, ds, psi):
    lib = _load()
    path = _d(path)
    n = path.size // 3
    xr, yr, thr = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib.orc_path_lookup(_ptr(path), n, float(ds), float(psi), ctypes.byref(xr), ctypes.byref(yr),
                        ctypes.byref(thr))
    return xr.value, yr.value, thr.value


def stage_cost(p: dict, x, u, path, ds) -> float:
    lib = _load()
    P = _params(p)
    path = _d(path)
    return lib.orc_stage_cost(ctypes.byref(P), _ptr(_d(x, 7)), _ptr(_d(u, 3)), _ptr(path),
                              path.size // 3, float(ds))


def softmin(J, lam):
    lib = _load()
    J = _d(J)
    g = np.zeros_like(J)
    st = lib.orc_softmin(J.size, _ptr(J), float(lam), _ptr(g))
    return st, g


def rollout_sample(p: dict, x0, U_nom, obs, path, ds, seed, counter, s):
    """One rollout; returns dict(states, u, alpha, z_des, z_star, J, status)."""
    lib = _load()
    H = int(p["H"])
    obs = _d(obs).reshape(-1, obs_stride(p))
    n_obs = obs.shape[0]
    Nc = 1 + n_obs * int(p.get("n_discs", 1))
    d = 3 + Nc
    path = _d(path)
    nx = state_dim(p)
    out = dict(states=np.zeros((H + 1, nx)), u=np.zeros((H, 3)), alpha=np.zeros((H + 1, Nc)),
               z_des=np.zeros((H, d)), z_star=np.zeros((H, d)))
    J = ctypes.c_double()
    P = _params(p)
    st = lib.orc_rollout_sample(ctypes.byref(P), _ptr(_d(x0, nx)), _ptr(_d(U_nom, 3 * H)),
                                _ptr(obs) if n_obs else None, n_obs, _ptr(path), path.size // 3,
                                float(ds), int(seed), int(counter), int(s),
                                _ptr(out["states"]), _ptr(out["u"]), _ptr(out["alpha"]),
                                _ptr(out["z_des"]), _ptr(out["z_star"]), ctypes.byref(J))
    out["J"] = J.value
    out["status"] = st
    return out


def solve(p: dict, x0, U_nom, obs, path, ds, seed, counter, *, want_J=True, want_uhist=False,
          want_states=False, S: int | None = None):
    """The full solve. Returns dict(U, traj, J, u_hist, states, status)."""
    lib = _load()
    S = int(p["S"]) if S is None else int(S)
    H = int(p["H"])
    obs = _d(obs).reshape(-1, obs_stride(p))
    n_obs = obs.shape[0]
    path = _d(path)
    nx = state_dim(p)
    U = np.zeros((H, 3))
    traj = np.zeros((H + 1, nx))
    J = np.zeros(S) if want_J else None
    uh = np.zeros((S, H, 3)) if want_uhist else None
    xs = np.zeros((S, H + 1, nx)) if want_states else None
    P = _params(p, S=S)
    st = lib.orc_solve(ctypes.byref(P), _ptr(_d(x0, nx)), _ptr(_d(U_nom, 3 * H)),
                       _ptr(obs) if n_obs else None, n_obs, _ptr(path), path.size // 3,
                       float(ds), int(seed), int(counter), _ptr(U), _ptr(traj), _ptr(J),
                       _ptr(uh), _ptr(xs))
    return dict(U=U, traj=traj, J=J, u_hist=uh, states=xs, status=st)


def update(J, u_hist, lam, U_nom):
    """The MPPI update of Sec. II-B from given costs J (S,) and applied
    inputs u_hist (S, H, 3): softmin weights, then the weighted sum in
    sample order.  Returns (status, U (H, 3), gamma_bar (S,))."""
    lib = _load()
    J = _d(J)
    uh = _d(u_hist)
    S = J.size
    H = uh.size // (3 * S) if S else 0
    U = np.zeros((H, 3))
    g = np.zeros(S)
    st = lib.orc_update(S, H, _ptr(J), _ptr(uh), float(lam), _ptr(_d(U_nom, 3 * H)), _ptr(g), _ptr(U))
    return st, U, g


def rollouts(p: dict, x0, U_nom, obs, path, ds, seed, counter, s0: int, s1: int, *, want_uhist=True,
             want_states=False):
    """Rollouts of samples s0 .. s1-1 of one solve (each as rollout_sample):
    dict(J (n,), u_hist (n, H, 3) or None, states (n, H+1, NX) or None,
    status).  A solve's samples can be spread over worker processes and
    joined with `update`."""
    lib = _load()
    n = int(s1) - int(s0)
    H = int(p["H"])
    obs = _d(obs).reshape(-1, obs_stride(p))
    n_obs = obs.shape[0]
    path = _d(path)
    nx = state_dim(p)
    J = np.zeros(n)
    uh = np.zeros((n, H, 3)) if want_uhist else None
    xs = np.zeros((n, H + 1, nx)) if want_states else None
    P = _params(p)
    st = lib.orc_rollout_range(ctypes.byref(P), _ptr(_d(x0, nx)), _ptr(_d(U_nom, 3 * H)),
                               _ptr(obs) if n_obs else None, n_obs, _ptr(path), path.size // 3,
                               float(ds), int(seed), int(counter), int(s0), int(s1), _ptr(J),
                               _ptr(uh), _ptr(xs))
    return dict(J=J, u_hist=uh, states=xs, status=st)


def noise_table(seed: int, counter: int, n_samples: int, H: int, n_blocks: int):
    """The noise stream block by block: (words uint32, normals float64), each
    of shape (n_samples, H, n_blocks, 4)."""
    lib = _load()
    w = np.zeros((n_samples, H, n_blocks, 4), dtype=np.uint32)
    n = np.zeros((n_samples, H, n_blocks, 4))
    lib.orc_noise_table(int(seed), int(counter), int(n_samples), int(H), int(n_blocks),
                        w.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), _ptr(n))
    return w, n
