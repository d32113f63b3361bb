"""Seeded synthetic inputs for BR-MPPI solves: parameters, reference paths,
obstacle sets and initial states.

This module builds *inputs* only.  It holds none of the method's arithmetic
(no dynamics, barriers, projection, cost or weighting), so both the CUDA path
and the CPU oracle can be fed from it without sharing method code.

The workloads stand in for the paper's CarMaker parking scenes (Sec. V),
which are not reproducible here; the recipes are:

* ``config1``: S=256, H=30, one ellipse 3 m left of the path midpoint; path a
  20 m straight then a 90 deg left arc of R=12 m, driven in reverse from
  x0 = (0, 0, pi, pi, -1, 0, 0).
* ``config1b``: as config1 with the obstacle on the path 2.5 m behind the
  vehicle (the rows are active).
* ``config2``: S=4096, H=50, 8 random ellipses within 6 m of a reverse-parking
  path (15 m straight, 90 deg arc of R=10 m, 8 m straight).
* ``config3``: 256 uneven instances (S, H, obstacle count, path) from seed 1.
* ``config5``: S=65536, H=100, 64 ellipses in a 60 x 60 m lot, a 120 m
  multi-arc path at ds=0.05.
"""
from __future__ import annotations

import math

import numpy as np

#: Default parameters (tractor-trailer geometry and weights of the workloads;
#: where the paper leaves a value open, the value chosen here is a reading
#: of it: alpha0 = 0.5, the alpha-input noise and bounds, w_alpha, rho,
#: h_floor, nu_bar).
DEFAULT_PARAMS = dict(
    S=256, H=30, flags=0,
    Ts=0.05, **{"lambda": 1.0},
    l1=4.0, lh=0.5, l2=8.0, dtheta_max=0.9, kappa=0.1, r_inflate=0.0,
    Qc=10.0, Ql=10.0, Qth=5.0, R=(0.1, 0.1, 0.01), mu=1.0, nu_bar=3.0,
    z_lo=(-2.0, -0.6, 0.0), z_hi=(2.0, 0.6, 3.0), sigma=(0.5, 0.3, 0.5),
    alpha0=0.5, sigma_alpha=0.1, ua_lo=-0.5, ua_hi=0.5,
    w_u=(1.0, 1.0, 1.0), w_alpha=1.0, rho=0.01, h_floor=1e-6,
    q_coll=100.0, alpha_stab=0.5, q_stab=(1.0, 1.0), q_abuf=10.0, h_buf=0.5,
    n_discs=1, disc_trailer_mask=0, disc_off=(0.0,) * 8,
)

#: A tractor-trailer footprint of five discs: three along the tractor (rear
#: axle, mid, front) and two along the trailer (axle, front).
FIVE_DISCS = dict(n_discs=5, disc_trailer_mask=0b11000,
                  disc_off=(0.0, 2.0, 4.0, 0.0, 4.0, 0.0, 0.0, 0.0))

FLAG_PROJ_NONE = 1
FLAG_COLLISION_COST = 2
FLAG_OBS8 = 4
FLAG_ALPHA_BUFFER = 8
FLAG_THIRD_ORDER = 16
FLAG_JERK = 32


def params(**overrides) -> dict:
    p = dict(DEFAULT_PARAMS)
    p.update(overrides)
    return p


def as_float32(p: dict) -> dict:
    """Round every real parameter to binary32 (the precision the CUDA path
    receives), so a second consumer sees identical numbers."""
    out = {}
    for k, v in p.items():
        if k in ("S", "H", "flags", "n_discs", "disc_trailer_mask"):
            out[k] = int(v)
        elif isinstance(v, (tuple, list, np.ndarray)):
            out[k] = tuple(float(np.float32(x)) for x in v)
        else:
            out[k] = float(np.float32(v))
    return out


# ----------------------------------------------------------------------------
# Reference paths: a table of (x, y, heading) sampled every ds of arc length.
def path_table(segments, ds: float, reverse: bool, start=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Sample a path made of straights ("S", length) and arcs
    ("A", radius, signed_angle_rad) every ``ds`` metres.

    The heading column is the vehicle heading, unwrapped: the travel tangent,
    plus pi on a path driven in reverse.  Returns float32 (n, 3) with
    n = floor(L / ds) + 1 (a tail shorter than ds is dropped).
    """
    # segment start poses
    x, y, phi = start
    starts = []
    total = 0.0
    for seg in segments:
        starts.append((total, x, y, phi, seg))
        if seg[0] == "S":
            L = float(seg[1])
            x += L * math.cos(phi)
            y += L * math.sin(phi)
        else:
            R, ang = float(seg[1]), float(seg[2])
            L = R * abs(ang)
            k = math.copysign(1.0 / R, ang)
            phi1 = phi + ang
            x += (math.sin(phi1) - math.sin(phi)) / k
            y += -(math.cos(phi1) - math.cos(phi)) / k
            phi = phi1
        total += L
    n = int(math.floor(total / ds + 1e-9)) + 1
    out = np.zeros((n, 3), dtype=np.float64)
    si = 0
    for j in range(n):
        s = j * ds
        while si + 1 < len(starts) and s >= starts[si + 1][0]:
            si += 1
        s0, x0, y0, phi0, seg = starts[si]
        t = s - s0
        if seg[0] == "S":
            px, py, ph = x0 + t * math.cos(phi0), y0 + t * math.sin(phi0), phi0
        else:
            R, ang = float(seg[1]), float(seg[2])
            k = math.copysign(1.0 / R, ang)
            ph = phi0 + k * t
            px = x0 + (math.sin(ph) - math.sin(phi0)) / k
            py = y0 - (math.cos(ph) - math.cos(phi0)) / k
        out[j] = (px, py, ph + (math.pi if reverse else 0.0))
    return out.astype(np.float32)


def _path_point(segments, s, start=(0.0, 0.0, 0.0)):
    """Pose (x, y, tangent) at arc length s (for placing obstacles)."""
    tab = path_table(segments, 0.01, False, start).astype(np.float64)
    j = min(int(round(s / 0.01)), tab.shape[0] - 1)
    return tab[j]


def _segments_length(segments) -> float:
    return sum(float(s[1]) if s[0] == "S" else float(s[1]) * abs(float(s[2])) for s in segments)


def _far_from(c, pts, semi):
    """Conservative keep-out test: the centre is farther than the larger
    semi-axis plus 0.5 m from every point."""
    return all(math.hypot(c[0] - p[0], c[1] - p[1]) > max(semi) + 0.5 for p in pts)


def _scenario(p, x0, path, ds, obs, seed=0, counter=0, U_nom=None):
    H = int(p["H"])
    width = 8 if int(p.get("flags", 0)) & FLAG_OBS8 else 6
    obs = np.asarray(obs, dtype=np.float32).reshape(-1, width)
    if U_nom is None:
        U_nom = np.zeros((H, 3), dtype=np.float32)
    return dict(params=p, x0=np.asarray(x0, dtype=np.float64), U_nom=np.asarray(U_nom, np.float32),
                obs=obs, path=np.asarray(path, np.float32), ds=float(ds), seed=int(seed),
                counter=int(counter))


# ----------------------------------------------------------------------------
C1_SEGMENTS = [("S", 20.0), ("A", 12.0, math.pi / 2)]
C2_SEGMENTS = [("S", 15.0), ("A", 10.0, math.pi / 2), ("S", 8.0)]


def config1(seed: int = 0, S: int = 256, H: int = 30) -> dict:
    p = params(S=S, H=H)
    path = path_table(C1_SEGMENTS, 0.1, reverse=True)
    L = _segments_length(C1_SEGMENTS)
    px, py, ph = _path_point(C1_SEGMENTS, 0.5 * L)
    cx, cy = px - 3.0 * math.sin(ph), py + 3.0 * math.cos(ph)
    obs = [(cx, cy, 1.0, 0.6, 0.3, 2.0)]
    x0 = (0.0, 0.0, math.pi, math.pi, -1.0, 0.0, 0.0)
    return _scenario(p, x0, path, 0.1, obs, seed=seed)


def config1b(seed: int = 0, S: int = 256, H: int = 30) -> dict:
    sc = config1(seed, S, H)
    sc["obs"] = np.asarray([(2.5, 0.3, 1.0, 0.6, 0.3, 2.0)], dtype=np.float32)
    return sc


def config2(seed: int = 2, S: int = 4096, H: int = 50, n_obs: int = 8) -> dict:
    rng = np.random.default_rng(seed)
    p = params(S=S, H=H)
    path = path_table(C2_SEGMENTS, 0.1, reverse=True)
    L = _segments_length(C2_SEGMENTS)
    x0 = (0.0, 0.0, math.pi, math.pi, -1.0, 0.0, 0.0)
    end = path[-1].astype(np.float64)
    keep_out = [(x0[0], x0[1]), (float(end[0]), float(end[1]))]
    obs = []
    while len(obs) < n_obs:
        ax, ay = rng.uniform(0.3, 1.5, size=2)
        th = rng.uniform(0.0, math.pi)
        s = rng.uniform(0.0, L)
        lat = rng.uniform(-6.0, 6.0)
        px, py, ph = _path_point(C2_SEGMENTS, s)
        c = (px - lat * math.sin(ph), py + lat * math.cos(ph))
        if _far_from(c, keep_out, (ax, ay)):
            obs.append((c[0], c[1], ax, ay, th, 2.0))
    return _scenario(p, x0, path, 0.1, obs, seed=seed)


def random_instance(rng: np.random.Generator, S_choices=(1024, 2048, 4096, 8192), H_range=(30, 80),
                    obs_range=(0, 16), ds: float = 0.1, seed: int = 0) -> dict:
    """One uneven instance of the batched workload: straight U[10, 25] m then
    an arc of radius U[8, 15] m and angle U[45, 120] deg with random turn
    sign, forward or reverse with probability 1/2; config-1 shaped
    obstacles 3 m to a random side of random path points."""
    S = int(rng.choice(S_choices))
    H = int(rng.integers(H_range[0], H_range[1] + 1))
    n_obs = int(rng.integers(obs_range[0], obs_range[1] + 1))
    straight = float(rng.uniform(10.0, 25.0))
    R = float(rng.uniform(8.0, 15.0))
    ang = math.radians(float(rng.uniform(45.0, 120.0))) * float(rng.choice((-1.0, 1.0)))
    reverse = bool(rng.random() < 0.5)
    segs = [("S", straight), ("A", R, ang)]
    path = path_table(segs, ds, reverse=reverse)
    L = _segments_length(segs)
    head = math.pi if reverse else 0.0
    v0 = -1.0 if reverse else 1.0
    x0 = (0.0, 0.0, head, head, v0, 0.0, 0.0)
    obs = []
    while len(obs) < n_obs:
        s = float(rng.uniform(0.0, L))
        side = float(rng.choice((-1.0, 1.0)))
        px, py, ph = _path_point(segs, s)
        c = (px - 3.0 * side * math.sin(ph), py + 3.0 * side * math.cos(ph))
        if _far_from(c, [(0.0, 0.0)], (1.0, 0.6)):
            obs.append((c[0], c[1], 1.0, 0.6, 0.3, 2.0))
    p = params(S=S, H=H)
    return _scenario(p, x0, path, ds, obs, seed=int(rng.integers(0, 2**63 - 1)))


def config3(seed: int = 1, n_instances: int = 256) -> list:
    rng = np.random.default_rng(seed)
    return [random_instance(rng) for _ in range(n_instances)]


def config5(seed: int = 5, S: int = 65536, H: int = 100, n_obs: int = 64) -> dict:
    rng = np.random.default_rng(seed)
    segs = []
    total, sign = 0.0, 1.0
    while total < 120.0 - 1e-9:
        for seg in (("S", 10.0), ("A", 12.0, sign * math.pi / 3)):
            L = seg[1] if seg[0] == "S" else 12.0 * math.pi / 3
            if total + L > 120.0:
                rem = 120.0 - total
                seg = ("S", rem) if seg[0] == "S" else ("A", 12.0, sign * rem / 12.0)
                L = rem
            segs.append(seg)
            total += L
            if total >= 120.0 - 1e-9:
                break
        sign = -sign
    path = path_table(segs, 0.05, reverse=False)
    cxm, cym = path[:, 0].astype(np.float64).mean(), path[:, 1].astype(np.float64).mean()
    x0 = (0.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0)
    obs = []
    while len(obs) < n_obs:
        ax, ay = rng.uniform(0.2, 2.0, size=2)
        th = rng.uniform(0.0, math.pi)
        c = (cxm + rng.uniform(-30.0, 30.0), cym + rng.uniform(-30.0, 30.0))
        if _far_from(c, [(0.0, 0.0)], (ax, ay)):
            obs.append((c[0], c[1], ax, ay, th, 2.0))
    return _scenario(params(S=S, H=H), x0, path, 0.05, obs, seed=seed)


def small_random(seed: int, S: int = 64, H: int = 12, n_obs: int = 3, reverse: bool = True,
                 near: bool = True) -> dict:
    """Tiny random case for fuzzing: obstacles placed 1-3 m from the first
    metres of the path so that their rows are active."""
    rng = np.random.default_rng(seed)
    segs = [("S", float(rng.uniform(5.0, 12.0))),
            ("A", float(rng.uniform(6.0, 12.0)), float(rng.uniform(-1.5, 1.5)))]
    path = path_table(segs, 0.1, reverse=reverse)
    head = math.pi if reverse else 0.0
    v0 = -1.0 if reverse else 1.0
    x0 = (0.0, 0.0, head, head, v0, float(rng.uniform(-0.1, 0.1)), 0.0)
    obs = []
    while len(obs) < n_obs:
        s = float(rng.uniform(0.5, 4.0)) if near else float(rng.uniform(0.0, 15.0))
        lat = float(rng.uniform(-2.5, 2.5))
        px, py, ph = _path_point(segs, s)
        c = (px - lat * math.sin(ph), py + lat * math.cos(ph))
        ax, ay = rng.uniform(0.3, 1.0, size=2)
        if _far_from(c, [(0.0, 0.0)], (ax, ay)):
            obs.append((c[0], c[1], ax, ay, float(rng.uniform(0, math.pi)), 2.0))
    p = params(S=S, H=H)
    U_nom = rng.uniform(-0.3, 0.3, size=(H, 3)).astype(np.float32)
    U_nom[:, 2] = np.abs(U_nom[:, 2]) * 3.0
    return _scenario(p, x0, path, 0.1, obs, seed=int(rng.integers(0, 2**63 - 1)),
                     counter=int(rng.integers(0, 2**32)), U_nom=U_nom)


def with_moving(c: dict, seed: int, e4_frac: float = 0.5, speed=(0.3, 1.5)) -> dict:
    """The scenario with 8-float obstacle rows (flag FLAG_OBS8): a share
    e4_frac of its obstacles become e = 4 super-ellipses (parked vehicles,
    Sec. IV-C), the others move at a speed U[speed] m/s in a random
    direction (predicted pedestrians; constant-velocity prediction)."""
    rng = np.random.default_rng(seed)
    p = dict(c["params"], flags=int(c["params"].get("flags", 0)) | FLAG_OBS8)
    rows = []
    for o in np.asarray(c["obs"], np.float64).reshape(-1, 6):
        if rng.random() < e4_frac:
            rows.append((*o[:5], 4.0, 0.0, 0.0))
        else:
            sp = rng.uniform(*speed)
            ang = rng.uniform(-math.pi, math.pi)
            rows.append((*o[:5], 2.0, sp * math.cos(ang), sp * math.sin(ang)))
    out = dict(c)
    out["params"] = p
    out["obs"] = np.asarray(rows, dtype=np.float32).reshape(-1, 8)
    return out


def crossing(seed: int = 6, S: int = 4096, H: int = 50, n_parked: int = 6, n_ped: int = 2) -> dict:
    """Reverse parking with parked vehicles and crossing pedestrians (the
    scene type of Sec. V): config-2's reverse-parking path, parked vehicles
    as e = 4 super-ellipses with semi-axes (2.3, 0.95) m beside the path
    (3.5-6 m lateral, either side), pedestrians as e = 2 circles of radius
    0.5 m starting 3-5 m to one side of a path point and walking across the
    path at 1.0-1.5 m/s.  Obstacle rows of 8 (flag FLAG_OBS8)."""
    rng = np.random.default_rng(seed)
    p = params(S=S, H=H, flags=FLAG_OBS8)
    path = path_table(C2_SEGMENTS, 0.1, reverse=True)
    L = _segments_length(C2_SEGMENTS)
    x0 = (0.0, 0.0, math.pi, math.pi, -1.0, 0.0, 0.0)
    end = path[-1].astype(np.float64)
    keep_out = [(x0[0], x0[1]), (float(end[0]), float(end[1]))]
    obs = []
    while len(obs) < n_parked:
        s = rng.uniform(0.0, L)
        lat = float(rng.choice((-1.0, 1.0))) * rng.uniform(3.5, 6.0)
        px, py, ph = _path_point(C2_SEGMENTS, s)
        c = (px - lat * math.sin(ph), py + lat * math.cos(ph))
        if _far_from(c, keep_out, (2.3, 0.95)):
            obs.append((c[0], c[1], 2.3, 0.95, ph, 4.0, 0.0, 0.0))
    while len(obs) < n_parked + n_ped:
        s = rng.uniform(2.0, 12.0)
        side = float(rng.choice((-1.0, 1.0)))
        px, py, ph = _path_point(C2_SEGMENTS, s)
        d = rng.uniform(3.0, 5.0)
        c = (px - side * d * math.sin(ph), py + side * d * math.cos(ph))
        sp = rng.uniform(1.0, 1.5)
        vel = (side * sp * math.sin(ph), -side * sp * math.cos(ph))  # toward the path
        obs.append((c[0], c[1], 0.5, 0.5, 0.0, 2.0, vel[0], vel[1]))
    return _scenario(p, x0, path, 0.1, obs, seed=seed)


def jerk_model(c: dict, a0: float = 0.0, seed: int = 0) -> dict:
    """The scenario under the paper's jerk-input model (flag FLAG_JERK): the
    state gains the acceleration a (x0[7] = a0) and the inputs become
    (jerk, steer rate, progress rate), jerk bounded by +-2 m/s^3 (Sec. V);
    the nominal jerk is drawn small."""
    rng = np.random.default_rng(seed)
    p = dict(c["params"], flags=int(c["params"].get("flags", 0)) | FLAG_JERK,
             z_lo=(-2.0,) + tuple(c["params"]["z_lo"][1:]), z_hi=(2.0,) + tuple(c["params"]["z_hi"][1:]))
    out = dict(c)
    out["params"] = p
    out["x0"] = np.concatenate([np.asarray(c["x0"], np.float64)[:7], [a0]])
    U = np.array(c["U_nom"], np.float32)
    U[:, 0] = rng.uniform(-0.3, 0.3, size=U.shape[0]).astype(np.float32)
    out["U_nom"] = U
    return out

