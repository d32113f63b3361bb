#!/usr/bin/env python
"""Benchmark of the BR-MPPI solve on GB300.

Workload: the paper-scale closed loop -- S = 4096 rollouts, horizon H = 50,
Ts = 0.05 s, 8 random ellipses along a 38.7 m reverse-parking path (15 m
straight, 90 deg arc of R = 10 m, 8 m straight), tractor-trailer with
l1 = 4.0, lh = 0.5, l2 = 8.0 m.  One step = one control solve (all rollouts,
projection, costs, softmin, update, optimal trajectory, warm start).

* ``value``: rollout-steps/s = S * H * solves / device time, inputs resident
  in HBM, warm start produced on the device (ping-pong), counter = tick.
  Each step is bracketed by CUDA events on the launching stream; the L2 is
  flushed (256 MiB write) between steps outside the bracketed intervals.
* ``e2e``: the closed loop through the public host entry point
  ``brmppi_solve``: per tick the host buffers (state, nominal, obstacles,
  path) go to the device, U* and the optimal trajectory come back, the FP64
  host plant advances by U*[0] and the nominal is shifted.
* ``cpu_baseline``: the FP64 oracle on the host, single thread, on a bounded
  sample of the same solves.
* ``--impl reference``: the oracle as the reference arm (no reference code
  exists for this path), bounded samples of the same solve per step.

Several GPUs (torchrun): one process per GPU, each running the same
independent solves (different seeds) -- the path shards by instance and has
no data-path collective; the ranks only agree on the timed window.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "rollout-steps/s (S·H·solves/s) batched vs plain; p50/p99 solve latency"
UNIT = "rollout-steps/s"
L2_FLUSH_BYTES = 256 << 20


# ----------------------------------------------------------------------------
# Algorithmic work of one rollout-step, in FP32/INT32 lane operations for one
# sample on one lane (the Woodbury algorithm without the kernel's
# compensated sums and without team redundancy): every +, -, *, fma, min,
# max, compare/select, integer mul.lo / mul.hi / xor / add / shift / convert
# and every elementary function (sin, cos, tan, log, sqrt, exp, reciprocal)
# counts one; abs and negation are operand modifiers and count nothing.  The
# tally follows the formulation the kernel evaluates (parked ellipses in
# world axes through the staged quadratic form, shared per-step factors):
PHILOX_BLOCK_OPS = 124    # 10 rounds x (2 mul.lo, 2 mul.hi, 4 xor, 2 key adds) less the last round's
#                           dead key adds 98; 4 uniform maps x 3 (shift, or, subtract); 2 Box-Muller pairs x 7
#                           (log, -2 scale, sqrt, sin, cos, 2 products)
STEP_BASE_OPS = 115       # z_des 9, state trig 14, p_u 6, 2x2 solve 17, clip 6, Euler 14, path + cost 49
ROW_FACTOR_OPS = 12       # per-step factors shared by the ellipse rows (-2 Ts v, -Ts^2 v th1dot, -Ts^2 v^2 x
#                           (c1^2, 2 c1 s1, s1^2))
HITCH_OPS = 51            # row 27, projection terms 21, alpha update 3
OBSTACLE_OPS = 35         # offset 2, Q d 4, h 2, grad . e1 2, grad . n1 2, rest 5, a-column 1;
#                           projection terms 15 (floor, sign, alpha sample 3, p_alpha, b, r 2, reciprocal,
#                           u, rho, two sums, c); alpha update 2


def ops_per_rollout_step(n_obs: int, proj: bool = True) -> int:
    if not proj:
        return PHILOX_BLOCK_OPS + STEP_BASE_OPS - 6 - 17  # no p_u, no 2x2 solve
    P = (3 + 1 + n_obs + 3) // 4
    return (PHILOX_BLOCK_OPS * P + STEP_BASE_OPS + HITCH_OPS + OBSTACLE_OPS * n_obs +
            (ROW_FACTOR_OPS if n_obs > 0 else 0))


# Of those, the elementary functions the step evaluates on the XU (the
# special-function pipe, 16 lanes a clock per SM against 128 for FP32): per
# Philox block the reciprocals of the two Box-Muller logarithms' reductions
# and the two radii (reciprocal square root); per constraint row one
# reciprocal (1 / h~); per step the steer angle's tangent and the 2x2
# determinant (one reciprocal each).  The logarithms' series, Box-Muller's
# sin / cos of 2 pi u and the state angles' sin / cos are FP32 polynomials.
def xu_ops_per_rollout_step(n_obs: int, proj: bool = True) -> int:
    if not proj:
        return 4 + 1
    P = (3 + 1 + n_obs + 3) // 4
    return 4 * P + 2 + (1 + n_obs)


# ----------------------------------------------------------------------------
# Measured pipe peaks (issue-rate microbenchmarks, brmppi_measure_pipe): the
# roofline denominators of the ALU-bound kernels, measured on the device the
# bench runs on, with the clocks sampled while they run.
_PIPE_PEAKS = None


def pipe_peaks(local: int = 0):
    global _PIPE_PEAKS
    if _PIPE_PEAKS is not None:
        return _PIPE_PEAKS
    import torch
    import paper_2508_05773_gb300 as pkg
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.2)
    fma, t_fma = pkg.brmppi_measure_pipe(pkg.PIPE_FMA, 300000)
    imad, t_imad = pkg.brmppi_measure_pipe(pkg.PIPE_IMAD, 150000)
    xu, t_xu = pkg.brmppi_measure_pipe(pkg.PIPE_XU, 40000)
    clk = clocks.stop()
    _PIPE_PEAKS = {
        "fp32_fma_lane_ops_per_s": fma, "int_imad_lane_ops_per_s": imad, "xu_lane_ops_per_s": xu,
        "seconds": {"fma": t_fma, "imad": t_imad, "xu": t_xu}, "sms": sms, "clocks": clk,
        "how": "brmppi_measure_pipe: 4 CTAs x 512 threads per SM, 8 independent chains a thread of FFMA / "
               "IMAD / MUFU.RSQ; lane operations per second of the timed launch (CUDA events)",
    }
    return _PIPE_PEAKS


def alu_roofline(ops: float, xu_ops: float, seconds: float, kernel: str, kernel_mhz=None) -> dict:
    """Roofline of an ALU-bound launch against the measured peaks: every
    algorithmic lane operation takes an issue slot (peak = the FP32 FMA issue
    rate); the XU operations also against the XU pipe's own measured rate.
    If the kernel ran at a higher SM clock than the microbenchmark (which can
    meet the power cap), the peaks are scaled up to the kernel's clock (never
    down), so that the fraction is not flattered."""
    pk = pipe_peaks()
    fma, xu = pk["fp32_fma_lane_ops_per_s"], pk["xu_lane_ops_per_s"]
    peak_mhz = (pk.get("clocks") or {}).get("sm_mhz")
    scale = 1.0
    if kernel_mhz and peak_mhz and kernel_mhz > peak_mhz:
        scale = kernel_mhz / peak_mhz
    achieved = ops / seconds
    return {"bound": "alu", "achieved": achieved / 1e12, "peak": scale * fma / 1e12, "unit": "Tops/s (FP32 lane ops)",
            "frac": achieved / (scale * fma), "kernel": kernel, "ops_per_launch": ops,
            "peak_note": "of measured: FP32 FFMA issue-rate microbenchmark on this GPU "
                         f"({fma / 1e12:.2f} T lane-ops/s at a median {peak_mhz} MHz, {pk['sms']} SMs)"
                         + (f", scaled to the kernel's {kernel_mhz:.0f} MHz" if scale > 1.0 else ""),
            "xu": {"achieved": xu_ops / seconds / 1e12, "peak": scale * xu / 1e12,
                   "frac": xu_ops / seconds / (scale * xu), "ops_per_launch": xu_ops}}


# ----------------------------------------------------------------------------
def _dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def kernel_source_hash() -> str:
    """First 16 hex digits of the SHA-256 of the solve kernel's device code
    and launch logic (trig.cuh, rollout.cuh, then kernels.cu)."""
    import hashlib
    h = hashlib.sha256()
    for name in ("trig.cuh", "rollout.cuh", "kernels.cu"):
        with open(os.path.join(ROOT, "paper_2508_05773_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _traffic_for_current_kernel():
    """DRAM bytes per launch of the config-2 solve from the committed ncu
    capture, or None when the kernel source changed since that capture."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic_config2.json")) as f:
            rec = json.load(f)
        if kernel_source_hash() != rec["kernel_source_sha256_16"]:
            return None
        return int(rec["dram_read_bytes"]) + int(rec["dram_write_bytes"])
    except Exception:
        return None


def reduce_job(units: float, seconds: float, dist=None, device=None):
    """Whole-job throughput over the ranks of a weak-scaling run: the units
    every rank processed are summed and the time is the slowest rank's.
    Returns (units / second, total units, max seconds)."""
    if dist is None:
        return units / seconds, units, seconds
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / float(t.item()), float(u.item()), float(t.item())


def _measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
def _workload(rank: int):
    from paper_2508_05773_gb300 import scenarios as sc
    return sc.config2(seed=2 + 1000 * rank)


def _config_block(c, extra=None):
    p = c["params"]
    cfg = {
        "workload": "paper-scale closed-loop tick: S=4096 rollouts, H=50, Ts=0.05 s, "
                    "8 elliptical obstacles, 38.7 m reverse-parking path (ds=0.1 m)",
        "S": int(p["S"]), "H": int(p["H"]), "n_obstacles": int(c["obs"].shape[0]),
        "path_points": int(c["path"].shape[0]), "solves_per_step": 1,
        "l2": "flushed between steps (256 MiB write, outside the timed intervals)",
        "timing": "sum of per-step CUDA-event intervals on the launching stream",
    }
    if extra:
        cfg.update(extra)
    return cfg


def measure_batched(dev, reps: int = 10):
    """Uneven batch (256 instances: S in {1024..8192}, H in [30, 80], 0..16
    obstacles, random paths, seed 1): one persistent launch per batch
    replayed from a CUDA graph, against one plain launch per instance
    (brmppi_solve_device, back to back on one stream)."""
    import torch
    import paper_2508_05773_gb300 as pkg
    from paper_2508_05773_gb300 import scenarios as sc

    cases, insts = _config3_instances(dev)
    work = sum(int(c["params"]["S"]) * int(c["params"]["H"]) for c in cases)
    Smax = max(int(c["params"]["S"]) for c in cases)
    Hmax = max(int(c["params"]["H"]) for c in cases)
    npts = max(c["path"].shape[0] for c in cases)
    base = dict(cases[0]["params"], S=Smax, H=Hmax)
    solver = pkg.Solver(base, max_obstacles=16, max_path_pts=npts, max_batch=len(cases))
    stream = torch.cuda.current_stream(dev)
    solver.autotune_batch(insts, reps=2, stream=stream)
    batch_launch = solver.batch_launch()
    graph = solver.capture_batch(insts)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    times = []
    for r in range(reps + 2):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if pkg.brmppi_graph_launch(graph, stream) != 0:
            raise RuntimeError(pkg.brmppi_last_error(solver.ctx))
        e1.record(stream)
        torch.cuda.synchronize()
        if r >= 2:
            times.append(e0.elapsed_time(e1))
    assert all(int(d["status"].item()) == 0 for d in insts)
    pkg.brmppi_graph_destroy(graph)
    solver.close()
    batched_ms = float(np.median(times))

    # plain: one launch per instance, contexts per (S, H)
    ctxs = {}
    for c in cases:
        key = (int(c["params"]["S"]), int(c["params"]["H"]))
        if key not in ctxs:
            ctxs[key] = pkg.Solver(c["params"], max_obstacles=16, max_path_pts=npts)
    plain_times = []
    for r in range(max(3, reps // 2) + 1):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for c, d in zip(cases, insts):
            s = ctxs[(int(c["params"]["S"]), int(c["params"]["H"]))]
            rc = s.solve_device(d["x0"], d["U_nom"], d["obs"], d["path"], d["ds"], d["seed"], 0,
                                d["U_out"], d["traj_out"], None, d["U_next"], d["status"], stream)
            if rc != 0:
                raise RuntimeError(pkg.brmppi_last_error(s.ctx))
        e1.record(stream)
        torch.cuda.synchronize()
        if r >= 1:
            plain_times.append(e0.elapsed_time(e1))
    for s in ctxs.values():
        s.close()
    plain_ms = float(np.median(plain_times))
    ops = sum(int(c["params"]["S"]) * int(c["params"]["H"]) * ops_per_rollout_step(int(c["obs"].shape[0]))
              for c in cases)
    xu_ops = sum(int(c["params"]["S"]) * int(c["params"]["H"]) * xu_ops_per_rollout_step(int(c["obs"].shape[0]))
                 for c in cases)
    return {"workload": "256 uneven solves: S in {1024,2048,4096,8192}, H in [30,80], "
                        "0-16 ellipses, random straight+arc paths (seed 1)",
            "rollout_steps": work, "value": work / (batched_ms * 1e-3), "unit": UNIT,
            "ms_per_batch": batched_ms, "plain_value": work / (plain_ms * 1e-3),
            "plain_ms_per_batch": plain_ms, "speedup_vs_plain": plain_ms / batched_ms,
            "launches_per_batch": 1, "plain_launches_per_batch": len(cases), "launch": batch_launch,
            "roofline": alu_roofline(ops, xu_ops, batched_ms * 1e-3, "solve_kernel (persistent batch launch)"),
            "how": "CUDA-graph replay of one persistent launch vs brmppi_solve_device per "
                   "instance on one stream; L2 flushed between batches; median"}


def measure_stress(dev, reps: int = 5):
    """Config 5: S=65536, H=100, 64 ellipses in a 60x60 m lot, 120 m
    multi-arc path at ds=0.05 (2401 rows).  One solve with and without the
    stored-trajectory variant (every sample's states, S x (H+1) x 7 FP32 =
    185 MB); HBM GB/s of the stored variant against the measured copy peak."""
    import torch
    import paper_2508_05773_gb300 as pkg
    from paper_2508_05773_gb300 import scenarios as sc

    c = sc.config5()
    S, H = int(c["params"]["S"]), int(c["params"]["H"])
    n_obs = int(c["obs"].shape[0])
    t = lambda a, dt=torch.float32: torch.tensor(np.asarray(a), dtype=dt, device=dev)
    base = dict(x0=t(c["x0"], torch.float64), U_nom=t(c["U_nom"]), obs=t(c["obs"]), path=t(c["path"]),
                ds=c["ds"], S=S, seed=c["seed"], counter=0,
                U_out=torch.empty((H, 3), device=dev), traj_out=torch.empty((H + 1, 7), device=dev),
                status=torch.zeros(1, dtype=torch.int32, device=dev))
    states = torch.empty((S, H + 1, 7), device=dev)
    solver = pkg.Solver(c["params"], max_obstacles=n_obs, max_path_pts=c["path"].shape[0])
    stream = torch.cuda.current_stream(dev)
    solver.autotune(base["x0"], base["U_nom"], base["obs"], base["path"], c["ds"], reps=1,
                    stream=stream)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    res = {}
    for label, extra in (("plain", {}), ("stored", {"states_out": states})):
        inst = dict(base, **extra)
        ts = []
        for r in range(reps + 2):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            solver.solve_device_ex(inst, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            if r >= 2:
                ts.append(e0.elapsed_time(e1))
        res[label] = float(np.median(ts))
    assert int(base["status"].item()) == 0
    launch = solver.launch(n_obs)
    solver.close()
    peaks = _measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    ops = S * H * ops_per_rollout_step(n_obs)
    roof = alu_roofline(ops, S * H * xu_ops_per_rollout_step(n_obs), res["plain"] * 1e-3, "solve_kernel")
    state_bytes = S * (H + 1) * 7 * 4
    gbs = state_bytes / (res["stored"] * 1e-3) / 1e9
    return {"workload": "S=65536, H=100, 64 ellipses (60x60 m lot), 120 m multi-arc path, ds=0.05",
            "launch": launch, "ms_per_solve": res["plain"], "ms_per_solve_stored": res["stored"],
            "rollout_steps_per_s": S * H / (res["plain"] * 1e-3),
            "alu_frac": roof["frac"], "roofline": roof,
            "stored_bytes": state_bytes, "stored_hbm_gbs": gbs,
            "stored_hbm_frac": gbs / hbm,
            "note": "the stored variant writes 185 MB per solve at the solve's compute rate; "
                    "ALU-bound, so its HBM fraction is low by construction"}


def _time_solve(solver, inst, stream, flush, reps):
    import torch
    ts = []
    for r in range(reps + 3):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solver.solve_device_ex(inst, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if r >= 3:
            ts.append(e0.elapsed_time(e1))
    return float(np.median(ts))


def measure_variants(dev, reps: int = 20):
    """The comparison of Table I on GB300: standard MPPI, MPPI + collision
    cost and BR-MPPI on the same scene (8 obstacles), at the config-2 size
    (S=4096, H=50) and at the paper's own sampling (S=5000, H=120); plus
    BR-MPPI with the buffer cost and with third-order obstacle rows, the
    crossing scene (parked e = 4
    super-ellipses and moving pedestrians), and the hitch stabilizer (fused
    into a solve, and as a batched kernel over 2^20 states)."""
    import torch
    import paper_2508_05773_gb300 as pkg
    from paper_2508_05773_gb300 import scenarios as sc

    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    t = lambda a, dt=torch.float32: torch.tensor(np.asarray(a), dtype=dt, device=dev)
    out = {"table1_paper_ms": {"mppi": [3.20, 3.00], "mppi_collision": [13.0, 14.0],
                               "br_mppi": [9.92, 9.75],
                               "note": "forward / backward parking, S=5000, H=120, JAX, the "
                                       "paper's GPU; context, not a target"}}
    methods = (("br_mppi", 0), ("mppi", pkg.BRMPPI_FLAG_PROJ_NONE),
               ("mppi_collision", pkg.BRMPPI_FLAG_PROJ_NONE | pkg.BRMPPI_FLAG_COLLISION_COST),
               ("br_mppi_buffer", pkg.BRMPPI_FLAG_ALPHA_BUFFER),
               ("br_mppi_third_order", pkg.BRMPPI_FLAG_THIRD_ORDER))
    for size, (S, H) in (("config2", (4096, 50)), ("paper_table1", (5000, 120))):
        c = sc.config2(S=S, H=H)
        row = {}
        for name, flags in methods:
            p = dict(c["params"], flags=flags)
            solver = pkg.Solver(p, max_obstacles=16, max_path_pts=1024)
            inst = dict(x0=t(c["x0"], torch.float64), U_nom=t(c["U_nom"]), obs=t(c["obs"]),
                        path=t(c["path"]), ds=c["ds"], S=S, seed=c["seed"], counter=0,
                        U_out=torch.empty((H, 3), device=dev), traj_out=torch.empty((H + 1, 7), device=dev))
            solver.autotune(inst["x0"], inst["U_nom"], inst["obs"], inst["path"], c["ds"], reps=2,
                            stream=stream)
            ms = _time_solve(solver, inst, stream, flush, reps)
            row[name] = {"ms_per_solve": ms, "rollout_steps_per_s": S * H / (ms * 1e-3),
                         "launch": solver.launch(8)}
            if name == "br_mppi":
                inst_s = dict(inst, u_safe_out=torch.empty(4, device=dev))
                row["br_mppi_with_stabilizer"] = {"ms_per_solve": _time_solve(solver, inst_s, stream, flush,
                                                                               reps)}
            solver.close()
        # the paper's jerk-input model (third-order obstacle rows bring the
        # inputs in; x0 gains the acceleration)
        cj = sc.jerk_model(c)
        pj = dict(cj["params"], flags=int(cj["params"]["flags"]) | pkg.BRMPPI_FLAG_THIRD_ORDER)
        solver = pkg.Solver(pj, max_obstacles=16, max_path_pts=1024)
        inst = dict(x0=t(cj["x0"], torch.float64), U_nom=t(cj["U_nom"]), obs=t(cj["obs"]), path=t(cj["path"]),
                    ds=cj["ds"], S=S, seed=cj["seed"], counter=0, U_out=torch.empty((H, 3), device=dev),
                    traj_out=torch.empty((H + 1, 7), device=dev))
        solver.autotune(inst["x0"], inst["U_nom"], inst["obs"], inst["path"], cj["ds"], reps=2, stream=stream)
        ms = _time_solve(solver, inst, stream, flush, reps)
        row["br_mppi_jerk_model_third_order"] = {"ms_per_solve": ms, "rollout_steps_per_s": S * H / (ms * 1e-3),
                                                 "launch": solver.launch(8)}
        solver.close()
        out[size] = dict(row, S=S, H=H, n_obs=8)
    # crossing scene: 6 parked e = 4 super-ellipses, 2 crossing pedestrians
    c = sc.crossing()
    S, H = int(c["params"]["S"]), int(c["params"]["H"])
    solver = pkg.Solver(c["params"], max_obstacles=16, max_path_pts=1024)
    inst = dict(x0=t(c["x0"], torch.float64), U_nom=t(c["U_nom"]), obs=t(c["obs"]), path=t(c["path"]),
                ds=c["ds"], S=S, seed=c["seed"], counter=0, U_out=torch.empty((H, 3), device=dev))
    solver.autotune(inst["x0"], inst["U_nom"], inst["obs"], inst["path"], c["ds"], reps=2, stream=stream)
    ms = _time_solve(solver, inst, stream, flush, reps)
    out["crossing"] = {"workload": "S=4096, H=50, 6 parked e=4 super-ellipses + 2 pedestrians crossing "
                                   "at 1-1.5 m/s (8-float obstacle rows)",
                       "ms_per_solve": ms, "rollout_steps_per_s": S * H / (ms * 1e-3),
                       "launch": solver.launch(8)}
    solver.close()
    # the same scene seen from a five-disc tractor-trailer footprint (40 rows)
    solver = pkg.Solver(dict(c["params"], **sc.FIVE_DISCS), max_obstacles=16, max_path_pts=1024)
    solver.autotune(inst["x0"], inst["U_nom"], inst["obs"], inst["path"], c["ds"], reps=2, stream=stream)
    ms = _time_solve(solver, inst, stream, flush, reps)
    out["crossing_five_discs"] = {"workload": "the crossing scene, footprint of 3 tractor + 2 trailer discs "
                                              "(8 obstacles x 5 discs = 40 barrier rows)",
                                  "ms_per_solve": ms, "rollout_steps_per_s": S * H / (ms * 1e-3),
                                  "launch": solver.launch(8)}
    # batched stabilizer: 2^23 states (0.7 GB, larger than L2; a kernel of
    # ~0.1 ms, so launch latency does not dominate the interval)
    n = 1 << 23
    rng = np.random.default_rng(3)
    th1 = rng.uniform(-3, 3, n)
    X = np.stack([rng.uniform(-50, 50, n), rng.uniform(-50, 50, n), th1, th1 + rng.uniform(-1.0, 1.0, n),
                  rng.uniform(-2, 2, n), rng.uniform(-0.5, 0.5, n), rng.uniform(0, 30, n)], 1)
    Ur = np.stack([rng.uniform(-3, 3, n), rng.uniform(-1, 1, n), rng.uniform(0, 3, n)], 1)
    xd, ud = t(X, torch.float64), t(Ur)
    od = torch.empty((n, 4), device=dev)
    ts = []
    for r in range(reps + 3):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solver.hitch_stabilize_device(xd, ud, od, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if r >= 3:
            ts.append(e0.elapsed_time(e1))
    ms = float(np.median(ts))
    solver.close()
    peaks = _measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    nbytes = n * (7 * 8 + 3 * 4 + 4 * 4)
    out["stabilizer_batched"] = {"states": n, "ms": ms, "states_per_s": n / (ms * 1e-3),
                                 "bytes": nbytes, "hbm_gbs": nbytes / (ms * 1e-3) / 1e9,
                                 "hbm_frac": nbytes / (ms * 1e-3) / 1e9 / hbm}
    return out


def _config3_instances(dev):
    import torch
    from paper_2508_05773_gb300 import scenarios as sc
    cases = sc.config3()
    t = lambda a, dt=torch.float32: torch.tensor(np.asarray(a), dtype=dt, device=dev)
    insts = []
    for c in cases:
        H, S = int(c["params"]["H"]), int(c["params"]["S"])
        insts.append(dict(x0=t(c["x0"], torch.float64), U_nom=t(c["U_nom"]),
                          obs=t(c["obs"]) if c["obs"].shape[0] else None, path=t(c["path"]),
                          ds=c["ds"], S=S, seed=c["seed"], counter=0,
                          U_out=torch.empty((H, 3), device=dev),
                          traj_out=torch.empty((H + 1, 7), device=dev),
                          U_next=torch.empty((H, 3), device=dev),
                          status=torch.zeros(1, dtype=torch.int32, device=dev)))
    return cases, insts


def run_profile(args):
    """A few launches of one workload for ncu (no timing): `solve` = the
    config-2 solve (S=4096, H=50, 8 ellipses), `batch` = the config-3 batch
    (256 uneven instances, one persistent launch), each with a fixed launch
    shape (--tps / --threads; defaults: the shapes the autotuners pick on
    GB300), `stress` / `stress_stored` = the config-5 solve (S=65536, H=100,
    64 ellipses) without / with every sample's states stored (185 MB),
    `stabilizer` = the batched hitch stabilizer on 2^20 states.  Four
    launches with an L2 flush before each; capture the last."""
    import torch
    import paper_2508_05773_gb300 as pkg
    from paper_2508_05773_gb300 import scenarios as sc
    dev = torch.device("cuda", 0)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    t = lambda a, dt=torch.float32: torch.tensor(np.asarray(a), dtype=dt, device=dev)
    if args.profile == "solve":
        c = sc.config2()
        H = int(c["params"]["H"])
        solver = pkg.Solver(c["params"], max_obstacles=16, max_path_pts=1024,
                            threads_per_sample=args.tps or 4, block_threads=args.threads or 128)
        x0, U, obs, path = t(c["x0"], torch.float64), t(c["U_nom"]), t(c["obs"]), t(c["path"])
        Uo, tr = torch.empty((H, 3), device=dev), torch.empty((H + 1, 7), device=dev)
        for r in range(4):
            flush.zero_()
            if solver.solve_device(x0, U, obs, path, c["ds"], c["seed"], r, Uo, tr) != 0:
                raise RuntimeError(pkg.brmppi_last_error(solver.ctx))
    elif args.profile == "stabilizer":
        n = 1 << 20
        rng = np.random.default_rng(3)
        th1 = rng.uniform(-3, 3, n)
        X = np.stack([rng.uniform(-50, 50, n), rng.uniform(-50, 50, n), th1, th1 + rng.uniform(-1.0, 1.0, n),
                      rng.uniform(-2, 2, n), rng.uniform(-0.5, 0.5, n), rng.uniform(0, 30, n)], 1)
        Ur = np.stack([rng.uniform(-3, 3, n), rng.uniform(-1, 1, n), rng.uniform(0, 3, n)], 1)
        xd, ud = t(X, torch.float64), t(Ur)
        od = torch.empty((n, 4), device=dev)
        solver = pkg.Solver(sc.config2()["params"], max_obstacles=16, max_path_pts=1024)
        stream = torch.cuda.current_stream(dev)
        for r in range(4):
            flush.zero_()
            solver.hitch_stabilize_device(xd, ud, od, stream)
        torch.cuda.synchronize()
    elif args.profile in ("stress", "stress_stored"):
        c = sc.config5()
        S, H = int(c["params"]["S"]), int(c["params"]["H"])
        n_obs = int(c["obs"].shape[0])
        solver = pkg.Solver(c["params"], max_obstacles=n_obs, max_path_pts=c["path"].shape[0],
                            threads_per_sample=args.tps or 4, block_threads=args.threads or 256)
        inst = dict(x0=t(c["x0"], torch.float64), U_nom=t(c["U_nom"]), obs=t(c["obs"]), path=t(c["path"]),
                    ds=c["ds"], S=S, seed=c["seed"], counter=0,
                    U_out=torch.empty((H, 3), device=dev), traj_out=torch.empty((H + 1, 7), device=dev),
                    status=torch.zeros(1, dtype=torch.int32, device=dev))
        if args.profile == "stress_stored":
            inst["states_out"] = torch.empty((S, H + 1, 7), device=dev)
        stream = torch.cuda.current_stream(dev)
        for r in range(4):
            flush.zero_()
            solver.solve_device_ex(dict(inst, counter=r), stream)
        torch.cuda.synchronize()
        if int(inst["status"].item()) != 0:
            raise RuntimeError("config-5 solve failed")
    else:
        cases, insts = _config3_instances(dev)
        Smax = max(int(c["params"]["S"]) for c in cases)
        Hmax = max(int(c["params"]["H"]) for c in cases)
        npts = max(c["path"].shape[0] for c in cases)
        solver = pkg.Solver(dict(cases[0]["params"], S=Smax, H=Hmax), max_obstacles=16, max_path_pts=npts,
                            max_batch=len(cases), batch_threads_per_sample=args.tps or 1,
                            batch_block_threads=args.threads or 256)
        for r in range(4):
            flush.zero_()
            solver.solve_batch(insts)
    torch.cuda.synchronize()
    solver.close()
    print(json.dumps({"profile": args.profile, "launches": 4}), flush=True)
    return 0


def measure_serving(rates=(2000, 10000, 50000, 80000, 100000, 200000), duration=2.0, warm=0.5, n_vehicles=512, seed=4,
                    block_threads=0):
    """Serving loop: Poisson arrivals from 512 vehicles (S=4096, H=50, 0-16
    ellipses per request, fresh state = the vehicle's start + N(0, 0.05)
    jitter), admitted into batches as lanes free up.  Latency is submit ->
    result ready (measured by the library), against the 10 ms deadline.
    Served throughput counts the solves completed from the first measured
    arrival to the last measured completion (past saturation the queue
    grows and the served rate stays below the offered one).  A last pass
    keeps `saturate` requests outstanding at all times: the loop's ceiling."""
    import ctypes
    import paper_2508_05773_gb300 as pkg
    from paper_2508_05773_gb300 import scenarios as sc
    from paper_2508_05773_gb300 import _native as nat

    rng = np.random.default_rng(seed)
    S, H = 4096, 50
    fleet = [sc.random_instance(rng, S_choices=(S,), H_range=(H, H), obs_range=(0, 16))
             for _ in range(n_vehicles)]
    npts = max(c["path"].shape[0] for c in fleet)
    srv = pkg.Solver(sc.params(S=S, H=H), max_obstacles=16, max_path_pts=npts,
                     max_vehicles=n_vehicles, serve_lanes=3, serve_max_batch=128, serve_queue=8192,
                     batch_block_threads=block_threads)
    for v, c in enumerate(fleet):
        srv.register(v, c["path"], c["ds"], None, c["seed"])
    lib = nat.load()
    ctx = srv.ctx
    Dp = ctypes.POINTER(ctypes.c_double)
    Fp = ctypes.POINTER(ctypes.c_float)
    pool = []
    for v in range(n_vehicles):
        o = fleet[v]["obs"]
        pool.append(np.ascontiguousarray(o.reshape(-1), dtype=np.float32) if o.shape[0] else None)
    U = np.empty((H, 3), np.float32)
    Uptr = U.ctypes.data_as(Fp)
    lat = ctypes.c_double()
    tk = ctypes.c_uint64()

    def run(n_req, arrival, saturate=0):
        vids = rng.integers(0, n_vehicles, size=n_req).astype(np.uint32)
        X = np.stack([fleet[v]["x0"] for v in vids]).astype(np.float64)
        X[:, :3] += rng.normal(0.0, 0.05, size=(n_req, 3))
        X = np.ascontiguousarray(X)
        nobs = np.array([0 if pool[v] is None else pool[v].size // 6 for v in vids], dtype=np.int32)
        xptr = [X[i].ctypes.data_as(Dp) for i in range(n_req)]
        optr = [None if pool[v] is None else pool[v].ctypes.data_as(Fp) for v in vids]
        pending, head, busy = [], 0, 0
        lats, t_sub, t_done = [], [], []
        t0 = time.perf_counter()
        i = 0
        while i < n_req or head < len(pending):
            now = time.perf_counter() - t0
            while i < n_req and (arrival[i] <= now if not saturate else len(pending) - head < saturate):
                st = lib.brmppi_submit(ctx, int(vids[i]), xptr[i], optr[i], int(nobs[i]), ctypes.byref(tk))
                if st == -7:  # EBUSY: retry on the next pass
                    busy += 1
                    break
                if st != 0:
                    raise RuntimeError(f"submit failed: {st}")
                pending.append((tk.value, i, time.perf_counter() - t0))
                i += 1
            while head < len(pending):
                st = lib.brmppi_poll(ctx, pending[head][0], Uptr, None, ctypes.byref(lat))
                if st == -3:
                    break
                if st != 0:
                    raise RuntimeError(f"served solve failed: {st}")
                if pending[head][2] >= warm:
                    lats.append(lat.value)
                    t_sub.append(pending[head][2])
                    t_done.append(time.perf_counter() - t0)
                head += 1
        span = max(t_done) - min(t_sub) if t_done else float("nan")
        lats = np.array(lats) * 1e3
        return lats, span, busy, time.perf_counter() - t0

    results = []
    for rate in rates:
        n_req = int(rate * (warm + duration))
        arr = np.cumsum(rng.exponential(1.0 / rate, size=n_req))
        lats, span, busy, el = run(n_req, arr)
        results.append({
            "target_rate": rate, "offered_rate": n_req / arr[-1],
            "solves_measured": int(lats.size),
            "served_rollout_steps_per_s": lats.size * S * H / span,
            "p50_ms": float(np.percentile(lats, 50)), "p99_ms": float(np.percentile(lats, 99)),
            "p999_ms": float(np.percentile(lats, 99.9)), "deadline_ms": 10.0,
            "deadline_misses": int(np.sum(lats > 10.0)), "ebusy_retries": busy, "wall_s": el})
    saturate = 4096
    n_req = 200000
    lats, span, busy, el = run(n_req, None, saturate=saturate)
    sat = {"outstanding": saturate, "solves_measured": int(lats.size),
           "served_rollout_steps_per_s": lats.size * S * H / span, "served_solves_per_s": lats.size / span,
           "p50_ms": float(np.percentile(lats, 50)), "p99_ms": float(np.percentile(lats, 99)),
           "deadline_misses": int(np.sum(lats > 10.0)), "wall_s": el}
    stats = srv.server_stats()
    launch = pkg.brmppi_get_batch_launch(srv.ctx)
    srv.close()
    return {"workload": "512 vehicles, Poisson arrivals, S=4096, H=50, 0-16 ellipses per request",
            "lanes": stats["lanes"], "max_batch": stats["max_batch"], "launch": launch,
            "max_inflight_batches": stats["max_inflight_batches"],
            "mean_batch": stats["solves_in_batches"] / max(1, stats["batches"]),
            "rates": results, "saturated": sat}


_WORKER_CASE = None


def _oracle_worker(task):
    """One worker process of the CPU baseline: FP64 oracle solves of the
    config-2 workload (S_run rollouts each, counters from `first` on) until
    `budget_s` has passed (at least `min_solves`).  Returns (solves, seconds)."""
    S_run, first, budget_s, min_solves = task
    import oracle
    global _WORKER_CASE
    if _WORKER_CASE is None:
        from paper_2508_05773_gb300 import scenarios as sc
        c = sc.config2()
        _WORKER_CASE = c, sc.as_float32(c["params"])
    c, p = _WORKER_CASE
    t0 = time.perf_counter()
    n = 0
    while n < min_solves or time.perf_counter() - t0 < budget_s:
        oracle.solve(p, c["x0"], c["U_nom"], c["obs"], c["path"], c["ds"], c["seed"], first + n, S=S_run,
                     want_J=False)
        n += 1
    return n, time.perf_counter() - t0


def _oracle_pool():
    """Worker processes on every host core (spawned: a forked child of a
    CUDA process can hang), imports done before any timing."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    pool = mp.get_context("spawn").Pool(cores)
    pool.map(_oracle_worker, [(1, 10 ** 6 + i, 0.0, 1) for i in range(cores)])
    return pool, cores


def _cpu_model():
    """The host CPU's model name (x86: `model name`; Arm: implementer/part)."""
    import platform
    try:
        info = open("/proc/cpuinfo").read().splitlines()
    except OSError:
        return platform.machine()
    for key in ("model name", "Model"):
        for ln in info:
            if ln.startswith(key) and ":" in ln:
                return ln.split(":", 1)[1].strip()
    part = [ln.split(":", 1)[1].strip() for ln in info if ln.startswith(("CPU implementer", "CPU part"))]
    return f"{platform.machine()} (implementer/part {'/'.join(part[:2])})" if part else platform.machine()


def run_cpu_baseline(budget_s: float = 12.0):
    """The FP64 oracle on the host cores, full config-2 solves: first one
    process alone (about a third of budget_s), then one process per core
    (independent solves, different noise counters) for the rest;
    rollout-steps per wall second of all cores, the single core beside it."""
    from paper_2508_05773_gb300 import scenarios as sc
    p = sc.config2()["params"]
    S, H = int(p["S"]), int(p["H"])
    pool, cores = _oracle_pool()
    try:
        n1, el1 = pool.apply(_oracle_worker, ((S, 5 * 10 ** 6, budget_s / 3.0, 1),))
        t0 = time.perf_counter()
        res = pool.map(_oracle_worker, [(S, 1000 * w, 2.0 * budget_s / 3.0, 1) for w in range(cores)])
        el = time.perf_counter() - t0
    finally:
        pool.close()
        pool.join()
    n = sum(r[0] for r in res)
    return {"value": n * S * H / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "single_core_value": n1 * S * H / el1, "cpu": _cpu_model(),
            "sample": f"{n} full solves (S={S}, H={H}, 8 obstacles) of the same workload on {cores} "
                      f"processes (one per core), FP64, {el:.1f} s; single core: {n1} solves in {el1:.1f} s"}


def run_reference(args, world, rank):
    """Reference arm: the oracle as it stands, on every host core; each
    step is a bounded sample of the workload (512 of the 4096 rollouts of a
    solve per core, one process per core, different noise counters)."""
    if rank != 0:
        return 0
    from paper_2508_05773_gb300 import scenarios as sc
    c = sc.config2()
    p = c["params"]
    S_sample, H = 512, int(p["H"])
    pool, cores = _oracle_pool()
    try:
        for i in range(args.warmup):
            pool.map(_oracle_worker, [(S_sample, 10 ** 5 * i + w, 0.0, 1) for w in range(cores)])
        t0 = time.perf_counter()
        for i in range(args.steps):
            pool.map(_oracle_worker, [(S_sample, 10 ** 7 + 10 ** 5 * i + w, 0.0, 1) for w in range(cores)])
        el = time.perf_counter() - t0
    finally:
        pool.close()
        pool.join()
    value = args.steps * cores * S_sample * H / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": _config_block(c, {"rollouts_per_step": cores * S_sample,
                                                       "solves_per_step": cores * S_sample / int(p["S"]),
                                                       "l2": "not applicable (host cores)",
                                                       "timing": "host wall clock over the timed steps"}),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{S_sample} of the {int(p['S'])} rollouts of a solve on each of {cores} "
                                   "processes (one per core) per step, FP64 oracle"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, world, rank, local):
    import torch
    import paper_2508_05773_gb300 as pkg
    from paper_2508_05773_gb300 import plant

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    c = _workload(rank)
    p = c["params"]
    S, H = int(p["S"]), int(p["H"])
    n_obs = int(c["obs"].shape[0])
    pinned = args.tps > 0 and args.threads > 0  # a fixed launch shape in place of the autotuner's pick
    shape = dict(threads_per_sample=args.tps, block_threads=args.threads) if pinned else {}
    solver = pkg.Solver(p, device=local, max_obstacles=max(16, n_obs), max_path_pts=1024, **shape)

    # ---------------- device-resident inputs
    x0 = torch.tensor(c["x0"], dtype=torch.float64, device=dev)
    Ubuf = [torch.tensor(c["U_nom"], device=dev), torch.empty((H, 3), device=dev)]
    obs = torch.tensor(c["obs"], device=dev)
    path = torch.tensor(c["path"], device=dev)
    U_out = torch.empty((H, 3), device=dev)
    traj = torch.empty((H + 1, 7), device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    if rank == 0:
        pipe_peaks(local)  # the roofline denominators, measured before anything is timed
    if not pinned:
        solver.autotune(x0, Ubuf[0], obs, path, c["ds"], reps=3, stream=stream)

    def solve(tick: int):
        rc = solver.solve_device(x0, Ubuf[tick % 2], obs, path, c["ds"], c["seed"], tick, U_out,
                                 traj, None, Ubuf[(tick + 1) % 2], status, stream)
        if rc != 0:
            raise RuntimeError(pkg.brmppi_last_error(solver.ctx))

    for i in range(args.warmup):
        flush.zero_()
        solve(i)
    torch.cuda.synchronize()
    assert int(status.item()) == 0

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local) if rank == 0 else None
    if clocks:
        clocks.start()
        time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.zero_()
        starts[i].record(stream)
        solve(args.warmup + i)
        ends[i].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop() if clocks else None
    per = [s.elapsed_time(e) for s, e in zip(starts, ends)]  # ms
    value, _, total_s = reduce_job(args.steps * S * H, float(sum(per)) * 1e-3, dist, dev)
    total_ms = total_s * 1e3
    lat = np.array(per)

    # ---------------- end to end: closed loop through the host entry point
    e2e = None
    e2e_lat = None
    h2d, d2h = solver.transfer_bytes(n_obs, int(c["path"].shape[0]))
    x = np.array(c["x0"], dtype=np.float64)
    Unom = np.array(c["U_nom"], dtype=np.float32)
    for i in range(args.warmup):
        out = solver.solve(x, Unom, c["obs"], c["path"], c["ds"], c["seed"], i)
    x = np.array(c["x0"], dtype=np.float64)
    Unom = np.array(c["U_nom"], dtype=np.float32)
    if dist:
        dist.barrier()
    tick_s = []
    t0 = time.perf_counter()
    for i in range(args.steps):
        ts = time.perf_counter()
        out = solver.solve(x, Unom, c["obs"], c["path"], c["ds"], c["seed"], i)
        x = plant.step(p, x, out["U"][0])
        Unom = plant.shift(out["U"])
        tick_s.append(time.perf_counter() - ts)
    el = time.perf_counter() - t0
    e2e_value, _, el = reduce_job(args.steps * S * H, el, dist, dev)
    e2e = {"value": e2e_value, "unit": UNIT,
           "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
           "p50_ms": 1e3 * float(np.percentile(tick_s, 50)),
           "p99_ms": 1e3 * float(np.percentile(tick_s, 99)),
           "what": "closed loop: brmppi_solve on host buffers + FP64 host plant + shift"}

    if rank == 0:
        ops = S * H * ops_per_rollout_step(n_obs)
        kernel_s = total_ms * 1e-3 / args.steps
        roof = alu_roofline(ops, S * H * xu_ops_per_rollout_step(n_obs), kernel_s, "solve_kernel",
                            kernel_mhz=(clk or {}).get("sm_mhz"))
        roof["ops_per_rollout_step"] = ops_per_rollout_step(n_obs)
        roof["traffic"] = _traffic_for_current_kernel()
        launch = solver.launch(n_obs)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": _config_block(c, {"launch": launch}),
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "p999": float(np.percentile(lat, 99.9)), "deadline": 10.0,
                           "misses": int(np.sum(lat > 10.0))},
            "roofline": roof,
            "pipe_peaks": pipe_peaks(local),
            "e2e": e2e,
            "gpu_launches": args.steps,
            "clocks": clk,
        }
        if world == 1 and not args.no_batched:
            line["batched"] = measure_batched(dev)
        if world == 1 and not args.no_serving:
            line["serving"] = measure_serving()
        if world == 1 and not args.no_stress:
            line["stress"] = measure_stress(dev)
        if world == 1 and not args.no_variants:
            line["variants"] = measure_variants(dev)
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = run_cpu_baseline()
        print(json.dumps(line), flush=True)
    solver.close()
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-stress", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--profile", choices=("solve", "batch", "stress", "stress_stored", "stabilizer"), default=None,
                    help="a few launches of one workload for ncu, no timing")
    ap.add_argument("--tps", type=int, default=0,
                    help="threads per sample of the timed solve (with --threads: no autotuning; --profile too)")
    ap.add_argument("--threads", type=int, default=0,
                    help="threads per block of the timed solve (with --tps: no autotuning; --profile too)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world, rank, local = _dist_env()
    if args.profile:
        return run_profile(args)
    if args.impl == "reference":
        return run_reference(args, world, rank)
    return run_ours(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
