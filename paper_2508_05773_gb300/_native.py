"""ctypes binding of libbrmppi.so (include/brmppi.h): argument marshalling
only.  Every step of a solve runs in the library's CUDA kernels; there is no
Python or CPU fallback, and a missing library is an error."""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbrmppi.so")

BRMPPI_ABI_VERSION = 7
BRMPPI_OK = 0
BRMPPI_EINVAL = -1
BRMPPI_ENOMEM = -2
BRMPPI_EAGAIN = -3
BRMPPI_ETIMEDOUT = -4
BRMPPI_ENONFINITE = -5
BRMPPI_ECUDA = -6
BRMPPI_EBUSY = -7
BRMPPI_FLAG_PROJ_NONE = 0x1
BRMPPI_FLAG_COLLISION_COST = 0x2
BRMPPI_FLAG_OBS8 = 0x4
BRMPPI_FLAG_ALPHA_BUFFER = 0x8
BRMPPI_FLAG_THIRD_ORDER = 0x10
BRMPPI_FLAG_JERK_MODEL = 0x20

STATUS_NAMES = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "EAGAIN", -4: "ETIMEDOUT",
                -5: "ENONFINITE", -6: "ECUDA", -7: "EBUSY"}

#: every exported symbol the header declares
EXPORTS = (
    "brmppi_default_params", "brmppi_create", "brmppi_destroy", "brmppi_last_error",
    "brmppi_solve", "brmppi_solve_device", "brmppi_solve_device_ex", "brmppi_solve_batch", "brmppi_batch_capture",
    "brmppi_graph_launch", "brmppi_graph_destroy", "brmppi_autotune", "brmppi_autotune_batch",
    "brmppi_get_launch", "brmppi_transfer_bytes", "brmppi_vehicle_register", "brmppi_submit",
    "brmppi_poll", "brmppi_vehicle_export", "brmppi_vehicle_import", "brmppi_server_stats_get",
    "brmppi_solve_device_noalloc", "brmppi_hitch_stabilize_device", "brmppi_get_batch_launch",
    "brmppi_noise_blocks", "brmppi_measure_pipe", "brmppi_inject_alloc_failure",
    "brmppi_tile_layout", "brmppi_solve_tiles", "brmppi_merge_tiles",
)


class brmppi_params(ctypes.Structure):
    _fields_ = [
        ("abi_version", ctypes.c_uint32),
        ("S", ctypes.c_int32), ("H", ctypes.c_int32),
        ("max_obstacles", ctypes.c_int32), ("max_path_pts", ctypes.c_int32),
        ("flags", ctypes.c_int32), ("threads_per_sample", ctypes.c_int32),
        ("block_threads", ctypes.c_int32), ("max_batch", ctypes.c_int32),
        ("batch_threads_per_sample", ctypes.c_int32), ("batch_block_threads", ctypes.c_int32),
        ("max_vehicles", ctypes.c_int32), ("serve_lanes", ctypes.c_int32),
        ("serve_max_batch", ctypes.c_int32), ("serve_queue", ctypes.c_int32),
        ("wait_timeout_ms", ctypes.c_int32),
        ("Ts", ctypes.c_float), ("lambda_", ctypes.c_float),
        ("l1", ctypes.c_float), ("lh", ctypes.c_float), ("l2", ctypes.c_float),
        ("dtheta_max", ctypes.c_float), ("kappa", ctypes.c_float), ("r_inflate", ctypes.c_float),
        ("Qc", ctypes.c_float), ("Ql", ctypes.c_float), ("Qth", ctypes.c_float),
        ("R", ctypes.c_float * 3), ("mu", ctypes.c_float), ("nu_bar", ctypes.c_float),
        ("z_lo", ctypes.c_float * 3), ("z_hi", ctypes.c_float * 3), ("sigma", ctypes.c_float * 3),
        ("alpha0", ctypes.c_float), ("sigma_alpha", ctypes.c_float),
        ("ua_lo", ctypes.c_float), ("ua_hi", ctypes.c_float),
        ("w_u", ctypes.c_float * 3), ("w_alpha", ctypes.c_float),
        ("rho", ctypes.c_float), ("h_floor", ctypes.c_float),
        ("q_coll", ctypes.c_float), ("alpha_stab", ctypes.c_float),
        ("q_stab", ctypes.c_float * 2), ("q_abuf", ctypes.c_float), ("h_buf", ctypes.c_float),
        ("n_discs", ctypes.c_int32), ("disc_trailer_mask", ctypes.c_int32),
        ("disc_off", ctypes.c_float * 8),
    ]


class brmppi_instance(ctypes.Structure):
    _fields_ = [
        ("x0", ctypes.c_void_p), ("U_nom", ctypes.c_void_p), ("obs", ctypes.c_void_p),
        ("path", ctypes.c_void_p), ("n_obs", ctypes.c_int32), ("n_pts", ctypes.c_int32),
        ("ds", ctypes.c_float), ("S", ctypes.c_int32), ("H", ctypes.c_int32),
        ("seed", ctypes.c_uint64), ("counter", ctypes.c_uint64),
        ("U_out", ctypes.c_void_p), ("traj_out", ctypes.c_void_p), ("J_out", ctypes.c_void_p),
        ("U_next", ctypes.c_void_p), ("status", ctypes.c_void_p),
        ("states_out", ctypes.c_void_p), ("u_safe_out", ctypes.c_void_p),
        ("inputs_out", ctypes.c_void_p), ("J_lo_out", ctypes.c_void_p),
    ]


class brmppi_server_stats(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
        ("batches", ctypes.c_uint64), ("solves_in_batches", ctypes.c_uint64),
        ("request_slots", ctypes.c_int32), ("lanes", ctypes.c_int32),
        ("max_inflight_batches", ctypes.c_int32), ("max_batch", ctypes.c_int32),
    ]


_lock = threading.Lock()
_lib = None

_F = ctypes.POINTER(ctypes.c_float)
_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_VP = ctypes.c_void_p


class NativeLibraryMissing(RuntimeError):
    pass


def load() -> ctypes.CDLL:
    """Load libbrmppi.so (built by ``__graft_entry__.build()``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise NativeLibraryMissing(
                f"{LIB_PATH} is missing: build the CUDA library first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER(brmppi_params)
        sig = {
            "brmppi_default_params": (None, [P]),
            "brmppi_create": (ctypes.c_int, [P, ctypes.c_int, ctypes.POINTER(_VP)]),
            "brmppi_destroy": (ctypes.c_int, [_VP]),
            "brmppi_inject_alloc_failure": (None, [ctypes.c_int32]),
            "brmppi_tile_layout": (ctypes.c_int, [_VP, ctypes.POINTER(brmppi_instance),
                                                  ctypes.POINTER(ctypes.c_int32),
                                                  ctypes.POINTER(ctypes.c_int32)]),
            "brmppi_solve_tiles": (ctypes.c_int, [_VP, ctypes.POINTER(brmppi_instance), ctypes.c_int32,
                                                  ctypes.c_int32, _VP, _VP]),
            "brmppi_merge_tiles": (ctypes.c_int, [_VP, ctypes.POINTER(brmppi_instance), _VP,
                                                  ctypes.c_int32, _VP]),
            "brmppi_last_error": (ctypes.c_char_p, [_VP]),
            # pointers as plain addresses: the host entry point is the
            # closed loop's per-tick call, and typed pointer objects cost
            # microseconds each
            "brmppi_solve": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int32, _VP, ctypes.c_int32,
                                            ctypes.c_float, ctypes.c_uint64, ctypes.c_uint64, _VP, _VP,
                                            _VP]),
            "brmppi_solve_device": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int32, _VP,
                                                   ctypes.c_int32, ctypes.c_float, ctypes.c_uint64,
                                                   ctypes.c_uint64, _VP, _VP, _VP, _VP, _VP, _VP]),
            "brmppi_solve_device_ex": (ctypes.c_int, [_VP, ctypes.POINTER(brmppi_instance), _VP]),
            "brmppi_solve_batch": (ctypes.c_int, [_VP, ctypes.POINTER(brmppi_instance),
                                                  ctypes.c_int32, _VP]),
            "brmppi_batch_capture": (ctypes.c_int, [_VP, ctypes.POINTER(brmppi_instance),
                                                    ctypes.c_int32, ctypes.POINTER(_VP)]),
            "brmppi_graph_launch": (ctypes.c_int, [_VP, _VP]),
            "brmppi_graph_destroy": (None, [_VP]),
            "brmppi_autotune": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int32, _VP,
                                               ctypes.c_int32, ctypes.c_float, ctypes.c_int32, _VP]),
            "brmppi_autotune_batch": (ctypes.c_int, [_VP, ctypes.POINTER(brmppi_instance),
                                                     ctypes.c_int32, ctypes.c_int32, _VP]),
            "brmppi_get_launch": (ctypes.c_int, [_VP, ctypes.c_int32, _I32, _I32, _I32]),
            "brmppi_get_batch_launch": (ctypes.c_int, [_VP, _I32, _I32]),
            "brmppi_vehicle_register": (ctypes.c_int, [_VP, ctypes.c_uint32, _F, ctypes.c_int32,
                                                       ctypes.c_float, _F, ctypes.c_uint64]),
            "brmppi_submit": (ctypes.c_int, [_VP, ctypes.c_uint32, _D, _F, ctypes.c_int32,
                                             ctypes.POINTER(ctypes.c_uint64)]),
            "brmppi_poll": (ctypes.c_int, [_VP, ctypes.c_uint64, _F, _F,
                                           ctypes.POINTER(ctypes.c_double)]),
            "brmppi_vehicle_export": (ctypes.c_int, [_VP, ctypes.c_uint32, _F,
                                                     ctypes.POINTER(ctypes.c_uint64),
                                                     ctypes.POINTER(ctypes.c_uint64)]),
            "brmppi_vehicle_import": (ctypes.c_int, [_VP, ctypes.c_uint32, _F, ctypes.c_uint64,
                                                     ctypes.c_uint64]),
            "brmppi_server_stats_get": (ctypes.c_int, [_VP, ctypes.POINTER(brmppi_server_stats)]),
            "brmppi_solve_device_noalloc": (ctypes.c_int, [P, _VP, _VP, _VP, ctypes.c_int32, _VP,
                                                           ctypes.c_int32, ctypes.c_float,
                                                           ctypes.c_uint64, ctypes.c_uint64, _VP,
                                                           _VP, _VP, _VP, _VP, _VP]),
            "brmppi_hitch_stabilize_device": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int32, _VP,
                                                             _VP]),
            "brmppi_transfer_bytes": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32,
                                                     ctypes.POINTER(ctypes.c_uint64),
                                                     ctypes.POINTER(ctypes.c_uint64)]),
            "brmppi_noise_blocks": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int32,
                                                   ctypes.c_int32, ctypes.c_int32, _VP, _VP, _VP]),
            "brmppi_measure_pipe": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64,
                                                   ctypes.POINTER(ctypes.c_double),
                                                   ctypes.POINTER(ctypes.c_double), _VP]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


class BrmppiError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def brmppi_default_params() -> brmppi_params:
    p = brmppi_params()
    load().brmppi_default_params(ctypes.byref(p))
    return p


def params_from_dict(d: dict, max_obstacles: int = 16, max_path_pts: int = 4096,
                     threads_per_sample: int = 0, block_threads: int = 0, max_batch: int = 0,
                     batch_threads_per_sample: int = 0, batch_block_threads: int = 0,
                     max_vehicles: int = 0, serve_lanes: int = 0, serve_max_batch: int = 0,
                     serve_queue: int = 0, wait_timeout_ms: int = 0) -> brmppi_params:
    """brmppi_params from the parameter dict of ``scenarios`` (values are
    rounded to binary32 by the struct)."""
    p = brmppi_default_params()
    for name, _ in brmppi_params._fields_:
        key = "lambda" if name == "lambda_" else name
        if key in d:
            val = d[key]
            attr = getattr(p, name)
            if isinstance(attr, ctypes.Array):
                for i, v in enumerate(val):
                    attr[i] = float(v)
            elif isinstance(attr, int):
                setattr(p, name, int(val))
            else:
                setattr(p, name, float(val))
    p.max_obstacles = int(max_obstacles)
    p.max_path_pts = int(max_path_pts)
    p.threads_per_sample = int(threads_per_sample)
    p.block_threads = int(block_threads)
    p.max_batch = int(max_batch)
    p.batch_threads_per_sample = int(batch_threads_per_sample)
    p.batch_block_threads = int(batch_block_threads)
    p.max_vehicles = int(max_vehicles)
    p.serve_lanes = int(serve_lanes)
    p.serve_max_batch = int(serve_max_batch)
    p.serve_queue = int(serve_queue)
    p.wait_timeout_ms = int(wait_timeout_ms)
    p.abi_version = BRMPPI_ABI_VERSION
    return p


def brmppi_create(params: brmppi_params, device: int = 0) -> ctypes.c_void_p:
    lib = load()
    h = _VP()
    st = lib.brmppi_create(ctypes.byref(params), int(device), ctypes.byref(h))
    if st != BRMPPI_OK:
        raise BrmppiError(st, lib.brmppi_last_error(None).decode())
    return h


def brmppi_destroy(ctx) -> int:
    """Destroy a context; BRMPPI_ETIMEDOUT if a bounded wait for its work
    gave up (its buffers are then left allocated)."""
    if ctx:
        return load().brmppi_destroy(ctx)
    return BRMPPI_OK


def brmppi_inject_alloc_failure(n: int) -> None:
    """Testing hook: the n-th library allocation from now on fails as out of
    memory (n <= 0 disarms)."""
    load().brmppi_inject_alloc_failure(int(n))


def brmppi_last_error(ctx) -> str:
    return load().brmppi_last_error(ctx).decode()


def _rows(obs) -> int:
    """Obstacle count of an obstacle array: its first dimension when 2-D
    (rows of 6, or of 8 under BRMPPI_FLAG_OBS8), else its size / 6."""
    if obs is None:
        return 0
    shape = tuple(obs.shape)
    if len(shape) == 2:
        return int(shape[0])
    return int(np.prod(shape)) // 6


def _f32(a, n=None):
    arr = np.ascontiguousarray(a, dtype=np.float32)
    if n is not None and arr.size != n:
        raise ValueError(f"expected {n} floats, got {arr.size}")
    return arr


def brmppi_solve(ctx, x0, U_nom, obs, path, ds, seed, counter, H, S=None, want_traj=True,
                 want_J=False):
    """Host-buffer solve. Returns (status, U[H,3], traj[H+1,7] or None, J[S] or None)."""
    lib = _lib or load()
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    if x0.size not in (7, 8):
        raise ValueError("x0 must have 7 entries (8 under the jerk-input model)")
    U_nom = _f32(U_nom, 3 * H)
    n_obs = _rows(None if obs is None else np.asarray(obs))
    obs = _f32(obs) if n_obs else None
    path = _f32(path)
    n_pts = path.size // 3
    U = np.zeros((H, 3), dtype=np.float32)
    traj = np.zeros((H + 1, 7), dtype=np.float32) if want_traj else None
    J = np.zeros(S, dtype=np.float32) if want_J else None
    st = lib.brmppi_solve(ctx, x0.ctypes.data, U_nom.ctypes.data, obs.ctypes.data if n_obs else None, n_obs,
                          path.ctypes.data, n_pts, float(ds), int(seed) & (2**64 - 1),
                          int(counter) & (2**64 - 1), U.ctypes.data,
                          traj.ctypes.data if traj is not None else None,
                          J.ctypes.data if J is not None else None)
    return st, U, traj, J


def _dptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def brmppi_solve_device(ctx, x0, U_nom, obs, path, ds, seed, counter, U_out, traj_out=None,
                        J_out=None, U_next=None, status=None, stream=None) -> int:
    """Device-buffer solve on torch CUDA tensors (x0 float64[7], U_nom
    float32[H,3], obs float32[n,6], path float32[n,3], outputs float32;
    status int32[1]).  Enqueued on ``stream`` (torch stream or raw handle;
    default: torch's current stream); does not synchronise."""
    lib = load()
    n_obs = _rows(obs)
    n_pts = path.numel() // 3
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    elif hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    return lib.brmppi_solve_device(ctx, _dptr(x0), _dptr(U_nom), _dptr(obs) if n_obs else None,
                                   n_obs, _dptr(path), n_pts, float(ds), int(seed) & (2**64 - 1),
                                   int(counter) & (2**64 - 1), _dptr(U_out), _dptr(traj_out),
                                   _dptr(J_out), _dptr(U_next), _dptr(status),
                                   ctypes.c_void_p(int(stream)))


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def make_instances(insts) -> "ctypes.Array":
    """ctypes array of brmppi_instance from dicts of torch CUDA tensors
    (x0, U_nom, obs, path, U_out; optional traj_out, J_out, U_next, status,
    states_out, u_safe_out, inputs_out, J_lo_out)
    and scalars (ds, seed, counter)."""
    arr = (brmppi_instance * len(insts))()
    for i, d in enumerate(insts):
        q = arr[i]
        q.x0 = d["x0"].data_ptr()
        q.U_nom = d["U_nom"].data_ptr()
        obs = d.get("obs")
        q.n_obs = _rows(obs)
        q.obs = obs.data_ptr() if q.n_obs else None
        q.path = d["path"].data_ptr()
        q.n_pts = d["path"].numel() // 3
        q.ds = float(d["ds"])
        q.H = d["U_nom"].numel() // 3
        q.S = int(d["S"])
        q.seed = int(d["seed"]) & (2**64 - 1)
        q.counter = int(d.get("counter", 0)) & (2**64 - 1)
        q.U_out = d["U_out"].data_ptr() if d.get("U_out") is not None else None
        for key in ("traj_out", "J_out", "U_next", "status", "states_out", "u_safe_out", "inputs_out",
                    "J_lo_out"):
            t = d.get(key)
            setattr(q, key, None if t is None else t.data_ptr())
    return arr


def brmppi_solve_device_ex(ctx, inst, stream=None) -> int:
    """One solve from a dict of torch CUDA tensors (as for batches; may carry
    ``states_out`` of shape (S, H+1, 7))."""
    arr = make_instances([inst])
    return load().brmppi_solve_device_ex(ctx, arr, ctypes.c_void_p(_stream_handle(stream)))


def brmppi_tile_layout(ctx, inst):
    """(n_tiles, tile_floats) of a sample-partitioned solve of `inst`."""
    arr = make_instances([inst])
    nt, tf = ctypes.c_int32(), ctypes.c_int32()
    st = load().brmppi_tile_layout(ctx, arr, ctypes.byref(nt), ctypes.byref(tf))
    if st != BRMPPI_OK:
        raise BrmppiError(st, brmppi_last_error(ctx))
    return nt.value, tf.value


def brmppi_solve_tiles(ctx, inst, tile0: int, n_tiles: int, tiles_out, stream=None) -> int:
    """Tiles [tile0, tile0 + n_tiles) of `inst` (dict of torch CUDA tensors,
    U_out optional) into tiles_out (float32, n_tiles x tile_floats)."""
    arr = make_instances([inst])
    return load().brmppi_solve_tiles(ctx, arr, int(tile0), int(n_tiles), _dptr(tiles_out),
                                     ctypes.c_void_p(_stream_handle(stream)))


def brmppi_merge_tiles(ctx, inst, tiles, stream=None) -> int:
    """Merge every tile of `inst` (tiles: float32, n_tiles x tile_floats, in
    tile order) into its U_out (and traj_out, U_next, status if given)."""
    arr = make_instances([inst])
    n = tiles.shape[0]
    return load().brmppi_merge_tiles(ctx, arr, _dptr(tiles), int(n), ctypes.c_void_p(_stream_handle(stream)))


def brmppi_solve_batch(ctx, insts, stream=None) -> int:
    arr = insts if isinstance(insts, ctypes.Array) else make_instances(insts)
    return load().brmppi_solve_batch(ctx, arr, len(arr), ctypes.c_void_p(_stream_handle(stream)))


def brmppi_batch_capture(ctx, insts):
    arr = insts if isinstance(insts, ctypes.Array) else make_instances(insts)
    g = _VP()
    st = load().brmppi_batch_capture(ctx, arr, len(arr), ctypes.byref(g))
    if st != BRMPPI_OK:
        raise BrmppiError(st, brmppi_last_error(ctx))
    return g


def brmppi_graph_launch(graph, stream=None) -> int:
    return load().brmppi_graph_launch(graph, ctypes.c_void_p(_stream_handle(stream)))


def brmppi_graph_destroy(graph) -> None:
    if graph:
        load().brmppi_graph_destroy(graph)


def brmppi_autotune(ctx, x0, U_nom, obs, path, ds, reps=5, stream=None) -> int:
    n_obs = _rows(obs)
    return load().brmppi_autotune(ctx, _dptr(x0), _dptr(U_nom), _dptr(obs) if n_obs else None,
                                  n_obs, _dptr(path), path.numel() // 3, float(ds), int(reps),
                                  ctypes.c_void_p(_stream_handle(stream)))


def brmppi_autotune_batch(ctx, insts, reps=3, stream=None) -> int:
    arr = insts if isinstance(insts, ctypes.Array) else make_instances(insts)
    return load().brmppi_autotune_batch(ctx, arr, len(arr), int(reps),
                                        ctypes.c_void_p(_stream_handle(stream)))


def brmppi_solve_device_noalloc(params, x0, U_nom, obs, path, ds, seed, counter, U_out,
                                traj_out=None, J_out=None, U_next=None, status=None,
                                stream=None) -> int:
    """Allocation-free solve (no context) on torch CUDA tensors; see
    include/brmppi.h for its limits.  ``params``: brmppi_params."""
    n_obs = _rows(obs)
    return load().brmppi_solve_device_noalloc(
        ctypes.byref(params), _dptr(x0), _dptr(U_nom), _dptr(obs) if n_obs else None, n_obs,
        _dptr(path), path.numel() // 3, float(ds), int(seed) & (2**64 - 1),
        int(counter) & (2**64 - 1), _dptr(U_out), _dptr(traj_out), _dptr(J_out), _dptr(U_next),
        _dptr(status), ctypes.c_void_p(_stream_handle(stream)))


def brmppi_hitch_stabilize_device(ctx, x, u_ref, u_out, stream=None) -> int:
    """Hitch stabilizer for n states: x float64[n,7] (n x 8 under the
    jerk-input model), u_ref float32[n,3], u_out float32[n,4]
    (a or jerk, omega, nu, slack), torch CUDA tensors."""
    n = u_ref.numel() // 3
    return load().brmppi_hitch_stabilize_device(ctx, _dptr(x), _dptr(u_ref), n, _dptr(u_out),
                                                ctypes.c_void_p(_stream_handle(stream)))


def brmppi_noise_blocks(seed: int, counter: int, n_samples: int, H: int, n_blocks: int, words=None,
                        normals=None, stream=None) -> int:
    """The solves' noise stream: Philox words (uint32 viewed as int32) and
    normals (float32) of shape (n_samples, H, n_blocks, 4), torch CUDA
    tensors or None."""
    return load().brmppi_noise_blocks(int(seed), int(counter), int(n_samples), int(H), int(n_blocks),
                                      _dptr(words), _dptr(normals), ctypes.c_void_p(_stream_handle(stream)))


PIPE_FMA, PIPE_IMAD, PIPE_XU = 0, 1, 2


def brmppi_measure_pipe(pipe: int, iters: int, stream=None):
    """(lane operations per second, seconds) of one SM pipe's issue-rate
    microbenchmark on the current device (PIPE_FMA, PIPE_IMAD, PIPE_XU)."""
    rate, sec = ctypes.c_double(), ctypes.c_double()
    st = load().brmppi_measure_pipe(int(pipe), int(iters), ctypes.byref(rate), ctypes.byref(sec),
                                    ctypes.c_void_p(_stream_handle(stream)))
    if st != BRMPPI_OK:
        raise BrmppiError(st, brmppi_last_error(None))
    return rate.value, sec.value


def brmppi_get_launch(ctx, n_obs: int):
    tps, thr, blk = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    st = load().brmppi_get_launch(ctx, int(n_obs), ctypes.byref(tps), ctypes.byref(thr),
                                  ctypes.byref(blk))
    if st != BRMPPI_OK:
        raise BrmppiError(st, brmppi_last_error(ctx))
    return dict(threads_per_sample=tps.value, block_threads=thr.value, blocks=blk.value)


def brmppi_transfer_bytes(ctx, n_obs: int, n_pts: int):
    h2d, d2h = ctypes.c_uint64(), ctypes.c_uint64()
    st = load().brmppi_transfer_bytes(ctx, int(n_obs), int(n_pts), ctypes.byref(h2d),
                                      ctypes.byref(d2h))
    if st != BRMPPI_OK:
        raise BrmppiError(st, brmppi_last_error(ctx))
    return int(h2d.value), int(d2h.value)


def brmppi_get_batch_launch(ctx):
    tps, thr = ctypes.c_int32(), ctypes.c_int32()
    st = load().brmppi_get_batch_launch(ctx, ctypes.byref(tps), ctypes.byref(thr))
    if st != BRMPPI_OK:
        raise BrmppiError(st, brmppi_last_error(ctx))
    return dict(threads_per_sample=tps.value, block_threads=thr.value)


# ---- serving loop: vehicles with device-resident nominal sequences and RNG
# counters; requests queued by brmppi_submit and collected by brmppi_poll
def brmppi_vehicle_register(ctx, vehicle_id: int, path, ds: float, H: int, U_init=None,
                            seed: int = 0) -> None:
    path = _f32(path).reshape(-1)
    U = None if U_init is None else _f32(U_init, 3 * int(H))
    st = load().brmppi_vehicle_register(ctx, int(vehicle_id), path.ctypes.data_as(_F),
                                        path.size // 3, float(ds),
                                        None if U is None else U.ctypes.data_as(_F),
                                        int(seed) & (2**64 - 1))
    if st != BRMPPI_OK:
        raise BrmppiError(st, brmppi_last_error(ctx))


def brmppi_submit(ctx, vehicle_id: int, x0, obs=None, obs_row: int = 6):
    """Queue one solve; returns (status, ticket).  obs_row: floats per
    obstacle row (6, or 8 with BRMPPI_FLAG_OBS8)."""
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    ob = np.zeros(0, np.float32) if obs is None else _f32(obs).reshape(-1)
    t = ctypes.c_uint64()
    st = load().brmppi_submit(ctx, int(vehicle_id), x0.ctypes.data_as(_D),
                              ob.ctypes.data_as(_F) if ob.size else None, ob.size // int(obs_row),
                              ctypes.byref(t))
    return st, t.value


def brmppi_poll(ctx, ticket: int, H: int, want_traj: bool = False):
    """(status, U, traj, latency_s); status EAGAIN while the solve runs."""
    U = np.empty((int(H), 3), np.float32)
    traj = np.empty((int(H) + 1, 7), np.float32) if want_traj else None
    lat = ctypes.c_double()
    st = load().brmppi_poll(ctx, int(ticket), U.ctypes.data_as(_F),
                            traj.ctypes.data_as(_F) if traj is not None else None,
                            ctypes.byref(lat))
    return st, U, traj, lat.value


def brmppi_vehicle_export(ctx, vehicle_id: int, H: int):
    U = np.empty((int(H), 3), np.float32)
    seed, ctr = ctypes.c_uint64(), ctypes.c_uint64()
    st = load().brmppi_vehicle_export(ctx, int(vehicle_id), U.ctypes.data_as(_F),
                                      ctypes.byref(seed), ctypes.byref(ctr))
    if st != BRMPPI_OK:
        raise BrmppiError(st, brmppi_last_error(ctx))
    return U, seed.value, ctr.value


def brmppi_vehicle_import(ctx, vehicle_id: int, U_nom, H: int, seed: int, counter: int) -> None:
    U = _f32(U_nom, 3 * int(H))
    st = load().brmppi_vehicle_import(ctx, int(vehicle_id), U.ctypes.data_as(_F),
                                      int(seed) & (2**64 - 1), int(counter) & (2**64 - 1))
    if st != BRMPPI_OK:
        raise BrmppiError(st, brmppi_last_error(ctx))


def brmppi_server_stats_get(ctx) -> dict:
    out = brmppi_server_stats()
    st = load().brmppi_server_stats_get(ctx, ctypes.byref(out))
    if st != BRMPPI_OK:
        raise BrmppiError(st, brmppi_last_error(ctx))
    return {name: getattr(out, name) for name, _ in brmppi_server_stats._fields_}


class Solver:
    """Convenience owner of one context."""

    def __init__(self, params: dict, device: int = 0, max_obstacles: int = 16,
                 max_path_pts: int = 4096, threads_per_sample: int = 0, block_threads: int = 0,
                 max_batch: int = 0, batch_threads_per_sample: int = 0,
                 batch_block_threads: int = 0, max_vehicles: int = 0, serve_lanes: int = 0,
                 serve_max_batch: int = 0, serve_queue: int = 0, wait_timeout_ms: int = 0):
        self.ctx = None
        self.params = dict(params)
        self.S = int(params["S"])
        self.H = int(params["H"])
        self._p = params_from_dict(params, max_obstacles, max_path_pts, threads_per_sample,
                                   block_threads, max_batch, batch_threads_per_sample,
                                   batch_block_threads, max_vehicles, serve_lanes,
                                   serve_max_batch, serve_queue, wait_timeout_ms)
        self.ctx = brmppi_create(self._p, device)

    def close(self) -> int:
        """Destroy the context; the status of brmppi_destroy."""
        st = BRMPPI_OK
        if self.ctx:
            st = brmppi_destroy(self.ctx)
            self.ctx = None
        return st

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _host_buffers(self):
        """Host staging owned by the Solver for brmppi_solve: the inputs are
        copied into it and the outputs read from it, so that the per-call
        marshalling (the closed loop's per-tick cost) only copies arrays;
        every address is taken once."""
        if getattr(self, "_hb", None) is None:
            nx = 8 if int(self.params.get("flags", 0)) & BRMPPI_FLAG_JERK_MODEL else 7
            row = 8 if int(self.params.get("flags", 0)) & BRMPPI_FLAG_OBS8 else 6
            bufs = dict(x0=np.zeros(nx), U_nom=np.zeros((self.H, 3), np.float32),
                        obs=np.zeros((max(1, int(self._p.max_obstacles)), row), np.float32),
                        path=np.zeros((int(self._p.max_path_pts), 3), np.float32),
                        U=np.zeros((self.H, 3), np.float32), traj=np.zeros((self.H + 1, 7), np.float32),
                        J=np.zeros(self.S, np.float32))
            self._hb = (bufs, {k: v.ctypes.data for k, v in bufs.items()}, nx, row)
        return self._hb

    def solve(self, x0, U_nom, obs, path, ds, seed, counter, want_traj=True, want_J=False,
              check=True):
        bufs, adr, nx, row = self._host_buffers()
        x0 = np.asarray(x0)
        if x0.size != nx:
            raise ValueError(f"x0 must have {nx} entries")
        n_obs = _rows(None if obs is None else np.asarray(obs))
        path = np.asarray(path)
        n_pts = path.size // 3
        if n_obs > bufs["obs"].shape[0] or n_pts > bufs["path"].shape[0] or n_pts * 3 != path.size:
            # beyond the context's capacities: the library reports it
            st, U, traj, J = brmppi_solve(self.ctx, x0, U_nom, obs, path, ds, seed, counter, self.H,
                                          self.S, want_traj, want_J)
        else:
            np.copyto(bufs["x0"], x0.reshape(-1), casting="unsafe")
            np.copyto(bufs["U_nom"], np.asarray(U_nom).reshape(self.H, 3), casting="unsafe")
            if n_obs:
                np.copyto(bufs["obs"][:n_obs], np.asarray(obs).reshape(n_obs, row), casting="unsafe")
            np.copyto(bufs["path"][:n_pts], path.reshape(n_pts, 3), casting="unsafe")
            lib = _lib or load()
            st = lib.brmppi_solve(self.ctx, adr["x0"], adr["U_nom"], adr["obs"] if n_obs else None, n_obs,
                                  adr["path"], n_pts, float(ds), int(seed) & (2**64 - 1),
                                  int(counter) & (2**64 - 1), adr["U"], adr["traj"] if want_traj else None,
                                  adr["J"] if want_J else None)
            U = bufs["U"].copy()
            traj = bufs["traj"].copy() if want_traj else None
            J = bufs["J"].copy() if want_J else None
        if check and st != BRMPPI_OK:
            raise BrmppiError(st, brmppi_last_error(self.ctx))
        return dict(status=st, U=U, traj=traj, J=J)

    def solve_device(self, *args, **kw) -> int:
        return brmppi_solve_device(self.ctx, *args, **kw)

    def launch(self, n_obs: int) -> dict:
        return brmppi_get_launch(self.ctx, n_obs)

    def batch_launch(self) -> dict:
        return brmppi_get_batch_launch(self.ctx)

    def transfer_bytes(self, n_obs: int, n_pts: int):
        return brmppi_transfer_bytes(self.ctx, n_obs, n_pts)

    def solve_device_ex(self, inst, stream=None, check=True) -> int:
        st = brmppi_solve_device_ex(self.ctx, inst, stream)
        if check and st != BRMPPI_OK:
            raise BrmppiError(st, brmppi_last_error(self.ctx))
        return st

    def solve_batch(self, insts, stream=None, check=True) -> int:
        st = brmppi_solve_batch(self.ctx, insts, stream)
        if check and st != BRMPPI_OK:
            raise BrmppiError(st, brmppi_last_error(self.ctx))
        return st

    def hitch_stabilize_device(self, x, u_ref, u_out, stream=None, check=True) -> int:
        st = brmppi_hitch_stabilize_device(self.ctx, x, u_ref, u_out, stream)
        if check and st != BRMPPI_OK:
            raise BrmppiError(st, brmppi_last_error(self.ctx))
        return st

    def capture_batch(self, insts):
        return brmppi_batch_capture(self.ctx, insts)

    def autotune(self, x0, U_nom, obs, path, ds, reps=5, stream=None):
        st = brmppi_autotune(self.ctx, x0, U_nom, obs, path, ds, reps, stream)
        if st != BRMPPI_OK:
            raise BrmppiError(st, brmppi_last_error(self.ctx))

    # ---- serving loop
    def register(self, vehicle_id: int, path, ds: float, U_init=None, seed: int = 0):
        brmppi_vehicle_register(self.ctx, vehicle_id, path, ds, self.H, U_init, seed)

    def submit(self, vehicle_id: int, x0, obs=None):
        """Queue one solve; returns (status, ticket)."""
        row = 8 if int(self.params.get("flags", 0)) & BRMPPI_FLAG_OBS8 else 6
        return brmppi_submit(self.ctx, vehicle_id, x0, obs, row)

    def poll(self, ticket: int, want_traj: bool = False):
        """(status, U, traj, latency_s); status EAGAIN while running."""
        return brmppi_poll(self.ctx, ticket, self.H, want_traj)

    def vehicle_export(self, vehicle_id: int):
        return brmppi_vehicle_export(self.ctx, vehicle_id, self.H)

    def vehicle_import(self, vehicle_id: int, U_nom, seed: int, counter: int):
        brmppi_vehicle_import(self.ctx, vehicle_id, U_nom, self.H, seed, counter)

    def server_stats(self) -> dict:
        return brmppi_server_stats_get(self.ctx)

    def autotune_batch(self, insts, reps=3, stream=None):
        st = brmppi_autotune_batch(self.ctx, insts, reps, stream)
        if st != BRMPPI_OK:
            raise BrmppiError(st, brmppi_last_error(self.ctx))
