"""The allocation-free solve entry point (brmppi_solve_device_noalloc).

It exists for callers that cannot allocate device memory once running --
work enqueued during CUDA-graph capture, controllers with memory fixed at
start-up -- and keeps its scratch in a fixed device array shared by all
calls.  Checked through the C ABI against the context-based device entry
point on the same inputs, for two calls in a row (the second call finds the
first call's leftovers in the shared array), within the parity tolerances
of the other tests.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2508_05773_gb300 import scenarios as sc
from tests.parity import EPS_J, TOL_STATE, TOL_U, err_j, err_state, err_u

pytestmark = pytest.mark.gpu


def _tensors(c, dev):
    import torch
    t = lambda a, dt=torch.float32: torch.tensor(np.asarray(a), dtype=dt, device=dev)
    return (t(c["x0"], torch.float64), t(c["U_nom"]), t(c["obs"]) if c["obs"].shape[0] else None,
            t(c["path"]))


def _outs(H, S, dev):
    import torch
    return dict(U=torch.empty((H, 3), device=dev), traj=torch.empty((H + 1, 7), device=dev),
                J=torch.empty(S, device=dev), Un=torch.empty((H, 3), device=dev),
                st=torch.full((1,), 99, dtype=torch.int32, device=dev))


def test_noalloc_matches_device_entry_point_twice():
    import torch
    from paper_2508_05773_gb300 import build as native_build
    native_build.build()
    import paper_2508_05773_gb300 as pkg
    pkg.load()
    dev = torch.device("cuda:0")
    c = sc.config2()   # S = 4096, H = 50, 8 ellipses: inside the no-alloc maxima
    S, H = int(c["params"]["S"]), int(c["params"]["H"])
    params = pkg.params_from_dict(c["params"], max_obstacles=8, max_path_pts=512)
    x0, Un, ob, pa = _tensors(c, dev)
    solver = pkg.Solver(c["params"], max_obstacles=8, max_path_pts=512)
    try:
        for call, counter in enumerate((c["counter"], c["counter"] + 7)):
            ref = _outs(H, S, dev)
            rc = solver.solve_device(x0, Un, ob, pa, c["ds"], c["seed"], counter, ref["U"], ref["traj"],
                                     ref["J"], ref["Un"], ref["st"])
            assert rc == 0
            got = _outs(H, S, dev)
            rc = pkg.brmppi_solve_device_noalloc(params, x0, Un, ob, pa, c["ds"], c["seed"], counter,
                                                 got["U"], got["traj"], got["J"], got["Un"], got["st"])
            assert rc == 0, pkg.brmppi_last_error(None)
            torch.cuda.synchronize()
            assert int(ref["st"].item()) == 0 and int(got["st"].item()) == 0
            g = {k: v.cpu().numpy() for k, v in got.items()}
            r = {k: v.cpu().numpy() for k, v in ref.items()}
            assert err_u(g["U"], r["U"], params_dict(c)) <= TOL_U, call
            assert err_state(g["traj"], r["traj"]) <= TOL_STATE, call
            assert err_j(g["J"], r["J"]) <= EPS_J, call
            np.testing.assert_array_equal(g["Un"], np.vstack([g["U"][1:], g["U"][-1:]]))
    finally:
        solver.close()


def params_dict(c):
    return sc.as_float32(c["params"])


def test_noalloc_rejects_sizes_beyond_its_maximum():
    import torch
    import paper_2508_05773_gb300 as pkg
    pkg.load()
    dev = torch.device("cuda:0")
    c = sc.small_random(3, S=64, H=8, n_obs=2)
    x0, Un, ob, pa = _tensors(c, dev)
    out = _outs(8, 64, dev)
    for field, value in (("S", 4097), ("H", 65)):
        params = pkg.params_from_dict(dict(c["params"], **{field: value}))
        rc = pkg.brmppi_solve_device_noalloc(params, x0, Un, ob, pa, c["ds"], 1, 0, out["U"])
        assert rc == pkg.BRMPPI_EINVAL
        assert "maximum" in pkg.brmppi_last_error(None)


def test_noalloc_at_its_maxima_allocates_nothing():
    """S = 4095 (a ragged last tile), H = 64, 16 obstacles, 4096 path rows:
    the largest solve the entry point accepts.  A context solve in the same
    fixed launch shape (4 lanes per sample, 128-thread blocks) runs the same
    kernel variant on the same tiles, so the two agree bit for bit.  After a
    first call (which may load the kernel's module), a call leaves the
    device's free memory unchanged."""
    import torch
    import paper_2508_05773_gb300 as pkg
    pkg.load()
    dev = torch.device("cuda:0")
    c = sc.small_random(31, S=4095, H=64, n_obs=16)
    ds = 0.012
    c["path"] = sc.path_table([("S", 40.0), ("A", 15.0, 1.2)], ds, reverse=True)[:4096].copy()
    c["ds"] = ds
    assert c["path"].shape[0] == 4096
    S, H = 4095, 64
    params = pkg.params_from_dict(c["params"], max_obstacles=16, max_path_pts=4096)
    x0, Un, ob, pa = _tensors(c, dev)
    solver = pkg.Solver(c["params"], max_obstacles=16, max_path_pts=4096, threads_per_sample=4,
                        block_threads=128)
    try:
        ref = _outs(H, S, dev)
        assert solver.solve_device(x0, Un, ob, pa, ds, c["seed"], c["counter"], ref["U"], ref["traj"],
                                   ref["J"], ref["Un"], ref["st"]) == 0
        got = _outs(H, S, dev)
        for call in range(2):
            torch.cuda.synchronize()
            free0, _ = torch.cuda.mem_get_info(dev)
            rc = pkg.brmppi_solve_device_noalloc(params, x0, Un, ob, pa, ds, c["seed"], c["counter"],
                                                 got["U"], got["traj"], got["J"], got["Un"], got["st"])
            assert rc == 0, pkg.brmppi_last_error(None)
            torch.cuda.synchronize()
            free1, _ = torch.cuda.mem_get_info(dev)
            if call == 1:
                assert free1 == free0, (free0, free1)
            assert int(got["st"].item()) == 0 and int(ref["st"].item()) == 0
            for k in ("U", "traj", "J", "Un"):
                assert np.array_equal(got[k].cpu().numpy(), ref[k].cpu().numpy()), (call, k)
    finally:
        solver.close()
