"""Paper-scale closed loop (S=4096, H=50, 8 ellipses, reverse parking path):
1000 consecutive control ticks through the host entry point, FP64 host plant
advanced by U*[0], nominal sequence warm-started by the one-step shift.  The
GPU solve is checked against the FP64 oracle on the very inputs of ticks 0,
500 and 999; every tick's solve must stay under the 10 ms control deadline."""
import time

import numpy as np
import pytest

import oracle
from paper_2508_05773_gb300 import plant
from paper_2508_05773_gb300 import scenarios as sc
from tests.gpu_solve import device_solve
from tests.parity import assert_solve_matches

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from paper_2508_05773_gb300 import build as native_build
    native_build.build()
    import paper_2508_05773_gb300
    paper_2508_05773_gb300.load()
    return paper_2508_05773_gb300


def test_closed_loop_1000_ticks(pkg):
    c = sc.config2()
    p = c["params"]
    p32 = sc.as_float32(p)
    solver = pkg.Solver(p, max_obstacles=8, max_path_pts=512)
    checks = {0: None, 500: None, 999: None}
    x = np.array(c["x0"], dtype=np.float64)
    U = np.array(c["U_nom"], dtype=np.float32)
    lat = []
    try:
        for k in range(1000):
            t0 = time.perf_counter()
            out = solver.solve(x, U, c["obs"], c["path"], c["ds"], c["seed"], k, want_J=k in checks)
            lat.append(time.perf_counter() - t0)
            if k in checks:
                # the same inputs through the device-instance entry point,
                # which also returns the cost pairs and applied inputs
                full = device_solve(solver, c, x0=x, U_nom=U, counter=k)
                assert np.array_equal(full["U"], out["U"]) and np.array_equal(full["J"], out["J"])
                checks[k] = (x.copy(), U.copy(), full)
            assert np.all(np.isfinite(out["U"]))
            x = plant.step(p32, x, out["U"][0])
            U = plant.shift(out["U"])
    finally:
        solver.close()
    for k, (xk, Uk, out) in checks.items():
        ref = oracle.solve(p32, xk, Uk, c["obs"], c["path"], c["ds"], c["seed"], k,
                           want_uhist=True)
        assert ref["status"] == 0
        # tick 0 also at the flat 1e-4 against the oracle's own U*; later
        # ticks hold near-tied samples whose binary32 costs move U* (shift_J)
        assert_solve_matches(out, ref, p32, f"tick {k}", strict=(k == 0))
    assert np.percentile(lat, 99) < 10e-3  # host-path tick latency under the deadline
    # the loop made progress along the reference path
    assert x[6] > 1.0
