"""Failure paths of the library, made on the host (no GPU fault, hang or
trap): allocation failures injected through the library's allocation layer
(BRMPPI_ENOMEM, clean unwinding, the context usable afterwards), bounded host
waits that give up (BRMPPI_ETIMEDOUT from the serving loop and from
brmppi_destroy, the process healthy afterwards), and a solve in which no
rollout has a finite cost (BRMPPI_ENONFINITE with the nominal sequence as
U*)."""
import time

import numpy as np
import pytest

from paper_2508_05773_gb300 import scenarios as sc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from paper_2508_05773_gb300 import build as native_build
    native_build.build()
    import paper_2508_05773_gb300
    paper_2508_05773_gb300.load()
    return paper_2508_05773_gb300


def test_injected_allocation_failures_unwind(pkg):
    import torch
    p = sc.params(S=512, H=20)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    failures = 0
    try:
        for n in range(1, 80):
            pkg.brmppi_inject_alloc_failure(n)
            try:
                s = pkg.Solver(p, max_obstacles=8, max_path_pts=512, max_batch=4, max_vehicles=2, serve_lanes=2,
                               serve_queue=8)
            except pkg.BrmppiError as e:
                assert e.status == pkg.BRMPPI_ENOMEM, (n, e)
                failures += 1
                continue
            # n is past the allocations a context makes: the hook never fired
            pkg.brmppi_inject_alloc_failure(0)
            c = sc.small_random(3, S=512, H=20, n_obs=2)
            # a vehicle's buffers are allocated at registration: that fails too
            pkg.brmppi_inject_alloc_failure(1)
            with pytest.raises(pkg.BrmppiError) as ei:
                s.register(0, c["path"], c["ds"], c["U_nom"], c["seed"])
            assert ei.value.status == pkg.BRMPPI_ENOMEM
            s.register(0, c["path"], c["ds"], c["U_nom"], c["seed"])  # the hook fired once
            out = s.solve(c["x0"], c["U_nom"], c["obs"], c["path"], c["ds"], c["seed"], 0)
            assert out["status"] == 0 and np.all(np.isfinite(out["U"]))
            assert s.close() == pkg.BRMPPI_OK
            break
        else:
            raise AssertionError("the context never came up")
    finally:
        pkg.brmppi_inject_alloc_failure(0)
    assert failures >= 20  # every allocation of the context was made to fail in turn
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    # the failed creates released what they had allocated
    assert free1 >= free0 - (64 << 20), (free0, free1)


def _wait_done(srv, ticket, limit=30.0):
    t0 = time.time()
    while True:
        st, U, traj, lat = srv.poll(ticket, True)
        if st != -3:  # EAGAIN
            return st, U
        assert time.time() - t0 < limit
        time.sleep(1e-4)


def test_serving_wait_limit_gives_up_and_recovers(pkg):
    # a served solve that runs longer than the 1 ms wait limit (S = 65536,
    # H = 300, 16 ellipses: a few ms): its request is answered ETIMEDOUT; the
    # vehicle stays busy until the batch really ends, then everything is
    # usable again
    c = sc.config5(S=65536, H=300, n_obs=16)
    p = dict(c["params"])
    srv = pkg.Solver(p, max_obstacles=16, max_path_pts=c["path"].shape[0], max_vehicles=2, serve_lanes=1,
                     serve_queue=4, wait_timeout_ms=1)
    try:
        srv.register(0, c["path"], c["ds"], c["U_nom"], c["seed"])
        st, t = srv.submit(0, c["x0"], c["obs"])
        assert st == 0
        st, _ = _wait_done(srv, t)
        assert st == pkg.BRMPPI_ETIMEDOUT
        # the batch is still on the device or just finished: the vehicle is
        # busy until it ends, then free with its counter advanced
        t0 = time.time()
        while True:
            try:
                U1, seed1, ctr1 = srv.vehicle_export(0)
                break
            except pkg.BrmppiError as e:
                assert e.status == pkg.BRMPPI_EBUSY
                assert time.time() - t0 < 30
                time.sleep(1e-3)
        assert ctr1 == 1 and np.all(np.isfinite(U1))
        stats = srv.server_stats()
        assert stats["completed"] == 1
    finally:
        assert srv.close() == pkg.BRMPPI_OK


def test_destroy_gives_up_on_a_running_batch(pkg):
    import torch
    c = sc.config5(S=65536, H=200, n_obs=64)
    dev = torch.device("cuda:0")
    S, H = int(c["params"]["S"]), int(c["params"]["H"])
    t = lambda a, dt=torch.float32: torch.as_tensor(np.asarray(a), dtype=dt, device=dev)
    inst = dict(x0=t(c["x0"], torch.float64), U_nom=t(c["U_nom"]), obs=t(c["obs"]), path=t(c["path"]), ds=c["ds"],
                S=S, seed=c["seed"], counter=0, U_out=torch.empty((H, 3), device=dev),
                traj_out=torch.empty((H + 1, 7), device=dev),
                status=torch.full((1,), 99, dtype=torch.int32, device=dev))
    s = pkg.Solver(c["params"], max_obstacles=64, max_path_pts=c["path"].shape[0], max_batch=1,
                   wait_timeout_ms=1)
    stream = torch.cuda.Stream()
    s.solve_batch([inst], stream)  # a ~5 ms launch
    st = s.close()  # gives up after 1 ms: leaves the batch's buffers allocated
    assert st == pkg.BRMPPI_ETIMEDOUT
    torch.cuda.synchronize()
    assert int(inst["status"].item()) == 0  # the batch itself ran to its end
    # the process and the device are healthy: a new context solves
    c2 = sc.small_random(4, S=256, H=16, n_obs=3)
    s2 = pkg.Solver(c2["params"], max_obstacles=4, max_path_pts=512)
    try:
        out = s2.solve(c2["x0"], c2["U_nom"], c2["obs"], c2["path"], c2["ds"], c2["seed"], 0)
        assert out["status"] == 0
    finally:
        assert s2.close() == pkg.BRMPPI_OK


def test_no_finite_cost_returns_the_nominal(pkg):
    # a speed of 1e30 m/s is a finite input whose binary32 rollouts overflow:
    # every cost is infinite, no sample gets a weight, U* = U_nom
    import torch
    c = sc.small_random(5, S=300, H=12, n_obs=2)
    x0 = np.array(c["x0"], dtype=np.float64)
    x0[4] = 1e30
    s = pkg.Solver(c["params"], max_obstacles=4, max_path_pts=512)
    try:
        out = s.solve(x0, c["U_nom"], c["obs"], c["path"], c["ds"], c["seed"], 0, want_J=True, check=False)
        assert out["status"] == pkg.BRMPPI_ENONFINITE
        np.testing.assert_array_equal(out["U"], c["U_nom"])
        assert not np.any(np.isfinite(out["J"]))
        # the device entry point reports it in the status word
        dev = torch.device("cuda:0")
        t = lambda a, dt=torch.float32: torch.as_tensor(np.asarray(a), dtype=dt, device=dev)
        U = torch.empty((12, 3), device=dev)
        Un = torch.empty((12, 3), device=dev)
        stw = torch.full((1,), 99, dtype=torch.int32, device=dev)
        rc = s.solve_device(t(x0, torch.float64), t(c["U_nom"]), t(c["obs"]), t(c["path"]), c["ds"], c["seed"], 0,
                            U, None, None, Un, stw)
        assert rc == 0
        torch.cuda.synchronize()
        assert int(stw.item()) == pkg.BRMPPI_ENONFINITE
        np.testing.assert_array_equal(U.cpu().numpy(), c["U_nom"])
        # and the next solve on the context is unaffected
        out = s.solve(c["x0"], c["U_nom"], c["obs"], c["path"], c["ds"], c["seed"], 0)
        assert out["status"] == 0
    finally:
        s.close()
