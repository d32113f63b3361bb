"""Serving loop: requests from many vehicles admitted into batches as they
arrive (continuous batching over several lanes), device-resident warm starts
and noise counters, results equal alone and in the mix, parity with the FP64
oracle on the vehicle state each solve used."""
import time

import numpy as np
import pytest

import oracle
from paper_2508_05773_gb300 import scenarios as sc
from tests.parity import assert_solve_matches
from tests.served import served_costs

pytestmark = pytest.mark.gpu

S, H = 512, 20


@pytest.fixture(scope="module")
def pkg():
    from paper_2508_05773_gb300 import build as native_build
    native_build.build()
    import paper_2508_05773_gb300
    paper_2508_05773_gb300.load()
    return paper_2508_05773_gb300


def _fleet(n, seed=3):
    rng = np.random.default_rng(seed)
    return [sc.random_instance(rng, S_choices=(S,), H_range=(H, H), obs_range=(0, 10)) for _ in range(n)]


def _server(pkg, n_vehicles, **kw):
    p = sc.params(S=S, H=H)
    kw.setdefault("max_batch", 1)  # a batch of one reproduces a served solve (its costs)
    return pkg.Solver(p, max_obstacles=16, max_path_pts=1024, max_vehicles=n_vehicles, **kw)


def _wait(srv, ticket, want_traj=True, timeout=30.0):
    t0 = time.time()
    while True:
        st, U, traj, lat = srv.poll(ticket, want_traj)
        if st != -3:  # EAGAIN
            return st, U, traj, lat
        if time.time() - t0 > timeout:
            raise TimeoutError("request did not finish")
        time.sleep(1e-4)


def test_served_solves_match_oracle_and_warm_start(pkg):
    fleet = _fleet(6)
    srv = _server(pkg, 8)
    try:
        for v, c in enumerate(fleet):
            srv.register(v, c["path"], c["ds"], c["U_nom"], c["seed"])
        states = {v: srv.vehicle_export(v) for v in range(len(fleet))}
        tickets = {}
        for v, c in enumerate(fleet):
            st, t = srv.submit(v, c["x0"], c["obs"])
            assert st == 0
            tickets[v] = t
        for v, c in enumerate(fleet):
            st, U, traj, lat = _wait(srv, tickets[v])
            assert st == 0 and lat > 0
            U0, seed, ctr = states[v]
            assert ctr == 0
            p = sc.as_float32(sc.params(S=S, H=H))
            ref = oracle.solve(p, c["x0"], U0, c["obs"], c["path"], c["ds"], seed, ctr,
                               want_uhist=True)
            sv = served_costs(srv, c, U0, seed, ctr, U)
            assert_solve_matches(dict(U=U, traj=traj, **sv), ref, p, f"vehicle {v}")
            # warm start and counter advanced on the device
            U1, seed1, ctr1 = srv.vehicle_export(v)
            assert ctr1 == 1 and seed1 == seed
            np.testing.assert_array_equal(U1, np.vstack([U[1:], U[-1:]]))
        stats = srv.server_stats()
        assert stats["completed"] == len(fleet) and stats["batches"] >= 1
    finally:
        srv.close()


def test_alone_equals_mix(pkg):
    fleet = _fleet(40, seed=5)
    srv = _server(pkg, 40, serve_lanes=3, serve_max_batch=16)
    try:
        for v, c in enumerate(fleet):
            srv.register(v, c["path"], c["ds"], c["U_nom"], c["seed"])
        snap = srv.vehicle_export(0)
        # alone
        st, t = srv.submit(0, fleet[0]["x0"], fleet[0]["obs"])
        st, U_alone, traj_alone, _ = _wait(srv, t)
        assert st == 0
        # restore vehicle 0, then the same request inside a burst of others
        srv.vehicle_import(0, *snap)
        tick = {}
        for v in range(1, 20):
            tick[v] = srv.submit(v, fleet[v]["x0"], fleet[v]["obs"])[1]
        tick[0] = srv.submit(0, fleet[0]["x0"], fleet[0]["obs"])[1]
        for v in range(20, 40):
            tick[v] = srv.submit(v, fleet[v]["x0"], fleet[v]["obs"])[1]
        res = {v: _wait(srv, t) for v, t in tick.items()}
        assert all(r[0] == 0 for r in res.values())
        np.testing.assert_array_equal(res[0][1], U_alone)
        np.testing.assert_array_equal(res[0][2], traj_alone)
        stats = srv.server_stats()
        assert stats["batches"] >= 2
    finally:
        srv.close()


def test_requests_of_one_vehicle_run_in_order(pkg):
    fleet = _fleet(1, seed=9)
    c = fleet[0]
    xs = [np.asarray(c["x0"]) + np.array([0.1 * k, 0, 0, 0, 0, 0, 0]) for k in range(3)]
    srv = _server(pkg, 2)
    try:
        srv.register(0, c["path"], c["ds"], c["U_nom"], c["seed"])
        srv.register(1, c["path"], c["ds"], c["U_nom"], c["seed"])
        # vehicle 0: three requests queued back to back
        t0 = [srv.submit(0, x, c["obs"])[1] for x in xs]
        burst = [_wait(srv, t)[1] for t in t0]
        # vehicle 1 (same start): the same requests one at a time
        seq = []
        for x in xs:
            st, t = srv.submit(1, x, c["obs"])
            seq.append(_wait(srv, t)[1])
        for a, b in zip(burst, seq):
            np.testing.assert_array_equal(a, b)
        assert srv.vehicle_export(0)[2] == 3
    finally:
        srv.close()


def test_backpressure_and_errors(pkg):
    fleet = _fleet(2, seed=11)
    srv = _server(pkg, 2, serve_queue=3)
    try:
        c = fleet[0]
        assert srv.server_stats()["request_slots"] == 3
        st, _ = srv.submit(0, c["x0"], c["obs"])  # unregistered vehicle
        assert st == pkg.BRMPPI_EINVAL
        sharp = c["path"].copy()
        sharp[3:, 2] += 1.0  # consecutive headings more than pi/4 apart
        with pytest.raises(pkg.BrmppiError):
            srv.register(0, sharp, c["ds"], c["U_nom"], c["seed"])
        srv.register(0, c["path"], c["ds"], c["U_nom"], c["seed"])
        tickets = [srv.submit(0, c["x0"], c["obs"])[1] for _ in range(3)]
        st, _ = srv.submit(0, c["x0"], c["obs"])  # slots are held until polled
        assert st == pkg.BRMPPI_EBUSY
        with pytest.raises(pkg.BrmppiError):
            srv.vehicle_export(0)  # busy
        for t in tickets:
            assert _wait(srv, t)[0] == 0
        st, *_ = srv.poll(tickets[0])
        assert st == pkg.BRMPPI_EINVAL  # already released
        x = np.array(c["x0"], dtype=np.float64)
        x[0] = np.inf
        assert srv.submit(0, x, c["obs"])[0] == pkg.BRMPPI_ENONFINITE
    finally:
        srv.close()


def test_config4_full_size_request(pkg):
    """A served request of the config-4 size (S=4096, H=50, obstacles as in
    config 3) through the serving loop's own launch shape, against the
    oracle on the state and warm start it was solved from."""
    rng = np.random.default_rng(4)
    c = sc.random_instance(rng, S_choices=(4096,), H_range=(50, 50), obs_range=(12, 12))
    pd = sc.params(S=4096, H=50)
    srv = pkg.Solver(pd, max_obstacles=16, max_path_pts=1024, max_vehicles=4, serve_lanes=2,
                     serve_max_batch=16, max_batch=1)
    try:
        srv.register(0, c["path"], c["ds"], c["U_nom"], c["seed"])
        U0, seed, ctr = srv.vehicle_export(0)
        st, t = srv.submit(0, c["x0"], c["obs"])
        assert st == 0
        st, U, traj, lat = _wait(srv, t)
        assert st == 0
        p = sc.as_float32(pd)
        ref = oracle.solve(p, c["x0"], U0, c["obs"], c["path"], c["ds"], seed, ctr, want_uhist=True)
        sv = served_costs(srv, c, U0, seed, ctr, U)
        assert_solve_matches(dict(U=U, traj=traj, **sv), ref, p, "config-4 request", strict=True)
    finally:
        srv.close()
