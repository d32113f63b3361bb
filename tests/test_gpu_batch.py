"""Batched solves (one persistent launch over uneven instances): each result
is bit-identical alone (a batch of one) and in the mix, matches the FP64
oracle within the stated tolerance, and a captured CUDA graph replays the
same work on updated inputs."""
import numpy as np
import pytest

import oracle
from paper_2508_05773_gb300 import scenarios as sc
from tests.gpu_solve import device_solve, device_tensors, host_outputs
from tests.parity import assert_solve_matches

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from paper_2508_05773_gb300 import build as native_build
    native_build.build()
    import paper_2508_05773_gb300
    paper_2508_05773_gb300.load()
    return paper_2508_05773_gb300


def _device_inst(c, dev):
    import torch
    d = device_tensors(c, dev)
    d["U_next"] = torch.empty((int(c["params"]["H"]), 3), device=dev)
    return d


def _instances(n, seed=1, S_choices=(64, 200, 333), H_range=(5, 24), obs_range=(0, 12)):
    rng = np.random.default_rng(seed)
    return [sc.random_instance(rng, S_choices=S_choices, H_range=H_range, obs_range=obs_range)
            for _ in range(n)]


def _ctx(pkg, cases, max_batch, **kw):
    S = max(int(c["params"]["S"]) for c in cases)
    H = max(int(c["params"]["H"]) for c in cases)
    p = dict(cases[0]["params"], S=S, H=H)
    return pkg.Solver(p, max_obstacles=max(1, max(c["obs"].shape[0] for c in cases)),
                      max_path_pts=max(c["path"].shape[0] for c in cases), max_batch=max_batch, **kw)


def _out(d):
    return host_outputs(d)


def test_batch_alone_equals_mix_bitwise(pkg):
    import torch
    dev = torch.device("cuda:0")
    cases = _instances(12)
    s = _ctx(pkg, cases, max_batch=16)
    try:
        mix = [_device_inst(c, dev) for c in cases]
        s.solve_batch(mix)
        torch.cuda.synchronize()
        for i, c in enumerate(cases):
            one = [_device_inst(c, dev)]
            s.solve_batch(one)
            torch.cuda.synchronize()
            a, b = _out(mix[i]), _out(one[0])
            assert a["status"] == 0 and b["status"] == 0
            for k in ("U", "traj", "J", "U_next"):
                assert np.array_equal(a[k], b[k]), (i, k)
    finally:
        s.close()


@pytest.mark.parametrize("tps", [1, 2, 4])
def test_batch_matches_oracle(pkg, tps):
    import torch
    dev = torch.device("cuda:0")
    cases = _instances(6, seed=7)
    s = _ctx(pkg, cases, max_batch=8, batch_threads_per_sample=tps,
             batch_block_threads=max(64, 16 * tps))
    try:
        insts = [_device_inst(c, dev) for c in cases]
        s.solve_batch(insts)
        torch.cuda.synchronize()
        for c, d in zip(cases, insts):
            p = sc.as_float32(c["params"])
            ref = oracle.solve(p, c["x0"], c["U_nom"], c["obs"], c["path"], c["ds"], c["seed"],
                               c["counter"], want_uhist=True)
            out = _out(d)
            assert out["status"] == 0
            assert_solve_matches(out, ref, p, f"batch tps={tps}")
            np.testing.assert_array_equal(out["U_next"], np.vstack([out["U"][1:], out["U"][-1:]]))
    finally:
        s.close()


def test_batch_matches_plain_solves(pkg):
    # the same solves one launch each (plain path, its own launch shape) and
    # in one batch: equal within the parity tolerance (both against the oracle)
    import torch
    dev = torch.device("cuda:0")
    cases = _instances(4, seed=9)
    s = _ctx(pkg, cases, max_batch=4)
    try:
        insts = [_device_inst(c, dev) for c in cases]
        s.solve_batch(insts)
        torch.cuda.synchronize()
        for c, d in zip(cases, insts):
            plain = pkg.Solver(c["params"], max_obstacles=max(1, c["obs"].shape[0]),
                               max_path_pts=c["path"].shape[0])
            try:
                po = device_solve(plain, c)
            finally:
                plain.close()
            p = sc.as_float32(c["params"])
            ref = oracle.solve(p, c["x0"], c["U_nom"], c["obs"], c["path"], c["ds"], c["seed"],
                               c["counter"], want_uhist=True)
            assert_solve_matches(po, ref, p, "plain")
            assert_solve_matches(_out(d), ref, p, "batch")
    finally:
        s.close()


def test_graph_replay_tracks_updated_inputs(pkg):
    import torch
    dev = torch.device("cuda:0")
    cases = _instances(5, seed=11)
    s = _ctx(pkg, cases, max_batch=8)
    try:
        insts = [_device_inst(c, dev) for c in cases]
        g = s.capture_batch(insts)
        try:
            for rep in range(3):
                # move every vehicle a little (inputs updated in place)
                for d in insts:
                    d["x0"][0] += 0.05
                assert pkg.brmppi_graph_launch(g) == 0
                torch.cuda.synchronize()
                got = [_out(d) for d in insts]
                fresh = [_device_inst(c, dev) for c in cases]
                for f, d in zip(fresh, insts):
                    f["x0"].copy_(d["x0"])
                s.solve_batch(fresh)
                torch.cuda.synchronize()
                for a, f in zip(got, fresh):
                    b = _out(f)
                    assert np.array_equal(a["U"], b["U"]) and np.array_equal(a["J"], b["J"])
        finally:
            pkg.brmppi_graph_destroy(g)
    finally:
        s.close()


def test_batch_rejects_bad_instances(pkg):
    import torch
    dev = torch.device("cuda:0")
    cases = _instances(2, seed=13)
    s = _ctx(pkg, cases, max_batch=2)
    try:
        insts = [_device_inst(c, dev) for c in cases]
        assert s.solve_batch(insts + insts[:1], check=False) == pkg.BRMPPI_EINVAL  # > max_batch
        big = dict(insts[0], S=int(s.S) + 1)
        assert s.solve_batch([big], check=False) == pkg.BRMPPI_EINVAL
        assert s.solve_batch(insts) == 0
        torch.cuda.synchronize()
    finally:
        s.close()


def test_autotune_keeps_results_within_tolerance(pkg):
    import torch
    dev = torch.device("cuda:0")
    c = sc.small_random(21, S=700, H=18, n_obs=6)
    s = pkg.Solver(c["params"], max_obstacles=8, max_path_pts=1024)
    try:
        d = _device_inst(c, dev)
        s.autotune(d["x0"], d["U_nom"], d["obs"], d["path"], c["ds"], reps=2)
        launch = s.launch(6)
        out = device_solve(s, c)
        p = sc.as_float32(c["params"])
        ref = oracle.solve(p, c["x0"], c["U_nom"], c["obs"], c["path"], c["ds"], c["seed"],
                           c["counter"], want_uhist=True)
        assert_solve_matches(out, ref, p, f"autotuned {launch}")
    finally:
        s.close()
