"""Full-size parity: the two largest workloads solved on the GPU in the
launch shapes the bench times, against full FP64 oracle solves spread over
the host cores (`tests/oracle_pool.py`; bit-identical to `oracle.solve`).

* Stress solve (S = 65536, H = 100, 64 ellipses, 2401 path rows) with the
  stored-trajectory variant: every sample's cost and every sample's state
  trajectory, U* (update check at a flat 1e-4 on the GPU's costs) and the
  optimal trajectory.
* The 256 uneven solves of the batched workload in one persistent launch
  (one lane per sample, 256 threads, capacity 16 obstacles): every
  instance's costs, U* and optimal trajectory.
"""
import numpy as np
import pytest

from paper_2508_05773_gb300 import scenarios as sc
from tests.gpu_solve import device_tensors, host_outputs
from tests.oracle_pool import OraclePool
from tests.parity import TOL_STATE, assert_solve_matches

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def pool():
    # spawned before this module's first GPU call
    with OraclePool() as p:
        yield p


@pytest.fixture(scope="module")
def pkg(pool):
    from paper_2508_05773_gb300 import build as native_build
    native_build.build()
    import paper_2508_05773_gb300
    paper_2508_05773_gb300.load()
    return paper_2508_05773_gb300


def test_config5_every_sample(pkg, pool):
    import torch
    dev = torch.device("cuda:0")
    c = sc.config5()
    p = sc.as_float32(c["params"])
    s = pkg.Solver(c["params"], max_obstacles=64, max_path_pts=c["path"].shape[0])
    try:
        d = device_tensors(c, dev, states=True)
        s.solve_device_ex(d)
        torch.cuda.synchronize()
        assert int(d["status"].item()) == 0
        out = host_outputs(d)
        states = d["states_out"].cpu().numpy()
        del d
    finally:
        s.close()
    ref = pool.solve(c, p, gpu_states=states)
    assert ref["status"] == 0
    assert ref["err_states"] <= TOL_STATE, f"stored states rel err {ref['err_states']:.3e}"
    assert_solve_matches(out, ref, p, "config 5 (S=65536, H=100, 64 ellipses)", strict=True)


def test_config3_every_instance(pkg, pool):
    import torch
    dev = torch.device("cuda:0")
    cases = sc.config3()
    Smax = max(int(c["params"]["S"]) for c in cases)
    Hmax = max(int(c["params"]["H"]) for c in cases)
    npts = max(c["path"].shape[0] for c in cases)
    s = pkg.Solver(dict(cases[0]["params"], S=Smax, H=Hmax), max_obstacles=16, max_path_pts=npts,
                   max_batch=len(cases), batch_threads_per_sample=1, batch_block_threads=256)
    try:
        insts = [device_tensors(c, dev) for c in cases]
        s.solve_batch(insts)
        torch.cuda.synchronize()
        assert all(int(d["status"].item()) == 0 for d in insts)
        outs = [host_outputs(d) for d in insts]
        del insts
    finally:
        s.close()
    pairs = [(c, sc.as_float32(c["params"])) for c in cases]
    seen = 0
    for i, ref in pool.solve_many(pairs):
        assert ref["status"] == 0, i
        assert_solve_matches(outs[i], ref, pairs[i][1], f"config-3 instance {i}")
        seen += 1
    assert seen == len(cases)
