"""Full FP64 oracle solves spread over the host cores (test infrastructure).

A solve's samples are independent until the update (Sec. II-B), so the
oracle's rollouts of one solve run as sample ranges in worker processes
(`oracle.rollouts`) and are joined in sample order by the oracle's own
update (`oracle.update`): the result is bit-identical to `oracle.solve`.
Workers are spawned (a forked child of a process that has touched CUDA can
hang) and import the oracle once.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

CHUNK = 1024  # samples per task


def _work(task):
    """One sample range: the oracle's costs and applied inputs, and, when
    the GPU's states of the same samples are given, the largest relative
    state error against the oracle's rollouts (computed here so that the
    oracle's states never leave the worker)."""
    p, x0, U_nom, obs, path, ds, seed, counter, s0, s1, gpu_states = task
    import oracle
    r = oracle.rollouts(p, x0, U_nom, obs, path, ds, seed, counter, s0, s1, want_uhist=True,
                        want_states=gpu_states is not None)
    out = dict(J=r["J"], u_hist=r["u_hist"], status=r["status"], err_states=None)
    if gpu_states is not None:
        o = r["states"]
        g = np.asarray(gpu_states, np.float64)
        out["err_states"] = float(np.max(np.abs(g - o) / np.maximum(np.abs(o), 1.0)))
    return out


class OraclePool:
    """`with OraclePool() as pool: ref = pool.solve(c, p)`."""

    def __init__(self, processes: int | None = None):
        self.processes = processes or os.cpu_count() or 1
        self.pool = None

    def __enter__(self):
        self.pool = mp.get_context("spawn").Pool(self.processes)
        return self

    def __exit__(self, *exc):
        self.pool.close()
        self.pool.join()
        self.pool = None

    @staticmethod
    def _tasks(c, p, S, gpu_states=None, chunk=CHUNK):
        for s0 in range(0, S, chunk):
            s1 = min(S, s0 + chunk)
            st = None if gpu_states is None else np.asarray(gpu_states[s0:s1])
            yield (p, c["x0"], c["U_nom"], c["obs"], c["path"], c["ds"], c["seed"], c["counter"], s0, s1, st)

    @staticmethod
    def _join(c, p, parts):
        import oracle
        J = np.concatenate([r["J"] for r in parts])
        uh = np.concatenate([r["u_hist"] for r in parts])
        status = next((r["status"] for r in parts if r["status"] != 0), 0)
        st, U, _ = oracle.update(J, uh, float(p["lambda"]), c["U_nom"])
        traj = oracle.integrate(p, c["x0"], U)
        errs = [r["err_states"] for r in parts if r["err_states"] is not None]
        return dict(U=U, traj=traj, J=J, u_hist=uh, status=status or st,
                    err_states=max(errs) if errs else None)

    def solve(self, c, p, gpu_states=None):
        """The full solve of scenario c under params p (as oracle.solve with
        want_uhist=True); with gpu_states (S, H+1, 7), also `err_states`."""
        S = int(p["S"])
        parts = self.pool.map(_work, list(self._tasks(c, p, S, gpu_states)), chunksize=1)
        return self._join(c, p, parts)

    def solve_many(self, cases):
        """Full solves of several (c, p) pairs; yields (index, result) in
        order, each as soon as its sample ranges are done."""
        tasks, owner = [], []
        for i, (c, p) in enumerate(cases):
            for t in self._tasks(c, p, int(p["S"])):
                tasks.append(t)
                owner.append(i)
        pending, cur = [], 0
        for k, r in enumerate(self.pool.imap(_work, tasks, chunksize=1)):
            pending.append(r)
            if k + 1 == len(tasks) or owner[k + 1] != cur:
                c, p = cases[cur]
                yield cur, self._join(c, p, pending)
                pending = []
                cur = owner[k + 1] if k + 1 < len(tasks) else cur
