"""Costs of a served solve, for the update check of `tests/parity.py`.

The serving loop returns U* and the optimal trajectory but no per-sample
costs.  It runs the context's batch kernel variant in the batch's default
launch shape, and a solve gives the same bits alone and in any batch on one
context, so the same request solved as a batch of one on that context (with
its cost output) reproduces the served U* bit for bit: that equality is
asserted here, and the batch's costs are then the served solve's costs."""
import numpy as np


def served_costs(solver, c, U0, seed, counter, U_served, x0=None):
    """dict(J, J_lo, u_hist) of the served solve (see the module docstring)."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    S, H = int(solver.S), int(solver.H)
    t = lambda a, dt=torch.float32: torch.as_tensor(np.asarray(a), dtype=dt, device=dev)
    obs = c["obs"]
    inst = dict(x0=t(c["x0"] if x0 is None else x0, torch.float64), U_nom=t(U0),
                obs=t(obs) if len(obs) else None, path=t(c["path"]), ds=c["ds"], S=S, seed=seed,
                counter=counter, U_out=torch.empty((H, 3), device=dev),
                traj_out=torch.empty((H + 1, 7), device=dev), J_out=torch.empty(S, device=dev),
                inputs_out=torch.empty((S, H, 3), device=dev), J_lo_out=torch.empty(S, device=dev))
    solver.solve_batch([inst])
    torch.cuda.synchronize()
    U = inst["U_out"].cpu().numpy()
    assert np.array_equal(U, np.asarray(U_served, np.float32).reshape(U.shape)), \
        "a batch of one on the serving context must reproduce the served U* bit for bit"
    return dict(J=inst["J_out"].cpu().numpy(), J_lo=inst["J_lo_out"].cpu().numpy(),
                u_hist=inst["inputs_out"].cpu().numpy())
