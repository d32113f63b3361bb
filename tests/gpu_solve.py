"""One GPU solve with every output the parity checks use, through the
device-instance entry point (brmppi_solve_device_ex): U*, the optimal
trajectory, status, each sample's cost as the compensated pair the softmin
uses (J high parts, J_lo low parts) and each sample's applied inputs
(u_hist, S x H x 3).  It runs the same kernel variant and launch shape as
the host entry point brmppi_solve on the same context."""
import numpy as np


def device_tensors(c, dev, x0=None, U_nom=None, states=False, inputs=True):
    import torch
    S, H = int(c["params"]["S"]), int(c["params"]["H"])
    t = lambda a, dt=torch.float32: torch.as_tensor(np.asarray(a), dtype=dt, device=dev)
    d = dict(x0=t(c["x0"] if x0 is None else x0, torch.float64), U_nom=t(c["U_nom"] if U_nom is None else U_nom),
             obs=t(c["obs"]) if len(c["obs"]) else None, path=t(c["path"]), ds=c["ds"], S=S,
             seed=c["seed"], counter=c["counter"], U_out=torch.empty((H, 3), device=dev),
             traj_out=torch.empty((H + 1, 7), device=dev), J_out=torch.empty(S, device=dev),
             status=torch.full((1,), 99, dtype=torch.int32, device=dev))
    if inputs:
        d["inputs_out"] = torch.empty((S, H, 3), device=dev)
        d["J_lo_out"] = torch.empty(S, device=dev)
    if states:
        d["states_out"] = torch.empty((S, H + 1, 7), device=dev)
    return d


def add_cost_outputs(d, S, H):
    """Give an instance dict the per-sample outputs of the parity checks."""
    import torch
    dev = d["U_out"].device
    d["inputs_out"] = torch.empty((int(S), int(H), 3), device=dev)
    d["J_lo_out"] = torch.empty(int(S), device=dev)
    return d


def host_outputs(d):
    out = dict(U=d["U_out"].cpu().numpy(), traj=d["traj_out"].cpu().numpy(), J=d["J_out"].cpu().numpy())
    if d.get("status") is not None:
        out["status"] = int(d["status"].item())
    if d.get("inputs_out") is not None:
        out["u_hist"] = d["inputs_out"].cpu().numpy()
        out["J_lo"] = d["J_lo_out"].cpu().numpy()
    if d.get("U_next") is not None:
        out["U_next"] = d["U_next"].cpu().numpy()
    return out


def device_solve(solver, c, x0=None, U_nom=None, counter=None):
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    d = device_tensors(c, dev, x0=x0, U_nom=U_nom)
    if counter is not None:
        d["counter"] = counter
    solver.solve_device_ex(d)
    torch.cuda.synchronize()
    return host_outputs(d)
