"""One solve partitioned by samples over the ranks of a torch.distributed
process group (one GPU per rank).

The softmin and the update (paper Sec. II-B, Eq. MPPI_update_rule) need
every sample's cost, so the path's one exchange is there: the samples are
cut into the tiles of the context's plain launch shape, rank r rolls out a
contiguous range of them (``brmppi_solve_tiles``), the ranks all-gather the
tile partials (one collective of n_tiles x tile_floats floats: 80 KB for the
paper-scale solve), and every rank merges the complete set in tile order
(``brmppi_merge_tiles``).  That is the merge a single launch ends with, over
the same tiles in the same order, so every rank's U*, optimal trajectory and
warm start equal the one-GPU solve bit for bit.

All arithmetic runs in the library's kernels; this module only splits the
tile range and moves the partials.
"""
from __future__ import annotations


def rank_tiles(n_tiles: int, world: int, rank: int):
    """(first tile, tile count) of `rank`: contiguous ranges in rank order,
    the first n_tiles % world ranks one tile longer."""
    base, extra = divmod(int(n_tiles), int(world))
    count = base + (1 if rank < extra else 0)
    first = rank * base + min(rank, extra)
    return first, count


class _Native:
    """The library calls this module makes (replaceable in host-only tests)."""

    @staticmethod
    def tile_layout(ctx, inst):
        from . import _native
        return _native.brmppi_tile_layout(ctx, inst)

    @staticmethod
    def solve_tiles(ctx, inst, tile0, n_tiles, tiles_out, stream):
        from . import _native
        st = _native.brmppi_solve_tiles(ctx, inst, tile0, n_tiles, tiles_out, stream)
        if st != _native.BRMPPI_OK:
            raise _native.BrmppiError(st, _native.brmppi_last_error(ctx))

    @staticmethod
    def merge_tiles(ctx, inst, tiles, stream):
        from . import _native
        st = _native.brmppi_merge_tiles(ctx, inst, tiles, stream)
        if st != _native.BRMPPI_OK:
            raise _native.BrmppiError(st, _native.brmppi_last_error(ctx))


def solve_sharded(solver, inst: dict, group=None, stream=None, native=_Native):
    """Solve `inst` (a dict of device tensors as for ``Solver.solve_device_ex``;
    U_out required on every rank) with its samples split over the ranks of
    `group`.  Collective: every rank calls it with the same inputs and a
    context of the same parameters.  Each rank's cost outputs (J_out,
    J_lo_out, inputs_out, states_out) receive its own samples; U_out,
    traj_out, U_next and status receive the merged solve on every rank.
    Returns (first tile, tile count) of this rank."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    n_tiles, tile_floats = native.tile_layout(solver.ctx, inst)
    counts = [rank_tiles(n_tiles, world, r)[1] for r in range(world)]
    first, count = rank_tiles(n_tiles, world, rank)
    width = max(counts)
    dev = inst["x0"].device
    local = torch.zeros((width, tile_floats), dtype=torch.float32, device=dev)
    if count > 0:
        native.solve_tiles(solver.ctx, inst, first, count, local, stream)
    gathered = [torch.empty_like(local) for _ in range(world)]
    dist.all_gather(gathered, local, group=group)
    tiles = torch.cat([g[:c] for g, c in zip(gathered, counts)]).contiguous()
    native.merge_tiles(solver.ctx, inst, tiles, stream)
    return first, count
