"""GB300-native BR-MPPI solver (arXiv 2508.05773): the data-parallel hot path
of Barrier-Rate guided MPPI for a tractor-trailer, as sm_103a CUDA behind a C
ABI (``include/brmppi.h``, ``libbrmppi.so``).

``scenarios`` builds seeded synthetic inputs; the C-ABI functions are
re-exported here with their C names.  Importing the package does not load the
library; the first call does, and fails loudly if it has not been built.
"""
from ._native import (  # noqa: F401
    BRMPPI_ABI_VERSION, BRMPPI_EAGAIN, BRMPPI_EBUSY, BRMPPI_ECUDA, BRMPPI_EINVAL, BRMPPI_ENOMEM,
    BRMPPI_ENONFINITE, BRMPPI_ETIMEDOUT, BRMPPI_FLAG_ALPHA_BUFFER, BRMPPI_FLAG_COLLISION_COST, BRMPPI_FLAG_JERK_MODEL,
    BRMPPI_FLAG_OBS8, BRMPPI_FLAG_PROJ_NONE, BRMPPI_FLAG_THIRD_ORDER, BRMPPI_OK, EXPORTS, PIPE_FMA, PIPE_IMAD, PIPE_XU, BrmppiError,
    NativeLibraryMissing, Solver, brmppi_autotune, brmppi_autotune_batch, brmppi_batch_capture,
    brmppi_create, brmppi_default_params, brmppi_destroy, brmppi_get_batch_launch, brmppi_get_launch,
    brmppi_graph_destroy, brmppi_graph_launch, brmppi_hitch_stabilize_device, brmppi_inject_alloc_failure,
    brmppi_instance,
    brmppi_last_error, brmppi_measure_pipe, brmppi_noise_blocks, brmppi_params, brmppi_poll, brmppi_server_stats, brmppi_server_stats_get,
    brmppi_solve, brmppi_solve_batch, brmppi_solve_device, brmppi_solve_device_ex,
    brmppi_merge_tiles, brmppi_solve_device_noalloc, brmppi_solve_tiles, brmppi_submit, brmppi_tile_layout,
    brmppi_transfer_bytes, brmppi_vehicle_export,
    brmppi_vehicle_import, brmppi_vehicle_register, load, make_instances, params_from_dict,
)
from . import scenarios  # noqa: F401
from .sharded import rank_tiles, solve_sharded  # noqa: F401
