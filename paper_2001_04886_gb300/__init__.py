"""GB300 s-step Orthomin / s-step GMRES: Python binding of the C ABI in include/sstep.h.

Every function here only marshals arguments (tensor data pointers, sizes and
the current CUDA stream) into one call of libsstep.so; all arithmetic runs in
the library's CUDA kernels. There is no CPU fallback: if the library is not
built, the first call raises.

Importing the package loads nothing; `inputs` (seeded synthetic inputs) can be
used without a GPU.
"""
from __future__ import annotations

from ._binding import (  # noqa: F401
    BatchSolver,
    X0Net,
    SSTEP_MAX_COLS,
    SSTEP_MAX_M,
    SSTEP_MAX_S,
    SStepError,
    StencilMatrix,
    gmres_solve,
    lib,
    sstep_block_update,
    sstep_gmres_solve,
    set_tc_wait_limit,
    sstep_gram,
    sstep_gram_tc,
    sstep_gram_workspace_size,
    sstep_matrix_powers,
    sstep_newton_shifts,
    sstep_omin_solve,
    stencil_matrix_apply,
    stencil_matrix_smooth,
    stencil_matrix_smooth_batched,
    trace_enable,
    trace_read,
    trace_select,
    x0net_features,
    x0net_targets,
)

__all__ = [
    "BatchSolver",
    "X0Net",
    "StencilMatrix",
    "stencil_matrix_apply",
    "stencil_matrix_smooth",
    "stencil_matrix_smooth_batched",
    "sstep_matrix_powers",
    "sstep_gram",
    "sstep_gram_tc",
    "set_tc_wait_limit",
    "sstep_gram_workspace_size",
    "sstep_block_update",
    "sstep_gmres_solve",
    "gmres_solve",
    "sstep_omin_solve",
    "sstep_newton_shifts",
    "SStepError",
    "trace_enable",
    "trace_read",
    "trace_select",
    "x0net_features",
    "x0net_targets",
    "lib",
]
