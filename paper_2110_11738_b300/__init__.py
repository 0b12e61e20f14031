"""B300-native (sm_103a) Douglas-Rachford optimal-transport solver (DROT).

The solver itself is the CUDA library built from ``csrc/`` (C ABI in
``include/drot.h``); this package holds that source, the build step and a thin
ctypes binding.  See :mod:`paper_2110_11738_b300.drot`.
"""

from .drot import (  # noqa: F401
    DROT_ERR_CUDA,
    DROT_ERR_INVALID_ARG,
    DROT_ERR_MARGINALS,
    DROT_ERR_NONFINITE,
    DROT_ERR_OOM,
    DROT_ERR_TIMEOUT,
    DROT_NOT_CONVERGED,
    DROT_OK,
    DrotError,
    Solver,
    drot_create,
    drot_destroy,
    drot_get_profile,
    drot_reset_profile,
    drot_solve,
    drot_solve_batched,
    load,
    padded_matrix,
)
