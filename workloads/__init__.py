"""Seeded synthetic inputs for DROT (cost matrices, marginals, starting states).

This package holds input generation only: point clouds, squared-Euclidean cost
matrices, marginals and random starting states.  It contains none of the
Douglas-Rachford arithmetic, so both the CUDA path and the CPU oracle can draw
their inputs from it.
"""

from .synthetic import (  # noqa: F401
    CONFIGS,
    Problem,
    make_problem,
    make_batch,
    random_start,
    mlp_init_params,
    sq_euclidean_cost_np,
    sq_euclidean_cost_torch,
    default_rho,
    pad_ld,
)
