"""Seeded synthetic inputs for the octree-block multigrid workloads.

This package holds input generators only: leaf lists of octree forests (uniform, sphere-refined, box-refined,
2:1-balanced) and cell-centred fields (manufactured right-hand sides, Gaussian bumps with noise, log-normal
coefficients from a Gaussian random field, target fields for the adjoint loss, Dirichlet data at boundary face
centres).  It contains none of the
multigrid method's arithmetic, and both the CUDA path's tests and the CPU oracle take their inputs from here.
"""
from .forests import (uniform_leaves, refine_ball, refine_box, balance_2to1, leaves_array, leaf_keys,
                      count_cells, workload_forest, batch_problems, batch_leaves, paper_benchmark_forest)
from .fields import (cell_centres, sin_product, sin_product_rhs, gaussian_bump_with_noise, lognormal_k_rff,
                     uniform_rhs, sin_target, batch_fields, boundary_values)

__all__ = [
    "uniform_leaves", "refine_ball", "refine_box", "balance_2to1", "leaves_array", "leaf_keys", "count_cells",
    "workload_forest", "batch_problems", "batch_leaves", "paper_benchmark_forest", "cell_centres", "sin_product", "sin_product_rhs", "gaussian_bump_with_noise",
    "lognormal_k_rff", "uniform_rhs", "sin_target", "batch_fields", "boundary_values",
]
