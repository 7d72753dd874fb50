"""Seeded synthetic inputs for the K-cycle orthonormalization multigrid solve.

This package produces INPUTS only: the symmetric weighted interior-penalty (SWIP/SIPG)
block matrix of -div(nu grad u) = f on a Cartesian cell grid, the 2^d agglomeration
prolongation matrices of the cell hierarchy, the cell-wise coefficient field and seeded
right-hand sides.  It contains none of the solver's arithmetic (no operator application,
smoothing, orthonormalization, transfer, Galerkin product or coarse solve).  Both the CUDA
path and the CPU oracle consume what it returns; neither is imported here.
"""
from .sipg import (Problem, modes, reference_matrices, prolongation_matrices, assemble,
                   nu_field, make_problem, dense_matrix, eval_field, project,
                   neighbours)
from .configs import WORKLOADS, Workload, workload

__all__ = ["Problem", "modes", "reference_matrices", "prolongation_matrices", "assemble",
           "nu_field", "make_problem", "dense_matrix", "eval_field", "project",
           "neighbours", "WORKLOADS",
           "Workload", "workload"]
