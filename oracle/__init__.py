"""CPU oracle of the K-cycle orthonormalization multigrid solve (plain FP64 C).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU-baseline leg
use it; the product path never imports, loads or calls anything here.  It shares no code
with the CUDA library.  See kcmg_oracle.c for what each routine follows in the paper
(Alg. 1 residual minimization, Alg. 2 orthonormalization multigrid, Alg. BJ block Jacobi,
Sec. 4.2 level-local convergence criteria).

Parity pins (tests/test_oracle.py): dense LU on small meshes, GMRES/GCR equivalence of
Alg. 1 with z := r, the closed form of damped block-Jacobi sweeps, W^T W = I and A Z = W,
monotone residuals, manufactured solutions, P^T P = I and polynomial reproduction of the
transfers, the Galerkin energy identity, and central finite differences of the adjoint
gradient.
"""
from .oracle import (OracleSolver, build, grad_lognu, default_level_criteria, threads,
                     ORC_OK, ORC_NOT_CONVERGED, ORC_BREAKDOWN, ORC_NONFINITE, ORC_SINGULAR,
                     ORC_INVALID_ARG)

__all__ = ["OracleSolver", "build", "grad_lognu", "default_level_criteria", "threads", "ORC_OK",
           "ORC_NOT_CONVERGED", "ORC_BREAKDOWN", "ORC_NONFINITE", "ORC_SINGULAR",
           "ORC_INVALID_ARG"]
