"""GB300-native K-cycle orthonormalization multigrid (Toprak & Kummer, Alg. 1 and 2).

The solve runs in hand-written sm_103a CUDA kernels behind the C interface of
include/kcmg.h (libkcmg.so, built in-tree by build.build()); kcmg.py is the thin Python
binding and autograd.py the torch.autograd wrapper.  Importing the package does not load
the library; the first call does, and raises if it is missing.
"""
from .build import build
from .kcmg import (KCycleSolver, KcmgError, kcmg_apply, kcmg_coarse_solve, kcmg_default_params,
                   kcmg_destroy, kcmg_get_blocks, kcmg_grad_lognu, kcmg_level_cells,
                   kcmg_prolong, kcmg_restrict, kcmg_rm_sequence, kcmg_setup, kcmg_smooth,
                   kcmg_solve, kcmg_solve_adjoint, kcmg_residual_noalloc, kcmg_apply_multi,
                   kcmg_smooth_multi, kcmg_mrhs_tuning, load_library)

__all__ = ["build", "KCycleSolver", "KcmgError", "kcmg_apply", "kcmg_coarse_solve",
           "kcmg_default_params", "kcmg_destroy", "kcmg_get_blocks", "kcmg_grad_lognu",
           "kcmg_level_cells", "kcmg_prolong", "kcmg_restrict", "kcmg_rm_sequence",
           "kcmg_setup", "kcmg_smooth", "kcmg_solve", "kcmg_solve_adjoint",
           "kcmg_residual_noalloc", "kcmg_apply_multi", "kcmg_smooth_multi",
           "kcmg_mrhs_tuning", "load_library"]
