// Persistent coarse-cycle kernel, inner FP32 solve of the iterative-refinement form: FP32 vectors, operators,
// sweeps and inverses; FP64 reductions and Gram coefficients.
#define CC_TV float
#define CC_T float
#define CC_TI float
#include "coarse_cycle_inst.cuh"
