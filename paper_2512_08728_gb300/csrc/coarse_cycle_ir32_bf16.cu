// Persistent coarse-cycle kernel, inner FP32 solve of the iterative-refinement form with BF16-stored block
// inverses.
#define CC_TV float
#define CC_T float
#define CC_TI __nv_bfloat16
#include "coarse_cycle_inst.cuh"
