// Persistent coarse-cycle kernel, mixed form with BF16-stored block inverses.
#define CC_TV double
#define CC_T float
#define CC_TI __nv_bfloat16
#include "coarse_cycle_inst.cuh"
