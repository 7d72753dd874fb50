// Persistent coarse-cycle kernel, FP64 form: every step in FP64.
#define CC_TV double
#define CC_T double
#define CC_TI double
#include "coarse_cycle_inst.cuh"
