// Persistent coarse-cycle kernel, mixed form: FP32 smoother sweeps and inverses, FP64 vectors and minimisation.
#define CC_TV double
#define CC_T float
#define CC_TI float
#include "coarse_cycle_inst.cuh"
