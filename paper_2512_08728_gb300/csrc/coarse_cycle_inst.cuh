// Instantiation of the persistent coarse-cycle kernel (coarse_cycle.cuh) for one precision
// form.  The including translation unit defines CC_TV (vectors, basis, residual
// minimisation), CC_T (smoother sweeps) and CC_TI (stored block inverses); one
// translation unit per form keeps the build parallel.
#pragma once
#include "coarse_cycle.cuh"

namespace kcmg {

#define KCMG_CC_SWITCH(np, dim, ...)                                   \
  switch (np * 10 + dim) {                                             \
    case 32: { constexpr int NP = 3, DIM = 2; __VA_ARGS__; } break;    \
    case 62: { constexpr int NP = 6, DIM = 2; __VA_ARGS__; } break;    \
    case 102: { constexpr int NP = 10, DIM = 2; __VA_ARGS__; } break;  \
    case 43: { constexpr int NP = 4, DIM = 3; __VA_ARGS__; } break;    \
    case 103: { constexpr int NP = 10, DIM = 3; __VA_ARGS__; } break;  \
    case 203: { constexpr int NP = 20, DIM = 3; __VA_ARGS__; } break;  \
    default: break;                                                    \
  }

static void* coarse_kernel_ptr(int np, int dim) {
  void* f = nullptr;
  KCMG_CC_SWITCH(np, dim, { f = (void*)k_coarse_cycle<CC_TV, CC_T, CC_TI, NP, DIM>; });
  return f;
}

static size_t coarse_cycle_smem(int np, int dim, int threads) {
  // prolongation matrices (CC_TV), the smoother tile (threads x CC_T), and one gathered
  // patch residual per warp for the Schwarz smoother ((threads / 32) x 2^d np x CC_T)
  return (size_t)(1 << dim) * np * np * sizeof(CC_TV) + (size_t)threads * sizeof(CC_T) +
         (size_t)(threads / 32) * (1 << dim) * np * sizeof(CC_T);
}

template <>
cudaError_t coarse_cycle_grid<CC_TV, CC_T, CC_TI>(int np, int dim, int threads, int* grid) {
  void* f = coarse_kernel_ptr(np, dim);
  if (!f) return cudaErrorInvalidValue;
  int per_sm = 0, dev = 0, nsm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, threads,
                                                                coarse_cycle_smem(np, dim, threads));
  if (e != cudaSuccess) return e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  *grid = nsm;  // one resident block per SM: measured faster than two (fewer barrier arrivals)
  return cudaSuccess;
}

template <>
cudaError_t launch_coarse_cycle<CC_TV, CC_T, CC_TI>(const CoarseArgs& a, int grid, int threads, cudaStream_t s) {
  void* f = coarse_kernel_ptr(a.np, a.dim);
  if (!f) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = coarse_cycle_smem(a.np, a.dim, threads);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* args[] = {const_cast<CoarseArgs*>(&a)};
  return cudaLaunchKernelExC(&cfg, f, args);
}

}  // namespace kcmg
