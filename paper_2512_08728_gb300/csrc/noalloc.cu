// kcmg_residual_noalloc: the residual r = b - A x of the finest-level FP64 operator and its
// norm, for callers that must not allocate device memory.
//
// Which callers cannot allocate: processes whose device memory is already claimed, for
// example by a framework's caching allocator that holds most of the free memory (a
// cudaMalloc there fails or forces the framework to release its cache), code that runs
// under a fixed device-memory budget, and error-recovery paths that run after an
// out-of-memory failure.  They still build a context once with kcmg_setup (which
// allocates); this call then needs nothing beyond the caller's buffers.
//
// The regular residual kernel keeps its per-block partial sums and its reduction counter
// in buffers the context allocates.  This variant keeps them in one file-scope static
// device array instead, so the call itself allocates nothing (no cudaMalloc, no cudaFree,
// no allocating library routine).  kcmg_setup looks up the array's device address (with
// the context's device current) and loads this file's kernels, so that a later call does
// no set-up of its own.  The call reads ||r|| into host memory and synchronises the
// context's stream before it returns.
#include "kcmg_internal.h"

#include <mutex>

namespace kcmg {

// Scratch of the no-allocation residual: [0, kNoallocMaxBlocks) block partial sums, then
// the norm, then the reduction counter.  Every GPU that loads the library holds it (257 KB)
// until the process exits.  All calls share it and it keeps the last call's contents.
constexpr int kNoallocMaxBlocks = 32768;
constexpr int kNoallocDoubles = kNoallocMaxBlocks + 64;
static __device__ __align__(256) double g_noalloc_scratch[kNoallocDoubles];

namespace {

__device__ __forceinline__ double na_block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
  __syncthreads();
  if (ln == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = (ln < (int)((blockDim.x + 31) >> 5)) ? sh[ln] : 0.0;
#pragma unroll
    for (int o = 16; o; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  }
  return r;
}

// r = b - A x with ||r||^2 reduced through the static scratch.  One thread per DOF row,
// plain FP64 fused multiply-adds over the row's slots: r equals the plain FP64 operator
// application b - A x of the library's operator kernel to rounding (the solver's own
// level-0 residual is compensated, double-double, and may differ in the last bits).
template <int NP, int S>
__global__ void __launch_bounds__(320)
k_residual_noalloc(const double* __restrict__ A, const int* __restrict__ nbr, int N, int G,
                   const double* __restrict__ x, const double* __restrict__ b, double* __restrict__ r,
                   double* scratch) {
  constexpr int JP = (NP + 1) / 2;
  constexpr int NF = S - 1;
  __shared__ double sh[32];
  __shared__ int s_last;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  const int g = row >> 5, lane = row & 31;
  double out = 0.0;
  if (row < N) {
    const int K = row / NP;
    double acc = 0.0;
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const int J = (s == 0) ? K : __ldg(nbr + (size_t)K * NF + s - 1);
      if (J < 0) continue;
      const double2* Ap = reinterpret_cast<const double2*>(A) + ((size_t)(s * G + g) * JP) * 32 + lane;
      const double* xp = x + (size_t)J * NP;
#pragma unroll
      for (int jp = 0; jp < JP; ++jp) {
        const double2 a = __ldg(Ap + jp * 32);
        acc = fma(a.x, __ldg(xp + 2 * jp), acc);
        if (2 * jp + 1 < NP) acc = fma(a.y, __ldg(xp + 2 * jp + 1), acc);
      }
    }
    out = b[row] - acc;
    r[row] = out;
  }
  const double part = na_block_sum(out * out, sh);
  unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + kNoallocMaxBlocks + 1);
  if (threadIdx.x == 0) {
    scratch[blockIdx.x] = part;
    __threadfence();
    s_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (s_last) {   // last block: fixed-order sum of the partials, then reset the counter
    double t = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) t += __ldcg(scratch + i);
    t = na_block_sum(t, sh);
    if (threadIdx.x == 0) {
      scratch[kNoallocMaxBlocks] = sqrt(t);
      *counter = 0u;
    }
  }
}

// device address of the scratch, looked up once per device
std::mutex g_na_mutex;
void* g_na_ptr[256] = {};

}  // namespace

cudaError_t noalloc_prepare(int dev, double** scratch) {
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return e;
  if (cur != dev) return cudaErrorInvalidDevice;   // the caller makes dev current
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    // the host-side name of the array is not a device address: ask the runtime for it
    if ((e = cudaGetSymbolAddress(&p, g_noalloc_scratch)) != cudaSuccess) return e;
    // load the kernels now (lazy module loading would otherwise do it at the first call)
    cudaFuncAttributes fa;
    const void* fns[] = {(const void*)k_residual_noalloc<3, 5>, (const void*)k_residual_noalloc<6, 5>,
                         (const void*)k_residual_noalloc<10, 5>, (const void*)k_residual_noalloc<4, 7>,
                         (const void*)k_residual_noalloc<10, 7>, (const void*)k_residual_noalloc<20, 7>};
    for (const void* f : fns)
      if ((e = cudaFuncGetAttributes(&fa, f)) != cudaSuccess) return e;
    g_na_ptr[dev] = p;
  }
  *scratch = static_cast<double*>(g_na_ptr[dev]);
  return cudaSuccess;
}

cudaError_t residual_noalloc(const Level0View& v, const double* b, const double* x, double* r,
                             double* rnorm_host, int* too_large) {
  const int grid = v.rows_pad / v.block_rows;
  *too_large = grid > kNoallocMaxBlocks;
  if (*too_large) return cudaSuccess;
  double* scratch = v.scratch;
  if (!scratch) return cudaErrorInvalidValue;
  cudaError_t e;
  // the counter must start at zero (the previous call may have been interrupted)
  if ((e = cudaMemsetAsync(scratch + kNoallocMaxBlocks + 1, 0, sizeof(double), v.stream)) != cudaSuccess) return e;
  switch (v.np * 10 + v.dim) {
    case 32: k_residual_noalloc<3, 5><<<grid, v.block_rows, 0, v.stream>>>(v.A, v.nbr, v.N, v.G, x, b, r, scratch); break;
    case 62: k_residual_noalloc<6, 5><<<grid, v.block_rows, 0, v.stream>>>(v.A, v.nbr, v.N, v.G, x, b, r, scratch); break;
    case 102: k_residual_noalloc<10, 5><<<grid, v.block_rows, 0, v.stream>>>(v.A, v.nbr, v.N, v.G, x, b, r, scratch); break;
    case 43: k_residual_noalloc<4, 7><<<grid, v.block_rows, 0, v.stream>>>(v.A, v.nbr, v.N, v.G, x, b, r, scratch); break;
    case 103: k_residual_noalloc<10, 7><<<grid, v.block_rows, 0, v.stream>>>(v.A, v.nbr, v.N, v.G, x, b, r, scratch); break;
    case 203: k_residual_noalloc<20, 7><<<grid, v.block_rows, 0, v.stream>>>(v.A, v.nbr, v.N, v.G, x, b, r, scratch); break;
    default: return cudaErrorInvalidValue;
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(rnorm_host, scratch + kNoallocMaxBlocks, sizeof(double), cudaMemcpyDeviceToHost,
                           v.stream)) != cudaSuccess)
    return e;
  return cudaStreamSynchronize(v.stream);
}

}  // namespace kcmg
