// Block reductions shared by the kernel translation units of libkcmg.
#pragma once
#include <cuda_runtime.h>

namespace kcmg {

// Warp sums of NC values (NC a power of two, <= 32) by transposition: each exchange with
// partner lane^off halves the set of values a lane carries (a lane keeps one half and adds
// the partner's copy of it), so NC values take NC - 1 + log2(32 / NC) FP64 additions per
// lane instead of 5 NC.  FP64 adds are scarce on this GPU (about two per SM and clock).
// Returns the full warp sum of value *idx, held by all 32 / NC lanes of a group.
template <int NC>
static __device__ __forceinline__ double warp_sum_t(const double (&v)[NC], int lane, int& idx) {
  double cur[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) cur[c] = v[c];
  int base = 0;
  int off = 16;
#pragma unroll
  for (int half = NC / 2; half >= 1; half /= 2, off >>= 1) {
    const bool hi = (lane & off) != 0;
#pragma unroll
    for (int k = 0; k < half; ++k) {
      const double mine = hi ? cur[half + k] : cur[k];
      const double give = hi ? cur[k] : cur[half + k];
      cur[k] = mine + __shfl_xor_sync(0xffffffffu, give, off);
    }
    if (hi) base += half;
  }
  double s = cur[0];
  for (; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  idx = base;
  return s;
}

// NC block sums at once (one shared-memory exchange): results valid in thread 0.
// The order of every addition is fixed, so the sums are reproducible.
// sh: >= 32 * NC doubles.
template <int NC>
static __device__ __forceinline__ void bsum_n(double (&v)[NC], double* sh) {
  const int w = threadIdx.x >> 5, ln = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
  int idx = 0;
  const double s = warp_sum_t<NC>(v, ln, idx);
  __syncthreads();
  if ((ln & (32 / NC - 1)) == 0) sh[idx * 32 + w] = s;
  __syncthreads();
  if (w == 0) {
    double t = 0.0;
    if (ln < NC)
      for (int k = 0; k < nw; ++k) t += sh[ln * 32 + k];
#pragma unroll
    for (int c = 0; c < NC; ++c) v[c] = __shfl_sync(0xffffffffu, t, c);
  }
}

}  // namespace kcmg
