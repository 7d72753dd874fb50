// Device helpers of the additive Schwarz smoother (Alg. AS, Sec. 3.2 of Toprak & Kummer)
// on overlapping cell patches, shared by the per-kernel path (schwarz.cu) and the
// persistent coarse cycle (coarse_cycle.cuh).
//
// Subdomains: the 2^d-cell blocks of two partitions of a level's Cartesian cell grid.
// Partition 0 is aligned with the agglomeration (patch p holds cells 2p + c); partition 1
// is shifted by one cell in every direction (patch p holds cells 2p - 1 + c that lie in the
// grid, so boundary patches hold fewer cells).  Member a = cx + 2 cy + 4 cz.  Every cell
// lies in exactly one patch of each partition; neighbouring patches of the two partitions
// overlap by one cell.  The local matrix of a patch is the block of A that couples its
// members (an absent member gets an identity block and no coupling), of order
// m = 2^d np; its inverse is stored transposed, invT[q * m + j] = (A_i^-1)[j][q].
// One smoothing step: x += omega (z_0 + z_1), z_k the prolongated patch solutions
// A_i^-1 R_i (b - A x) of partition k.
#pragma once
#include "kcmg_internal.h"

namespace kcmg {

// patches per direction of partition part on a grid of n cells (n even)
__host__ __device__ __forceinline__ int as_patches_1d(int n, int part) { return n / 2 + part; }

__host__ __device__ __forceinline__ int as_npatch(const int* n, int dim, int part) {
  int c = as_patches_1d(n[0], part) * as_patches_1d(n[1], part);
  if (dim == 3) c *= as_patches_1d(n[2], part);
  return c;
}

// member cells of patch pi of partition part (-1 = outside the grid)
template <int DIM>
__device__ __forceinline__ void as_members(const int* n, int part, int pi, int* cell) {
  constexpr int NCH = 1 << DIM;
  const int p0 = as_patches_1d(n[0], part), p1 = as_patches_1d(n[1], part);
  const int pc[3] = {pi % p0, (pi / p0) % p1, DIM == 3 ? pi / (p0 * p1) : 0};
#pragma unroll
  for (int a = 0; a < NCH; ++a) {
    int c[3] = {0, 0, 0};
    bool in = true;
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      c[j] = 2 * pc[j] - part + ((a >> j) & 1);
      if (c[j] < 0 || c[j] >= n[j]) in = false;
    }
    cell[a] = in ? c[0] + n[0] * (c[1] + n[1] * c[2]) : -1;
  }
}

// one stored inverse entry in the arithmetic type T (FP64 and FP32 loads at full width)
template <typename T, typename TI> struct AsLoad {
  static __device__ __forceinline__ T get(const TI* p) { return (T)__ldg(p); }
};
template <> struct AsLoad<float, __nv_bfloat16> {
  static __device__ __forceinline__ float get(const __nv_bfloat16* p) { return __bfloat162float(*p); }
};

// z (m values of patch pi) = A_i^-1 R_i r for one patch, by one warp.  rs: m values of
// shared memory for the gathered residual.  T: vector type; TI: stored inverse type.
template <typename T, typename TI, int NP, int DIM>
__device__ __forceinline__ void as_patch_solve_warp(const int* n, int part, int pi, const TI* invT,
                                                    const T* r, T* z, T* rs) {
  constexpr int NCH = 1 << DIM, M = NCH * NP, JT = (M + 31) / 32;
  const int lane = threadIdx.x & 31;
  int cell[NCH];
  as_members<DIM>(n, part, pi, cell);
  for (int e = lane; e < M; e += 32) {
    const int a = e / NP, q = e - a * NP;
    rs[e] = cell[a] >= 0 ? __ldcg(r + (size_t)cell[a] * NP + q) : T(0);
  }
  __syncwarp();
  T acc[JT];
#pragma unroll
  for (int t = 0; t < JT; ++t) acc[t] = T(0);
  const TI* Ai = invT + (size_t)pi * M * M;
  for (int q = 0; q < M; ++q) {
    const T rq = rs[q];
#pragma unroll
    for (int t = 0; t < JT; ++t) {
      const int j = lane + 32 * t;
      if (j < M) acc[t] = fma(AsLoad<T, TI>::get(Ai + (size_t)q * M + j), rq, acc[t]);
    }
  }
#pragma unroll
  for (int t = 0; t < JT; ++t) {
    const int j = lane + 32 * t;
    if (j < M) z[(size_t)pi * M + j] = acc[t];
  }
  __syncwarp();
}

// x_new (DOF row) = x_old + omega (z_0 + z_1) (first sweep from x = 0: omega (z_0 + z_1));
// zP holds partition 0's patches first, then partition 1's
template <typename T, int NP, int DIM>
__device__ __forceinline__ T as_combine_row(const int* n, int row, const T* zP, int npatch0, const T* xold,
                                            T om, bool first) {
  constexpr int NCH = 1 << DIM, M = NCH * NP;
  const int K = row / NP, q = row - K * NP;
  const int c[3] = {K % n[0], (K / n[0]) % n[1], DIM == 3 ? K / (n[0] * n[1]) : 0};
  int p[2], a[2];
#pragma unroll
  for (int part = 0; part < 2; ++part) {
    const int s[3] = {c[0] + part, c[1] + part, c[2] + part};
    const int q0 = as_patches_1d(n[0], part), q1 = as_patches_1d(n[1], part);
    p[part] = (s[0] >> 1) + q0 * ((s[1] >> 1) + q1 * (DIM == 3 ? (s[2] >> 1) : 0));
    a[part] = (s[0] & 1) | ((s[1] & 1) << 1) | (DIM == 3 ? ((s[2] & 1) << 2) : 0);
  }
  const T z0 = __ldcg(zP + (size_t)p[0] * M + a[0] * NP + q);
  const T z1 = __ldcg(zP + ((size_t)npatch0 + p[1]) * M + a[1] * NP + q);
  const T e = z0 + z1;
  return first ? om * e : fma(om, e, __ldcg(xold + row));
}

}  // namespace kcmg
