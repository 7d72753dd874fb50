// Matrix-free coupling of the finest level for the SIPG operator of a cell-wise coefficient
// field.  On uniform Cartesian cells the fine operator's off-diagonal blocks are the face
// reference matrices scaled by the harmonic face coefficient gamma_F = 2 nu_K nu_J /
// (nu_K + nu_J): the block coupling cell K to its -e_k neighbour L is gamma F_k^{RL}, to
// its +e_k neighbour R gamma F_k^{LR} (F_k^{XY}: test side X, trial side Y of a face normal
// to e_k).  The FP32 block-Jacobi sweeps of level 0 then read the coefficient (one value per
// cell) and the stored block inverses instead of the six FP32 off-diagonal blocks.
#include "kcmg_internal.h"

#include <cstring>
#include <type_traits>

namespace kcmg {

namespace {

template <typename TI> struct MfInv;
template <> struct MfInv<float> {
  static __device__ __forceinline__ float2 load(const float* p, size_t i) {
    return __ldg(reinterpret_cast<const float2*>(p) + i);
  }
};
template <> struct MfInv<__nv_bfloat16> {
  static __device__ __forceinline__ float2 load(const __nv_bfloat16* p, size_t i) {
    return __bfloat1622float2(reinterpret_cast<const __nv_bfloat162*>(p)[i]);
  }
};

// One damped block-Jacobi sweep on level 0 in FP32 (Alg. BJ, as k_bj_sweep): t = r - A_off z
// with A_off applied matrix-free, z_new = (1 - omega) z_old + omega D^{-1} t.  A block holds
// whole cells (t exchanged through shared memory for the inverse product); the inverses use
// the row-interleaved layout of the stored operator.
template <typename TI, int NP, int DIM, bool FIRST>
__global__ void __launch_bounds__(320) k_bj_sweep_mf(const float* __restrict__ nu, const float* __restrict__ F,
                                                     const TI* __restrict__ Dinv, int n0, int n1, int n2, int N,
                                                     const float* __restrict__ r, const float* __restrict__ zold,
                                                     float* __restrict__ znew, float omega) {
  constexpr int JP = (NP + 1) / 2;
  constexpr int NN = NP * NP;
  __shared__ float Fs[DIM * 2 * NN];   // direction k: [RL | LR]
  extern __shared__ float ts_mf[];      // blockDim floats
  if (!FIRST) {
    for (int e = threadIdx.x; e < DIM * 2 * NN; e += blockDim.x) {
      const int k = e / (2 * NN), rem = e - k * 2 * NN, side = rem / NN, ij = rem - side * NN;
      Fs[e] = F[((size_t)k * 4 + (side == 0 ? 2 : 1)) * NN + ij];   // F[k][RL] then F[k][LR]
    }
    __syncthreads();
  }
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  const int g = row >> 5, lane = row & 31;
  float tv = 0.f;
  if (row < N) {
    tv = r[row];
    if (!FIRST) {
      const int K = row / NP, i = row - K * NP;
      const int nn[3] = {n0, n1, n2};
      const int c[3] = {K % n0, (K / n0) % n1, DIM == 3 ? K / (n0 * n1) : 0};
      const int stride[3] = {1, n0, n0 * n1};
      const float nuK = __ldg(nu + K);
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          const bool has = side == 0 ? c[k] > 0 : c[k] < nn[k] - 1;
          if (!has) continue;
          const int J = side == 0 ? K - stride[k] : K + stride[k];
          const float nuJ = __ldg(nu + J);
          const float gam = 2.f * (nuK * nuJ) / (nuK + nuJ);
          const float* Fr = Fs + ((k * 2 + side) * NP + i) * NP;
          const float* zp = zold + (size_t)J * NP;
          float sum = 0.f;
#pragma unroll
          for (int j = 0; j < NP; ++j) sum = fmaf(Fr[j], __ldg(zp + j), sum);
          acc = fmaf(gam, sum, acc);
        }
      }
      tv -= acc;
    }
  }
  ts_mf[threadIdx.x] = tv;
  __syncthreads();
  if (row < N) {
    const int base = (row / NP) * NP - blockIdx.x * blockDim.x;
    float d0s = 0.f, d1s = 0.f;
#pragma unroll
    for (int jp = 0; jp < JP; ++jp) {
      const float2 d = MfInv<TI>::load(Dinv, ((size_t)g * JP + jp) * 32 + lane);
      d0s = fmaf(d.x, ts_mf[base + 2 * jp], d0s);
      if (2 * jp + 1 < NP) d1s = fmaf(d.y, ts_mf[base + 2 * jp + 1], d1s);
    }
    const float dz = d0s + d1s;
    znew[row] = FIRST ? omega * dz : fmaf(1.f - omega, zold[row], omega * dz);
  }
}

// The largest |gamma F_k^{XY} - A[slot][K]| over every off-diagonal block (FP64, the
// assembly's own arithmetic for gamma) as an atomic maximum on the bit pattern, and the
// largest |A[slot][K]|: setup rejects coefficient data that does not reproduce the blocks.
template <int NP, int DIM>
__global__ void k_mf_check(const double* __restrict__ nu, const double* __restrict__ F,
                           const double* __restrict__ nat, int n0, int n1, int n2,
                           unsigned long long* maxdiff, unsigned long long* maxabs) {
  constexpr int S = 2 * DIM + 1, NN = NP * NP;
  const int C = n0 * n1 * (DIM == 3 ? n2 : 1);
  const int nn[3] = {n0, n1, n2};
  const int stride[3] = {1, n0, n0 * n1};
  const size_t total = (size_t)(S - 1) * C * NN;
  double md = 0.0, ma = 0.0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int s = 1 + (int)(e / ((size_t)C * NN));
    const size_t rem = e % ((size_t)C * NN);
    const int K = (int)(rem / NN), ij = (int)(rem % NN);
    const int k = (s - 1) / 2, side = (s - 1) % 2;   // side 0: -e_k neighbour, 1: +e_k
    const int c[3] = {K % n0, (K / n0) % n1, DIM == 3 ? K / (n0 * n1) : 0};
    const bool has = side == 0 ? c[k] > 0 : c[k] < nn[k] - 1;
    double want = 0.0;
    if (has) {
      const int J = side == 0 ? K - stride[k] : K + stride[k];
      const double a = nu[K], b = nu[J];
      const double gam = 2.0 * (a * b) / (a + b);
      want = gam * F[((size_t)k * 4 + (side == 0 ? 2 : 1)) * NN + ij];
    }
    const double got = nat[((size_t)s * C + K) * NN + ij];
    md = fmax(md, fabs(want - got));
    ma = fmax(ma, fabs(got));
  }
  atomicMax(maxdiff, (unsigned long long)__double_as_longlong(md));
  atomicMax(maxabs, (unsigned long long)__double_as_longlong(ma));
}

template <typename F>
bool mf_dispatch(int np, int dim, F&& f) {
  switch (np * 10 + dim) {
    case 32: f(std::integral_constant<int, 3>{}, std::integral_constant<int, 2>{}); return true;
    case 62: f(std::integral_constant<int, 6>{}, std::integral_constant<int, 2>{}); return true;
    case 102: f(std::integral_constant<int, 10>{}, std::integral_constant<int, 2>{}); return true;
    case 43: f(std::integral_constant<int, 4>{}, std::integral_constant<int, 3>{}); return true;
    case 103: f(std::integral_constant<int, 10>{}, std::integral_constant<int, 3>{}); return true;
    case 203: f(std::integral_constant<int, 20>{}, std::integral_constant<int, 3>{}); return true;
    default: return false;
  }
}

}  // namespace

template <typename TI>
void launch_bj_sweep_mf(int np, int dim, const int* n, const float* nu, const float* F, const TI* Dinv, int N,
                        int rows_pad, int block_rows, const float* r, const float* zold, float* znew,
                        double omega, int first, cudaStream_t s) {
  const int grid = rows_pad / block_rows;
  const size_t smem = (size_t)block_rows * sizeof(float);
  mf_dispatch(np, dim, [&](auto NPc, auto DIMc) {
    constexpr int NP = decltype(NPc)::value, DIM = decltype(DIMc)::value;
    const int n2 = DIM == 3 ? n[2] : 1;
    if (first)
      k_bj_sweep_mf<TI, NP, DIM, true><<<grid, block_rows, smem, s>>>(nu, F, Dinv, n[0], n[1], n2, N, r, zold,
                                                                        znew, (float)omega);
    else
      k_bj_sweep_mf<TI, NP, DIM, false><<<grid, block_rows, smem, s>>>(nu, F, Dinv, n[0], n[1], n2, N, r, zold,
                                                                         znew, (float)omega);
  });
}

cudaError_t mf_check(int np, int dim, const int* n, const double* nu, const double* F, const double* nat,
                     double* maxdiff, double* maxabs, cudaStream_t s) {
  unsigned long long* buf = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&buf), 2 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(buf, 0, 2 * sizeof(unsigned long long), s)) != cudaSuccess) return e;
  const bool ok = mf_dispatch(np, dim, [&](auto NPc, auto DIMc) {
    constexpr int NP = decltype(NPc)::value, DIM = decltype(DIMc)::value;
    k_mf_check<NP, DIM><<<4096, 256, 0, s>>>(nu, F, nat, n[0], n[1], DIM == 3 ? n[2] : 1, buf, buf + 1);
  });
  if (!ok) return cudaErrorInvalidValue;
  unsigned long long h[2] = {0, 0};
  if ((e = cudaMemcpyAsync(h, buf, sizeof h, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  cudaFreeAsync(buf, s);
  memcpy(maxdiff, &h[0], sizeof(double));
  memcpy(maxabs, &h[1], sizeof(double));
  return cudaGetLastError();
}

template void launch_bj_sweep_mf<float>(int, int, const int*, const float*, const float*, const float*, int, int,
                                        int, const float*, const float*, float*, double, int, cudaStream_t);
template void launch_bj_sweep_mf<__nv_bfloat16>(int, int, const int*, const float*, const float*,
                                                const __nv_bfloat16*, int, int, int, const float*, const float*,
                                                float*, double, int, cudaStream_t);

}  // namespace kcmg
