// Additive Schwarz smoother (Alg. AS, Sec. 3.2 of Toprak & Kummer) on overlapping cell
// patches: setup of the patch inverses and the kernels of one smoothing step on a level
// (patch definitions in schwarz.cuh).
#include "schwarz.cuh"

#include <cmath>
#include <type_traits>

namespace kcmg {

namespace {

// Local matrix of patch blockIdx.x (+ first) of partition part, assembled from the natural
// FP64 blocks [S][C][np][np] of the level into shared memory and inverted in place by
// Gauss-Jordan elimination with partial (row) pivoting; the inverse is written transposed.
// A zero pivot sets *fail.
template <int NP, int DIM>
__global__ void __launch_bounds__(256) k_patch_inverse(const double* __restrict__ nat, const int* __restrict__ nbr,
                                                       int n0, int n1, int n2, int part, int first,
                                                       double* __restrict__ invT, int* fail) {
  constexpr int NCH = 1 << DIM, M = NCH * NP, S = 2 * DIM + 1, NF = S - 1;
  extern __shared__ double smem_pi[];
  double* Mx = smem_pi;            // [M][M]
  double* col = Mx + M * M;        // [M]
  __shared__ int perm[M];
  __shared__ int cell[NCH];
  __shared__ int s_piv;
  const int n[3] = {n0, n1, n2};
  const int ncell = n0 * n1 * (DIM == 3 ? n2 : 1);
  const int pi = first + blockIdx.x;
  if (threadIdx.x == 0) {
    int c[NCH];
    as_members<DIM>(n, part, pi, c);
    for (int a = 0; a < NCH; ++a) cell[a] = c[a];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < M * M; e += blockDim.x) {
    const int i = e / M, j = e - i * M;
    const int a = i / NP, q = i - a * NP, b = j / NP, t = j - b * NP;
    double v = 0.0;
    if (cell[a] < 0 || cell[b] < 0) {
      v = (i == j && cell[a] < 0) ? 1.0 : 0.0;
    } else {
      int slot = -1;
      if (a == b) slot = 0;
      else
        for (int s = 1; s < S; ++s)
          if (nbr[(size_t)cell[a] * NF + s - 1] == cell[b]) slot = s;
      if (slot >= 0) v = nat[(((size_t)slot * ncell + cell[a]) * NP + q) * NP + t];
    }
    Mx[e] = v;
  }
  __syncthreads();
  for (int c = 0; c < M; ++c) {
    if (threadIdx.x < 32) {   // pivot: largest |M[i][c]| for i >= c (lowest index on ties)
      double best = -1.0;
      int bi = c;
      for (int i = c + threadIdx.x; i < M; i += 32) {
        const double v = fabs(Mx[i * M + c]);
        if (v > best) { best = v; bi = i; }
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (threadIdx.x == 0) {
        s_piv = bi;
        perm[c] = bi;
        if (!(best > 0.0)) atomicExch(fail, 1);
      }
    }
    __syncthreads();
    const int p = s_piv;
    if (p != c)
      for (int j = threadIdx.x; j < M; j += blockDim.x) {
        const double t = Mx[c * M + j];
        Mx[c * M + j] = Mx[p * M + j];
        Mx[p * M + j] = t;
      }
    __syncthreads();
    const double pinv = 1.0 / Mx[c * M + c];
    __syncthreads();
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
      const double v = (j == c) ? pinv : Mx[c * M + j] * pinv;
      Mx[c * M + j] = v;
    }
    for (int i = threadIdx.x; i < M; i += blockDim.x) col[i] = Mx[i * M + c];
    __syncthreads();
    for (int e = threadIdx.x; e < M * M; e += blockDim.x) {
      const int i = e / M, j = e - i * M;
      if (i == c) continue;
      const double base = (j == c) ? 0.0 : Mx[e];
      Mx[e] = base - Mx[c * M + j] * col[i];
    }
    __syncthreads();
  }
  // undo the row interchanges as column interchanges, last first
  for (int c = M - 1; c >= 0; --c) {
    const int p = perm[c];
    if (p != c)
      for (int i = threadIdx.x; i < M; i += blockDim.x) {
        const double t = Mx[i * M + c];
        Mx[i * M + c] = Mx[i * M + p];
        Mx[i * M + p] = t;
      }
    __syncthreads();
  }
  double* out = invT + (size_t)pi * M * M;
  for (int e = threadIdx.x; e < M * M; e += blockDim.x) {
    const int q = e / M, j = e - q * M;
    out[e] = Mx[j * M + q];
  }
}

// both partitions' patch solves, one warp per patch (partition 0's patches first)
template <typename T, typename TI, int NP, int DIM>
__global__ void __launch_bounds__(256) k_as_patch(int n0, int n1, int n2, int np0, int np1,
                                                  const TI* __restrict__ inv0, const TI* __restrict__ inv1,
                                                  const T* __restrict__ r, T* __restrict__ zP) {
  constexpr int M = (1 << DIM) * NP;
  __shared__ T rs[8][M];
  const int n[3] = {n0, n1, n2};
  const int warp = threadIdx.x >> 5;
  const int gw = blockIdx.x * (blockDim.x >> 5) + warp, nw = gridDim.x * (blockDim.x >> 5);
  for (int w = gw; w < np0 + np1; w += nw) {
    if (w < np0) as_patch_solve_warp<T, TI, NP, DIM>(n, 0, w, inv0, r, zP, rs[warp]);
    else as_patch_solve_warp<T, TI, NP, DIM>(n, 1, w - np0, inv1, r, zP + (size_t)np0 * M, rs[warp]);
  }
}

template <typename T, int NP, int DIM>
__global__ void __launch_bounds__(256) k_as_combine(int n0, int n1, int n2, int N, const T* __restrict__ zP,
                                                    int np0, const T* __restrict__ xold, T* __restrict__ xnew,
                                                    double omega, int first) {
  const int n[3] = {n0, n1, n2};
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < N; row += gridDim.x * blockDim.x)
    xnew[row] = as_combine_row<T, NP, DIM>(n, row, zP, np0, xold, (T)omega, first != 0);
}

template <typename F>
bool as_dispatch(int np, int dim, F&& f) {
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

int nblocks_cap(size_t n, int t, int cap) {
  size_t b = (n + t - 1) / t;
  if (b > (size_t)cap) b = cap;
  return b < 1 ? 1 : (int)b;
}

}  // namespace

cudaError_t launch_patch_inverse(int np, int dim, const double* nat, const int* nbr, const int* n, int part,
                                 double* invT, int* fail, cudaStream_t s) {
  cudaError_t err = cudaSuccess;
  const bool ok = as_dispatch(np, dim, [&](auto NPc, auto DIMc) {
    constexpr int NP = decltype(NPc)::value, DIM = decltype(DIMc)::value;
    constexpr int M = (1 << DIM) * NP;
    const size_t smem = (size_t)M * M * sizeof(double) + M * sizeof(double);
    auto kern = k_patch_inverse<NP, DIM>;
    if ((err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
      return;
    const int total = as_npatch(n, dim, part);
    for (int first = 0; first < total; first += 65535) {   // grid x limit of one launch
      const int cnt = total - first < 65535 ? total - first : 65535;
      kern<<<cnt, 256, smem, s>>>(nat, nbr, n[0], n[1], dim == 3 ? n[2] : 1, part, first, invT, fail);
    }
    err = cudaGetLastError();
  });
  return ok ? err : cudaErrorInvalidValue;
}

template <typename T, typename TI>
void launch_as_patch(int np, int dim, const int* n, const TI* inv0, const TI* inv1, const T* r, T* zP,
                     cudaStream_t s) {
  as_dispatch(np, dim, [&](auto NPc, auto DIMc) {
    constexpr int NP = decltype(NPc)::value, DIM = decltype(DIMc)::value;
    const int np0 = as_npatch(n, dim, 0), np1 = as_npatch(n, dim, 1);
    const int blocks = nblocks_cap((size_t)(np0 + np1), 8, 1 << 20);   // 8 warps per block
    k_as_patch<T, TI, NP, DIM><<<blocks, 256, 0, s>>>(n[0], n[1], dim == 3 ? n[2] : 1, np0, np1, inv0, inv1, r, zP);
  });
}

template <typename T>
void launch_as_combine(int np, int dim, const int* n, int N, const T* zP, const T* xold, T* xnew,
                       double omega, int first, cudaStream_t s) {
  as_dispatch(np, dim, [&](auto NPc, auto DIMc) {
    constexpr int NP = decltype(NPc)::value, DIM = decltype(DIMc)::value;
    const int np0 = as_npatch(n, dim, 0);
    k_as_combine<T, NP, DIM><<<nblocks_cap(N, 256, 1 << 20), 256, 0, s>>>(
        n[0], n[1], dim == 3 ? n[2] : 1, N, zP, np0, xold, xnew, omega, first);
  });
}

template void launch_as_patch<double, double>(int, int, const int*, const double*, const double*, const double*,
                                              double*, cudaStream_t);
template void launch_as_patch<float, float>(int, int, const int*, const float*, const float*, const float*,
                                            float*, cudaStream_t);
template void launch_as_patch<float, __nv_bfloat16>(int, int, const int*, const __nv_bfloat16*,
                                                    const __nv_bfloat16*, const float*, float*, cudaStream_t);
template void launch_as_combine<double>(int, int, const int*, int, const double*, const double*, double*, double,
                                        int, cudaStream_t);
template void launch_as_combine<float>(int, int, const int*, int, const float*, const float*, float*, double, int,
                                       cudaStream_t);

}  // namespace kcmg
