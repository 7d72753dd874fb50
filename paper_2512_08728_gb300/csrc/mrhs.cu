// Multi-right-hand-side K-cycle: R independent solves of Alg. 2 (with Alg. 1 after every
// correction) that share every operator application.
//
// Each right-hand side r keeps its own basis W_r, Z_r, Gram coefficients, residual norm
// and level-local criteria (Sec. 4.2), exactly as a single solve would; a level loop runs
// while any right-hand side is still active on it, and a right-hand side that is not
// (converged, or inactive on the calling level) is masked: its correction is discarded
// (alpha = 0, nothing appended).  All vectors are [N][R] with the right-hand sides
// fastest, so one warp covers the R values of a DOF row with coalesced accesses, and one
// pass over an operator block serves every right-hand side.
//
// Precision follows the single-right-hand-side forms: the residual minimisation (w = A z
// with the FP64 operator, W, Z, x, r, Gram coefficients), the transfers and the coarsest
// solve are FP64; the block-Jacobi sweeps run in FP64 (FP64 form) or on the tensor cores
// (mixed forms): each cell's 10x10 (generally np x np) blocks times the np x R block of
// iterates is an mma.sync m16n8k8 TF32 product with FP32 accumulation (optionally split
// into three TF32 products for FP32 accuracy), with the inverses stored in FP32 or BF16.
// The FP64 minimisation over these corrections is the iterative refinement: the attainable
// residual is FP64's.
//
// Control runs on the host: per loop test the engine reads three flags of the level's
// device state (any active, any restart due, any convergence claim).  Per-right-hand-side
// decisions (reorthogonalisation, discard, alpha, masks) are taken on the device by
// one-warp control kernels.
#include "kcmg_internal.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

namespace kcmg {

namespace {

constexpr int kGramWarps = 8;      // warps per block of the Gram / vector kernels
// blocks of the Gram / vector kernels: four per SM (k_mdots, 64 registers x 256 threads,
// fills the register file at four), so that 32 warps per SM keep their column loads in
// flight; one block per SM left these kernels latency-bound at 15-27 % of the FP64 rate
constexpr int kGramBlocks = 4 * 152;

enum : int { MF_REORTH = 1, MF_DISCARD = 2 };

// Device state of one level (one MG call is active per level at any time).
struct MState {
  int any, any_restart, any_claim, any_reorth;   // flags the host reads (first 32 bytes)
  int nact, pad_f0, pad_f1, pad_f2;              // active columns after the last test
  int R, lcap, maxit, it;
  int iters_total, nrestart, status, guard;
  int guard_cap, level, per_cycle, cap;    // restart when l + per_cycle > cap
  int act[kMaxRhs], l[kMaxRhs], flags[kMaxRhs], claim[kMaxRhs], brk[kMaxRhs], restart[kMaxRhs];
  double rtol, atol, brk_tol, pad2;
  double rnorm[kMaxRhs], rnorm0[kMaxRhs], eps[kMaxRhs], naz2[kMaxRhs], gam[kMaxRhs], alp[kMaxRhs];
};

enum CtlKind : int {
  CTL_INIT0,    // level 0 start: sums = ||b - A x0||^2
  CTL_BEGIN,    // level >= 1 start: sums = ||b_c||^2 (restricted residual)
  CTL_TEST,     // loop test (level-local criteria); restart / claim flags
  CTL_GRAM1,    // sums = W^T w (columns < l) and ||w||^2 (column lcap)
  CTL_GRAM2,    // sums = W^T w' (reorthogonalisation pass)
  CTL_UPDATE,   // sums = ||w_hat||^2, w_hat . r
  CTL_FINISH,   // sums = ||r||^2 after the update
  CTL_RESTART,  // sums = ||b - A x||^2 for the restarting right-hand sides
  CTL_CONFIRM,  // level 0: sums = true ||b - A x||^2 of the claiming right-hand sides
  CTL_ITEND     // end of an iteration
};

// ------------------------------------------------------------------ small helpers
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& t) {
  s = a + b;
  const double bb = s - a;
  t = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ uint32_t tf32_bits(float x) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return u;
}

// D += A (16x8, row) * B (8x8, col), TF32 inputs, FP32 accumulation
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// split x into a TF32 head and a TF32 tail (x ~ hi + lo to ~2^-22 relative)
__device__ __forceinline__ void tf32_split(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_bits(x);
  lo = tf32_bits(x - __uint_as_float(hi));
}

template <typename TI> __device__ __forceinline__ float to_f(TI v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

__device__ __forceinline__ int max_l(const MState* st) {
  int m = 0;
  for (int r = 0; r < st->R; ++r) m = max(m, st->l[r]);
  return m;
}

// ------------------------------------------------------------------ operator (FP64)
// y = A x (MODE 0), y = b - A x (MODE 1), y = b - A x with double-double accumulation
// (MODE 2).  One warp per cell; lane r = right-hand side.  A: natural blocks
// [S][C][NP][NP]; x, y, b: [C*NP][R].
template <int NP, int S, int MODE>
__global__ void __launch_bounds__(256) k_mspmm64(const double* __restrict__ A, const int* __restrict__ nbr,
                                                 int C, int R, const double* __restrict__ x,
                                                 double* __restrict__ y, const double* __restrict__ b) {
  constexpr int NF = S - 1;
  const int wpb = blockDim.x >> 5;
  const int r = threadIdx.x & 31;
  for (int K = blockIdx.x * wpb + (threadIdx.x >> 5); K < C; K += gridDim.x * wpb) {
    if (r >= R) continue;
    double acc[NP], cmp[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) { acc[i] = 0.0; cmp[i] = 0.0; }
#pragma unroll 1
    for (int s = 0; s < S; ++s) {
      const int J = (s == 0) ? K : __ldg(nbr + (size_t)K * NF + s - 1);
      if (J < 0) continue;
      const double* Ab = A + ((size_t)s * C + K) * NP * NP;
      const double* xb = x + (size_t)J * NP * R + r;
      double xv[NP];
#pragma unroll
      for (int q = 0; q < NP; ++q) xv[q] = __ldg(xb + (size_t)q * R);
#pragma unroll
      for (int i = 0; i < NP; ++i) {
#pragma unroll
        for (int q = 0; q < NP; ++q) {
          const double a = __ldg(Ab + i * NP + q);
          if (MODE == 2) {
            const double p = a * xv[q];
            const double e = fma(a, xv[q], -p);
            double s2, t2;
            two_sum(acc[i], p, s2, t2);
            acc[i] = s2;
            cmp[i] += t2 + e;
          } else {
            acc[i] = fma(a, xv[q], acc[i]);
          }
        }
      }
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      const size_t o = ((size_t)K * NP + i) * R + r;
      if (MODE == 0) {
        y[o] = acc[i];
      } else if (MODE == 1) {
        y[o] = __ldg(b + o) - acc[i];
      } else {
        double s2, t2;
        two_sum(__ldg(b + o), -acc[i], s2, t2);
        y[o] = s2 + (t2 - cmp[i]);
      }
    }
  }
}

// ------------------------------------------------------------------ smoother (FP64 form)
// One sweep of Alg. BJ: t = r - A_off zo (skipped when first), zn = (1-om) zo + om D^-1 t.
template <int NP, int S>
__global__ void __launch_bounds__(256) k_msweep64(const double* __restrict__ A, const double* __restrict__ D,
                                                  const int* __restrict__ nbr, int C, int R,
                                                  const double* __restrict__ rv, const double* __restrict__ zo,
                                                  double* __restrict__ zn, double om, int first) {
  constexpr int NF = S - 1;
  const int wpb = blockDim.x >> 5;
  const int r = threadIdx.x & 31;
  for (int K = blockIdx.x * wpb + (threadIdx.x >> 5); K < C; K += gridDim.x * wpb) {
    if (r >= R) continue;
    double t[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) t[i] = __ldg(rv + ((size_t)K * NP + i) * R + r);
    if (!first) {
#pragma unroll 1
      for (int s = 1; s < S; ++s) {
        const int J = __ldg(nbr + (size_t)K * NF + s - 1);
        if (J < 0) continue;
        const double* Ab = A + ((size_t)s * C + K) * NP * NP;
        double zv[NP];
#pragma unroll
        for (int q = 0; q < NP; ++q) zv[q] = __ldg(zo + ((size_t)J * NP + q) * R + r);
#pragma unroll
        for (int i = 0; i < NP; ++i)
#pragma unroll
          for (int q = 0; q < NP; ++q) t[i] = fma(-__ldg(Ab + i * NP + q), zv[q], t[i]);
      }
    }
    const double* Db = D + (size_t)K * NP * NP;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      double d = 0.0;
#pragma unroll
      for (int q = 0; q < NP; ++q) d = fma(__ldg(Db + i * NP + q), t[q], d);
      const size_t o = ((size_t)K * NP + i) * R + r;
      zn[o] = first ? om * d : fma(1.0 - om, __ldg(zo + o), om * d);
    }
  }
}

// ------------------------------------------------------------------ smoother (tensor cores)
// One sweep of Alg. BJ on the tensor cores.  A warp owns a cell K: it stages the cell's
// off-diagonal blocks and its inverse in shared memory, accumulates
//   T (np x R) = r_K - sum_s A_{K,s} zo_{nbr(K,s)}
// with one m16n8k8 TF32 MMA per (16-row tile, 8-column k step, 8-RHS tile), stores T in
// shared memory and forms D_K^{-1} T the same way; the epilogue applies the damping.
// x3: three TF32 products (hi*hi + hi*lo + lo*hi) for FP32-level accuracy.
// Ac: [C][S][NP][NP] FP32 (cell-major), D: [C][NP][NP] (TI); r32, zo: [C*NP][R] FP32.
template <int NP, int S> struct TcShape {
  static constexpr int MT = (NP + 15) / 16;   // 16-row tiles
  static constexpr int KS = (NP + 7) / 8;     // k steps per block
  static constexpr int RS = 40;               // row stride of T in shared memory (floats)
  static constexpr int NT = kMaxRhs / 8;      // 8-wide RHS tiles
  static constexpr int WS = (S - 1) * NP * NP + NP * NP + MT * 16 * RS;   // floats per warp
};

template <int NP, int S, typename TI, typename TOUT>
__global__ void __launch_bounds__(512) k_msweep_tc(const float* __restrict__ Ac, const TI* __restrict__ D,
                                                   const int* __restrict__ nbr, int C, int R,
                                                   const float* __restrict__ r32, const float* __restrict__ zo,
                                                   TOUT* __restrict__ zn, float om, int first, int x3) {
  using Sh = TcShape<NP, S>;
  constexpr int NF = S - 1, MT = Sh::MT, KS = Sh::KS, RS = Sh::RS, NT = Sh::NT;
  extern __shared__ float smem_tc[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
  float* As = smem_tc + (size_t)warp * Sh::WS;   // [NF][NP][NP]
  float* Ds = As + NF * NP * NP;                  // [NP][NP]
  float* Ts = Ds + NP * NP;                       // [MT*16][RS]
  const int wpb = blockDim.x >> 5;
  const int nt_used = (R + 7) >> 3;
  for (int K = blockIdx.x * wpb + warp; K < C; K += gridDim.x * wpb) {
    __syncwarp();
    if (!first) {
      const float* src = Ac + ((size_t)K * S + 1) * NP * NP;
      for (int e = lane; e < NF * NP * NP; e += 32) As[e] = __ldg(src + e);
    }
    {
      const TI* src = D + (size_t)K * NP * NP;
      for (int e = lane; e < NP * NP; e += 32) Ds[e] = to_f<TI>(src[e]);
    }
    __syncwarp();
    float c[MT][NT][4];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const int row0 = mt * 16 + gid, row1 = row0 + 8, col = nt * 8 + 2 * tig;
        const float* rb = r32 + (size_t)K * NP * R;
        c[mt][nt][0] = (row0 < NP && col < R) ? __ldg(rb + (size_t)row0 * R + col) : 0.f;
        c[mt][nt][1] = (row0 < NP && col + 1 < R) ? __ldg(rb + (size_t)row0 * R + col + 1) : 0.f;
        c[mt][nt][2] = (row1 < NP && col < R) ? __ldg(rb + (size_t)row1 * R + col) : 0.f;
        c[mt][nt][3] = (row1 < NP && col + 1 < R) ? __ldg(rb + (size_t)row1 * R + col + 1) : 0.f;
      }
    if (!first) {
#pragma unroll 1
      for (int s = 1; s < S; ++s) {
        const int J = __ldg(nbr + (size_t)K * NF + s - 1);
        if (J < 0) continue;
        const float* zb = zo + (size_t)J * NP * R;
        const float* Ab = As + (s - 1) * NP * NP;
#pragma unroll
        for (int kk = 0; kk < KS; ++kk) {
          const int q0 = kk * 8 + tig, q1 = q0 + 4;
          uint32_t bh[NT][2], bl[NT][2];
#pragma unroll
          for (int nt = 0; nt < NT; ++nt) {
            const int rr = nt * 8 + gid;
            const float v0 = (q0 < NP && rr < R) ? __ldg(zb + (size_t)q0 * R + rr) : 0.f;
            const float v1 = (q1 < NP && rr < R) ? __ldg(zb + (size_t)q1 * R + rr) : 0.f;
            tf32_split(v0, bh[nt][0], bl[nt][0]);
            tf32_split(v1, bh[nt][1], bl[nt][1]);
          }
#pragma unroll
          for (int mt = 0; mt < MT; ++mt) {
            const int row0 = mt * 16 + gid, row1 = row0 + 8;
            const float f0 = (row0 < NP && q0 < NP) ? -Ab[row0 * NP + q0] : 0.f;
            const float f1 = (row1 < NP && q0 < NP) ? -Ab[row1 * NP + q0] : 0.f;
            const float f2 = (row0 < NP && q1 < NP) ? -Ab[row0 * NP + q1] : 0.f;
            const float f3 = (row1 < NP && q1 < NP) ? -Ab[row1 * NP + q1] : 0.f;
            uint32_t ah[4], al[4];
            tf32_split(f0, ah[0], al[0]);
            tf32_split(f1, ah[1], al[1]);
            tf32_split(f2, ah[2], al[2]);
            tf32_split(f3, ah[3], al[3]);
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
              if (nt >= nt_used) break;
              if (x3) {
                mma_tf32(c[mt][nt], al, bh[nt]);
                mma_tf32(c[mt][nt], ah, bl[nt]);
              }
              mma_tf32(c[mt][nt], ah, bh[nt]);
            }
          }
        }
      }
    }
    // T -> shared memory (rows >= NP and columns >= R stay zero)
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const int row0 = mt * 16 + gid, row1 = row0 + 8, col = nt * 8 + 2 * tig;
        if (row0 < NP) { Ts[row0 * RS + col] = c[mt][nt][0]; Ts[row0 * RS + col + 1] = c[mt][nt][1]; }
        if (row1 < NP) { Ts[row1 * RS + col] = c[mt][nt][2]; Ts[row1 * RS + col + 1] = c[mt][nt][3]; }
      }
    __syncwarp();
    // E = D^{-1} T
    float e[MT][NT][4];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int k = 0; k < 4; ++k) e[mt][nt][k] = 0.f;
#pragma unroll
    for (int kk = 0; kk < KS; ++kk) {
      const int q0 = kk * 8 + tig, q1 = q0 + 4;
      uint32_t bh[NT][2], bl[NT][2];
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const int rr = nt * 8 + gid;
        const float v0 = (q0 < NP) ? Ts[q0 * RS + rr] : 0.f;
        const float v1 = (q1 < NP) ? Ts[q1 * RS + rr] : 0.f;
        tf32_split(v0, bh[nt][0], bl[nt][0]);
        tf32_split(v1, bh[nt][1], bl[nt][1]);
      }
#pragma unroll
      for (int mt = 0; mt < MT; ++mt) {
        const int row0 = mt * 16 + gid, row1 = row0 + 8;
        const float f0 = (row0 < NP && q0 < NP) ? Ds[row0 * NP + q0] : 0.f;
        const float f1 = (row1 < NP && q0 < NP) ? Ds[row1 * NP + q0] : 0.f;
        const float f2 = (row0 < NP && q1 < NP) ? Ds[row0 * NP + q1] : 0.f;
        const float f3 = (row1 < NP && q1 < NP) ? Ds[row1 * NP + q1] : 0.f;
        uint32_t ah[4], al[4];
        tf32_split(f0, ah[0], al[0]);
        tf32_split(f1, ah[1], al[1]);
        tf32_split(f2, ah[2], al[2]);
        tf32_split(f3, ah[3], al[3]);
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
          if (nt >= nt_used) break;
          if (x3) {
            mma_tf32(e[mt][nt], al, bh[nt]);
            mma_tf32(e[mt][nt], ah, bl[nt]);
          }
          mma_tf32(e[mt][nt], ah, bh[nt]);
        }
      }
    }
    // zn = (1 - om) zo + om E   (first sweep: om E)
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int row = mt * 16 + gid + ((k >> 1) << 3), col = nt * 8 + 2 * tig + (k & 1);
          if (row < NP && col < R) {
            const size_t o = ((size_t)K * NP + row) * R + col;
            const float v = first ? om * e[mt][nt][k] : fmaf(1.f - om, __ldg(zo + o), om * e[mt][nt][k]);
            zn[o] = (TOUT)v;
          }
        }
      }
  }
}

// ------------------------------------------------------------------ transfers, coarse solve
// b_c = P^T r_f per coarse cell (warp per coarse cell, lane = RHS); with rc: r_c = b_c and
// x_c = 0 (start of MG on the coarse level).  part[blk][32]: sum of b_c^2 per RHS.
template <int NP, int DIM>
__global__ void __launch_bounds__(256) k_mrestrict(const double* __restrict__ rf, int nfx, int nfy, int ncx,
                                                   int ncy, int Cc, const double* __restrict__ P, int R,
                                                   double* __restrict__ bc, double* __restrict__ rc,
                                                   double* __restrict__ xc, double* __restrict__ part) {
  constexpr int NCH = 1 << DIM;
  __shared__ double Ps[NCH * NP * NP];
  __shared__ double red[8][32];
  for (int i = threadIdx.x; i < NCH * NP * NP; i += blockDim.x) Ps[i] = P[i];
  __syncthreads();
  const int wpb = blockDim.x >> 5, warp = threadIdx.x >> 5, r = threadIdx.x & 31;
  double nrm = 0.0;
  for (int J = blockIdx.x * wpb + warp; J < Cc; J += gridDim.x * wpb) {
    if (r >= R) continue;
    const int jx = J % ncx, jy = (J / ncx) % ncy, jz = DIM == 3 ? J / (ncx * ncy) : 0;
    double s[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) s[i] = 0.0;
#pragma unroll 1
    for (int k = 0; k < NCH; ++k) {
      const int fx = 2 * jx + (k & 1), fy = 2 * jy + ((k >> 1) & 1), fz = DIM == 3 ? 2 * jz + ((k >> 2) & 1) : 0;
      const int Kf = fx + nfx * (fy + nfy * fz);
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        const double v = __ldg(rf + ((size_t)Kf * NP + q) * R + r);
#pragma unroll
        for (int i = 0; i < NP; ++i) s[i] = fma(Ps[(k * NP + q) * NP + i], v, s[i]);
      }
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      const size_t o = ((size_t)J * NP + i) * R + r;
      bc[o] = s[i];
      if (rc) { rc[o] = s[i]; xc[o] = 0.0; }
      nrm = fma(s[i], s[i], nrm);
    }
  }
  if (!part) return;
  red[warp][r] = nrm;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = 0.0;
    for (int w = 0; w < wpb; ++w) t += red[w][threadIdx.x];
    part[(size_t)blockIdx.x * 32 + threadIdx.x] = t;
  }
}

// z_f = P x_c (warp per fine cell, lane = RHS)
template <int NP, int DIM>
__global__ void __launch_bounds__(256) k_mprolong(const double* __restrict__ xc, int nfx, int nfy, int Cf,
                                                  int ncx, int ncy, const double* __restrict__ P, int R,
                                                  double* __restrict__ zf) {
  constexpr int NCH = 1 << DIM;
  __shared__ double Ps[NCH * NP * NP];
  for (int i = threadIdx.x; i < NCH * NP * NP; i += blockDim.x) Ps[i] = P[i];
  __syncthreads();
  const int wpb = blockDim.x >> 5, r = threadIdx.x & 31;
  for (int K = blockIdx.x * wpb + (threadIdx.x >> 5); K < Cf; K += gridDim.x * wpb) {
    if (r >= R) continue;
    const int ix = K % nfx, iy = (K / nfx) % nfy, iz = DIM == 3 ? K / (nfx * nfy) : 0;
    const int k = (ix & 1) | ((iy & 1) << 1) | (DIM == 3 ? ((iz & 1) << 2) : 0);
    const int J = (ix >> 1) + ncx * ((iy >> 1) + ncy * (iz >> 1));
    double xv[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) xv[i] = __ldg(xc + ((size_t)J * NP + i) * R + r);
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      double s = 0.0;
#pragma unroll
      for (int i = 0; i < NP; ++i) s = fma(Ps[(k * NP + q) * NP + i], xv[i], s);
      zf[((size_t)K * NP + q) * R + r] = s;
    }
  }
}

// x_c = A_c^{-1} b_c, warp per row, lane = RHS
__global__ void __launch_bounds__(256) k_mcoarse(const double* __restrict__ Ainv, int n, int R,
                                                 const double* __restrict__ bc, double* __restrict__ xc) {
  const int wpb = blockDim.x >> 5, r = threadIdx.x & 31;
  for (int row = blockIdx.x * wpb + (threadIdx.x >> 5); row < n; row += gridDim.x * wpb) {
    if (r >= R) continue;
    const double* a = Ainv + (size_t)row * n;
    double s0 = 0.0, s1 = 0.0;
    int j = 0;
    for (; j + 1 < n; j += 2) {
      s0 = fma(__ldg(a + j), __ldg(bc + (size_t)j * R + r), s0);
      s1 = fma(__ldg(a + j + 1), __ldg(bc + (size_t)(j + 1) * R + r), s1);
    }
    if (j < n) s0 = fma(__ldg(a + j), __ldg(bc + (size_t)j * R + r), s0);
    xc[(size_t)row * R + r] = s0 + s1;
  }
}

// ------------------------------------------------------------------ Gram kernels (FP64)
// Block reduction of NC per-lane values over the block's warps into part[blk][pc0 + c][32].
template <int NC>
__device__ __forceinline__ void block_cols(const double (&v)[NC], double* red /*[wpb][NC][32]*/, double* part,
                                           int pstride, int pc0, int ncmax) {
  const int wpb = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
#pragma unroll
  for (int c = 0; c < NC; ++c) red[(warp * NC + c) * 32 + lane] = v[c];
  __syncthreads();
  for (int t = threadIdx.x; t < NC * 32; t += blockDim.x) {
    const int c = t >> 5, ln = t & 31;
    if (c >= ncmax) continue;
    double s = 0.0;
    for (int w = 0; w < wpb; ++w) s += red[(w * NC + c) * 32 + ln];
    part[((size_t)blockIdx.x * pstride + pc0 + c) * 32 + ln] = s;
  }
}

// part[blk][c][32] = sum over the block's rows of W[c] . w (c < l_r); part[blk][lcap] = ||w||^2.
// gated: return at once unless some right-hand side reorthogonalises (second pass).
__global__ void __launch_bounds__(256) k_mdots(const double* __restrict__ W, const double* __restrict__ w,
                                               int N, int R, int lcap, const MState* __restrict__ st,
                                               double* __restrict__ part, int gated) {
  __shared__ double red[kGramWarps * 9 * 32];
  if (gated && !st->any_reorth) return;
  const int L = max_l(st);
  const int wpb = blockDim.x >> 5, lane = threadIdx.x & 31;
  const int lr = lane < R ? st->l[lane] : 0;
  const bool use = lane < R && (!gated || (st->flags[lane] & MF_REORTH));
  for (int c0 = 0; c0 == 0 || c0 < L; c0 += 8) {
    double acc[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) acc[c] = 0.0;
    if (use) {
      for (int j = blockIdx.x * wpb + (threadIdx.x >> 5); j < N; j += gridDim.x * wpb) {
        const double wv = __ldg(w + (size_t)j * R + lane);
        if (c0 == 0) acc[8] = fma(wv, wv, acc[8]);
#pragma unroll
        for (int c = 0; c < 8; ++c)
          if (c0 + c < lr) acc[c] = fma(__ldg(W + ((size_t)(c0 + c) * N + j) * R + lane), wv, acc[c]);
      }
    }
    double v8[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) v8[c] = acc[c];
    block_cols<8>(v8, red, part, lcap + 1, c0, min(8, lcap - c0));
    if (c0 == 0) {
      double vn[1] = {acc[8]};
      block_cols<1>(vn, red, part, lcap + 1, lcap, 1);
    }
  }
}

// out[c][32] = sum over blocks of part[blk][c][32] for c < ncols (columns c < lcols-limit
// with c >= max l are skipped when limit is set: they are unused)
__global__ void __launch_bounds__(256) k_mreduce(const double* __restrict__ part, int nblk, int ncols,
                                                 const MState* __restrict__ st, int limit,
                                                 double* __restrict__ out) {
  __shared__ double red[8][32];
  const int c = blockIdx.x;
  if (limit && c < ncols - 1 && c >= max_l(st)) return;
  const int wpb = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double s = 0.0;
  for (int b = warp; b < nblk; b += wpb) s += part[((size_t)b * ncols + c) * 32 + lane];
  red[warp][lane] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = 0.0;
    for (int w = 0; w < wpb; ++w) t += red[w][threadIdx.x];
    out[(size_t)c * 32 + threadIdx.x] = t;
  }
}

// w' = w - W h (reorthogonalising right-hand sides only)
__global__ void __launch_bounds__(256) k_mapply(const double* __restrict__ W, const double* __restrict__ w,
                                                double* __restrict__ wre, int N, int R,
                                                const MState* __restrict__ st, const double* __restrict__ h) {
  if (!st->any_reorth) return;
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  if (lane >= R || !(st->flags[lane] & MF_REORTH)) return;
  const int lr = st->l[lane];
  for (int j = blockIdx.x * wpb + (threadIdx.x >> 5); j < N; j += gridDim.x * wpb) {
    double s = __ldg(w + (size_t)j * R + lane);
    for (int i = 0; i < lr; ++i) s = fma(-h[(size_t)i * 32 + lane], __ldg(W + ((size_t)i * N + j) * R + lane), s);
    wre[(size_t)j * R + lane] = s;
  }
}

// w_hat = wsrc - W cw, z_hat = z - Z cz into column l_r; part[blk][0..1][32] = ||w_hat||^2, w_hat . r
__global__ void __launch_bounds__(256) k_mupdate(double* __restrict__ W, double* __restrict__ Z, int N, int R,
                                                 const double* __restrict__ w, const double* __restrict__ wre,
                                                 const double* __restrict__ z, const double* __restrict__ rv,
                                                 const MState* __restrict__ st, const double* __restrict__ cw,
                                                 const double* __restrict__ cz, double* __restrict__ part) {
  __shared__ double red[kGramWarps * 2 * 32];
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  double v[2] = {0.0, 0.0};
  if (lane < R && !(st->flags[lane] & MF_DISCARD)) {
    const int lr = st->l[lane];
    const double* wsrc = (st->flags[lane] & MF_REORTH) ? wre : w;
    double* Wl = W + (size_t)lr * N * R;
    double* Zl = Z + (size_t)lr * N * R;
    for (int j = blockIdx.x * wpb + (threadIdx.x >> 5); j < N; j += gridDim.x * wpb) {
      const size_t o = (size_t)j * R + lane;
      double av = wsrc[o], zv = __ldg(z + o);
      for (int i = 0; i < lr; ++i) {
        const size_t oi = ((size_t)i * N + j) * R + lane;
        av = fma(-cw[(size_t)i * 32 + lane], __ldg(W + oi), av);
        zv = fma(-cz[(size_t)i * 32 + lane], __ldg(Z + oi), zv);
      }
      Wl[o] = av;
      Zl[o] = zv;
      v[0] = fma(av, av, v[0]);
      v[1] = fma(av, __ldg(rv + o), v[1]);
    }
  }
  block_cols<2>(v, red, part, 2, 0, 2);
}

// normalise the new columns and update x, r; part[blk][32] = ||r||^2
__global__ void __launch_bounds__(256) k_mfinish(double* __restrict__ W, double* __restrict__ Z, int N, int R,
                                                 double* __restrict__ x, double* __restrict__ rv,
                                                 const MState* __restrict__ st, double* __restrict__ part) {
  __shared__ double red[kGramWarps * 32];
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  double v[1] = {0.0};
  if (lane < R) {
    const bool upd = !(st->flags[lane] & MF_DISCARD);
    const int lr = st->l[lane];
    const double g = st->gam[lane], al = st->alp[lane];
    double* Wl = W + (size_t)lr * N * R;
    double* Zl = Z + (size_t)lr * N * R;
    for (int j = blockIdx.x * wpb + (threadIdx.x >> 5); j < N; j += gridDim.x * wpb) {
      const size_t o = (size_t)j * R + lane;
      double r_ = rv[o];
      if (upd) {
        const double wv = Wl[o] * g, zv = Zl[o] * g;
        Wl[o] = wv;
        Zl[o] = zv;
        x[o] = fma(al, zv, x[o]);
        r_ = fma(-al, wv, r_);
        rv[o] = r_;
      }
      v[0] = fma(r_, r_, v[0]);
    }
  }
  block_cols<1>(v, red, part, 1, 0, 1);
}

// part[blk][32] = sum of v^2 per right-hand side
__global__ void __launch_bounds__(256) k_mnorm(const double* __restrict__ v, int N, int R, double* __restrict__ part) {
  __shared__ double red[kGramWarps * 32];
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  double a[1] = {0.0};
  if (lane < R)
    for (int j = blockIdx.x * wpb + (threadIdx.x >> 5); j < N; j += gridDim.x * wpb) {
      const double t = __ldg(v + (size_t)j * R + lane);
      a[0] = fma(t, t, a[0]);
    }
  block_cols<1>(a, red, part, 1, 0, 1);
}

// dst = src for the right-hand sides flagged in mask[] (restart / confirmation)
__global__ void k_mcopy_masked(const double* __restrict__ src, double* __restrict__ dst, int N, int R,
                               const int* __restrict__ mask) {
  const size_t n = (size_t)N * R;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    if (mask[i % R]) dst[i] = src[i];
}

__global__ void k_mto_f32(const double* __restrict__ src, float* __restrict__ dst, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

// [S][C][NP][NP] FP64 -> [C][S][NP][NP] FP32 (cell-major copy for the tensor-core sweep)
__global__ void k_cellmajor_f32(const double* __restrict__ nat, int S, int C, int bs, float* __restrict__ out) {
  const size_t n = (size_t)S * C * bs;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t s = i / ((size_t)C * bs), rem = i - s * C * bs, K = rem / bs, e = rem - K * bs;
    out[(K * S + s) * bs + e] = (float)nat[i];
  }
}

template <typename T>
__global__ void k_narrow(const double* __restrict__ src, T* __restrict__ dst, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = (T)src[i];
}

// ------------------------------------------------------------------ control (one warp)
__global__ void k_mctl(MState* st, const MState* parent, const double* __restrict__ sums, double* cw,
                       double* cz, int kind) {
  const int r = threadIdx.x;
  const int R = st->R, lcap = st->lcap;
  bool f_any = false, f_restart = false, f_claim = false, f_reorth = false;
  if (r < R) {
    switch (kind) {
      case CTL_INIT0: {
        const double n0 = sqrt(sums[r]);
        st->rnorm0[r] = n0;
        st->rnorm[r] = n0;
        st->eps[r] = fmax(st->rtol * n0, st->atol);
        st->act[r] = n0 > st->eps[r] && isfinite(n0);
        if (!isfinite(n0)) st->status = KCMG_NONFINITE;
        st->l[r] = 0;
        st->flags[r] = 0;
        st->brk[r] = 0;
        st->claim[r] = 0;
        st->restart[r] = 0;
        break;
      }
      case CTL_BEGIN: {
        const double n0 = sqrt(sums[r]);
        st->rnorm0[r] = n0;
        st->rnorm[r] = n0;
        st->eps[r] = st->rtol * n0;
        st->act[r] = parent->act[r] && n0 > 0.0;
        st->l[r] = 0;
        st->flags[r] = 0;
        st->restart[r] = 0;
        break;
      }
      case CTL_TEST: {
        const bool active = st->act[r] != 0;
        const bool conv = !(st->rnorm[r] > st->eps[r]);
        if (st->level == 0) {
          st->claim[r] = active && conv;    // confirmed by a true residual first
          f_claim = active && conv;
        } else if (active && conv) {
          st->act[r] = 0;
        }
        st->restart[r] = st->act[r] && !st->claim[r] && st->l[r] > 0 && st->l[r] + st->per_cycle > st->cap;
        f_restart = st->restart[r] != 0;
        f_any = st->act[r] != 0;
        break;
      }
      case CTL_GRAM1: {
        const int l = st->l[r];
        double hh = 0.0;
        for (int i = 0; i < l; ++i) {
          const double h = sums[(size_t)i * 32 + r];
          hh += h * h;
          cw[(size_t)i * 32 + r] = h;
          cz[(size_t)i * 32 + r] = h;
        }
        const double naz2 = sums[(size_t)lcap * 32 + r];
        st->naz2[r] = naz2;
        const bool discard = !st->act[r] || !isfinite(naz2) || !(naz2 > 0.0);
        const bool reorth = !discard && l > 0 && (naz2 - hh < 0.25 * naz2);
        st->flags[r] = (discard ? MF_DISCARD : 0) | (reorth ? MF_REORTH : 0);
        f_reorth = reorth;
        break;
      }
      case CTL_GRAM2: {
        if (st->flags[r] & MF_REORTH) {
          for (int i = 0; i < st->l[r]; ++i) {
            const double h2 = sums[(size_t)i * 32 + r];
            cz[(size_t)i * 32 + r] += h2;
            cw[(size_t)i * 32 + r] = h2;
          }
        }
        f_reorth = (st->flags[r] & MF_REORTH) != 0;
        break;
      }
      case CTL_UPDATE: {
        const double nw = sqrt(sums[r]);
        bool discard = (st->flags[r] & MF_DISCARD) != 0;
        if (!isfinite(nw) || !(nw > st->brk_tol * sqrt(st->naz2[r]))) discard = true;
        st->gam[r] = discard ? 0.0 : 1.0 / nw;
        st->alp[r] = discard ? 0.0 : sums[32 + r] / nw;
        if (discard) st->flags[r] |= MF_DISCARD;
        f_reorth = (st->flags[r] & MF_REORTH) != 0;
        break;
      }
      case CTL_FINISH: {
        const bool discard = (st->flags[r] & MF_DISCARD) != 0;
        if (!discard) {
          st->l[r] += 1;
          st->rnorm[r] = sqrt(sums[r]);
          st->brk[r] = 0;
        } else if (st->act[r]) {
          if (++st->brk[r] >= 2 && st->level == 0) {   // two consecutive discards
            st->status = KCMG_BREAKDOWN;
            st->act[r] = 0;
          }
        }
        if (!isfinite(st->rnorm[r])) {
          st->status = KCMG_NONFINITE;
          st->act[r] = 0;
        }
        break;
      }
      case CTL_RESTART: {
        if (st->restart[r]) {
          st->rnorm[r] = sqrt(sums[r]);
          st->l[r] = 0;
          st->restart[r] = 0;
        }
        break;
      }
      case CTL_CONFIRM: {
        if (st->claim[r]) {
          const double rn = sqrt(sums[r]);
          st->rnorm[r] = rn;
          st->l[r] = 0;
          st->act[r] = rn > st->eps[r];
          st->claim[r] = 0;
        }
        break;
      }
      case CTL_ITEND:
        break;
    }
  }
  const int nact = __popc(__ballot_sync(0xffffffffu, r < R && st->act[r]));
  f_any = __any_sync(0xffffffffu, f_any);
  f_restart = __any_sync(0xffffffffu, f_restart);
  f_claim = __any_sync(0xffffffffu, f_claim);
  f_reorth = __any_sync(0xffffffffu, f_reorth);
  if (r == 0) {
    switch (kind) {
      case CTL_TEST: {
        const bool go = f_any && st->it < st->maxit && st->guard < st->guard_cap;
        st->any = go;
        st->any_restart = go && f_restart;
        st->any_claim = f_claim;
        st->nact = nact;
        if (go && !f_restart && !f_claim) st->guard++;
        break;
      }
      case CTL_GRAM1:
      case CTL_GRAM2:
      case CTL_UPDATE:
        st->any_reorth = f_reorth;
        break;
      case CTL_RESTART:
        st->nrestart++;
        break;
      case CTL_CONFIRM:
        st->nrestart++;
        break;
      case CTL_ITEND:
        st->it++;
        st->iters_total++;
        break;
      case CTL_BEGIN:
        st->it = 0;
        break;
      case CTL_INIT0:
        st->it = 0;
        break;
      default:
        break;
    }
  }
}

// restart mask for the confirmation of claims: the masked copy reads st->claim
__global__ void k_claim_mask(const MState* st, int* mask) {
  const int r = threadIdx.x;
  if (r < kMaxRhs) mask[r] = (r < st->R) ? st->claim[r] : 0;
}
__global__ void k_restart_mask(const MState* st, int* mask) {
  const int r = threadIdx.x;
  if (r < kMaxRhs) mask[r] = (r < st->R) ? st->restart[r] : 0;
}

// ---- bulk-copy pipeline for the tensor-core sweep (cp.async.bulk + mbarrier, inline PTX)
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok = 0;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// 1-D bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

template <int NP, int S> struct TcbShape {
  static constexpr int NF = S - 1;
  // floats of one stage for R right-hand sides: blocks, inverse, r, the NF neighbour slabs
  static __host__ __device__ int stage(int R) { return NF * NP * NP + NP * NP + NP * R + NF * NP * R; }
  // floats per warp: two stages, the T tile, two mbarriers (as 4 floats)
  static __host__ __device__ int warp(int R) { return 2 * stage(R) + TcShape<NP, S>::MT * 16 * TcShape<NP, S>::RS + 4; }
};

// One damped block-Jacobi sweep on the tensor cores (as k_msweep_tc) with each warp's cell
// data staged by 1-D bulk copies into two shared-memory stages: while the warp computes
// cell K, the copies of its next cell (the six off-diagonal FP32 blocks, an FP32 inverse,
// r and the six neighbour iterate slabs of NP x R values) are in flight.  BF16 inverses
// (not a multiple of 16 bytes per cell) are prefetched by the lanes into registers.  Every
// wait on a stage is bounded: on a timeout the kernel sets *err, waits (bounded) for its
// other stage and returns.  Needs NP * NP * 4 and NP * R * 4 to be multiples of 16 bytes.
template <int NP, int S, typename TI, typename TOUT>
__global__ void __launch_bounds__(256) k_msweep_tcb(const float* __restrict__ Ac, const TI* __restrict__ D,
                                                    const int* __restrict__ nbr, int C, int R,
                                                    const float* __restrict__ r32, const float* __restrict__ zo,
                                                    TOUT* __restrict__ zn, float om, int first, int x3, int* err) {
  using Sh = TcShape<NP, S>;
  constexpr int NF = S - 1, MT = Sh::MT, KS = Sh::KS, RS = Sh::RS, NT = Sh::NT;
  constexpr bool kBulkD = std::is_same<TI, float>::value;
  constexpr int DPL = (NP * NP + 31) / 32;   // inverse entries per lane (register prefetch)
  extern __shared__ float smem_tcb[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
  const int stg = TcbShape<NP, S>::stage(R);
  float* base = smem_tcb + (size_t)warp * TcbShape<NP, S>::warp(R);
  float* stage[2] = {base, base + stg};
  float* Ts = base + 2 * stg;
  uint64_t* bar = reinterpret_cast<uint64_t*>(Ts + MT * 16 * RS);   // 16-byte aligned (see warp())
  const int wpb = blockDim.x >> 5;
  const int nt_used = (R + 7) >> 3;
  const int stride = gridDim.x * wpb;
  const int K0 = blockIdx.x * wpb + warp;
  if (K0 >= C) return;
  if (lane == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  // the copies of cell K into stage st (lane 0)
  auto issue = [&](int st, int K) {
    float* As = stage[st];
    float* Ds = As + NF * NP * NP;
    float* rs = Ds + NP * NP;
    float* zs = rs + NP * R;
    const uint32_t slab = (uint32_t)(NP * R * sizeof(float));
    uint32_t bytes = slab + (kBulkD ? NP * NP * sizeof(float) : 0);
    int nb[NF];
    for (int s = 0; s < NF; ++s) {
      nb[s] = first ? -1 : __ldg(nbr + (size_t)K * NF + s);
      if (nb[s] >= 0) bytes += slab;
    }
    if (!first) bytes += NF * NP * NP * sizeof(float);
    // order this warp's earlier generic-proxy reads of the stage before the async writes
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&bar[st], bytes);
    if (!first) bulk_g2s(As, Ac + ((size_t)K * S + 1) * NP * NP, NF * NP * NP * sizeof(float), &bar[st]);
    if (kBulkD) bulk_g2s(Ds, reinterpret_cast<const float*>(D) + (size_t)K * NP * NP, NP * NP * sizeof(float), &bar[st]);
    bulk_g2s(rs, r32 + (size_t)K * NP * R, slab, &bar[st]);
    for (int s = 0; s < NF; ++s)
      if (nb[s] >= 0) bulk_g2s(zs + (size_t)s * NP * R, zo + (size_t)nb[s] * NP * R, slab, &bar[st]);
  };
  // bounded wait on a stage (lane 0 polls; the result is broadcast)
  auto wait = [&](int st, uint32_t parity) -> bool {
    int ok = 1;
    if (lane == 0) {
      long long spins = 0;
      while (!mbar_try_wait(&bar[st], parity)) {
        if (++spins > (1LL << 24)) { ok = 0; break; }
      }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    return ok != 0;
  };
  float dreg[DPL];   // BF16 inverse of the next cell, prefetched by the lanes
  auto load_d = [&](int K) {
    if (!kBulkD)
#pragma unroll
      for (int t = 0; t < DPL; ++t) {
        const int e = lane + 32 * t;
        dreg[t] = e < NP * NP ? to_f<TI>(D[(size_t)K * NP * NP + e]) : 0.f;
      }
  };
  if (lane == 0) issue(0, K0);
  load_d(K0);
  uint32_t phase[2] = {0u, 0u};
  bool pending[2] = {true, false};
  int it = 0;
  for (int K = K0; K < C; K += stride, ++it) {
    const int cur = it & 1, nxt = cur ^ 1;
    const int Kn = K + stride;
    // this cell's BF16 inverse from the registers into its stage
    if (!kBulkD) {
      float* Ds = stage[cur] + NF * NP * NP;
#pragma unroll
      for (int t = 0; t < DPL; ++t) {
        const int e = lane + 32 * t;
        if (e < NP * NP) Ds[e] = dreg[t];
      }
    }
    __syncwarp();
    if (Kn < C) {
      if (lane == 0) issue(nxt, Kn);
      pending[nxt] = true;
      load_d(Kn);
    }
    if (!wait(cur, phase[cur])) {
      if (lane == 0) atomicExch(err, 1);
      if (pending[nxt] && Kn < C) wait(nxt, phase[nxt]);
      return;
    }
    phase[cur] ^= 1u;
    pending[cur] = false;
    const float* As = stage[cur];
    const float* Ds = As + NF * NP * NP;
    const float* rb = Ds + NP * NP;
    const float* zsl = rb + NP * R;
    float c[MT][NT][4];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const int row0 = mt * 16 + gid, row1 = row0 + 8, col = nt * 8 + 2 * tig;
        c[mt][nt][0] = (row0 < NP && col < R) ? rb[row0 * R + col] : 0.f;
        c[mt][nt][1] = (row0 < NP && col + 1 < R) ? rb[row0 * R + col + 1] : 0.f;
        c[mt][nt][2] = (row1 < NP && col < R) ? rb[row1 * R + col] : 0.f;
        c[mt][nt][3] = (row1 < NP && col + 1 < R) ? rb[row1 * R + col + 1] : 0.f;
      }
    if (!first) {
#pragma unroll 1
      for (int s = 1; s < S; ++s) {
        const int J = __ldg(nbr + (size_t)K * NF + s - 1);
        if (J < 0) continue;
        const float* zb = zsl + (size_t)(s - 1) * NP * R;
        const float* Ab = As + (s - 1) * NP * NP;
#pragma unroll
        for (int kk = 0; kk < KS; ++kk) {
          const int q0 = kk * 8 + tig, q1 = q0 + 4;
          uint32_t bh[NT][2], bl[NT][2];
#pragma unroll
          for (int nt = 0; nt < NT; ++nt) {
            const int rr = nt * 8 + gid;
            const float v0 = (q0 < NP && rr < R) ? zb[q0 * R + rr] : 0.f;
            const float v1 = (q1 < NP && rr < R) ? zb[q1 * R + rr] : 0.f;
            tf32_split(v0, bh[nt][0], bl[nt][0]);
            tf32_split(v1, bh[nt][1], bl[nt][1]);
          }
#pragma unroll
          for (int mt = 0; mt < MT; ++mt) {
            const int row0 = mt * 16 + gid, row1 = row0 + 8;
            const float f0 = (row0 < NP && q0 < NP) ? -Ab[row0 * NP + q0] : 0.f;
            const float f1 = (row1 < NP && q0 < NP) ? -Ab[row1 * NP + q0] : 0.f;
            const float f2 = (row0 < NP && q1 < NP) ? -Ab[row0 * NP + q1] : 0.f;
            const float f3 = (row1 < NP && q1 < NP) ? -Ab[row1 * NP + q1] : 0.f;
            uint32_t ah[4], al[4];
            tf32_split(f0, ah[0], al[0]);
            tf32_split(f1, ah[1], al[1]);
            tf32_split(f2, ah[2], al[2]);
            tf32_split(f3, ah[3], al[3]);
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
              if (nt >= nt_used) break;
              if (x3) {
                mma_tf32(c[mt][nt], al, bh[nt]);
                mma_tf32(c[mt][nt], ah, bl[nt]);
              }
              mma_tf32(c[mt][nt], ah, bh[nt]);
            }
          }
        }
      }
    }
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const int row0 = mt * 16 + gid, row1 = row0 + 8, col = nt * 8 + 2 * tig;
        if (row0 < NP) { Ts[row0 * RS + col] = c[mt][nt][0]; Ts[row0 * RS + col + 1] = c[mt][nt][1]; }
        if (row1 < NP) { Ts[row1 * RS + col] = c[mt][nt][2]; Ts[row1 * RS + col + 1] = c[mt][nt][3]; }
      }
    __syncwarp();
    float e[MT][NT][4];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int k = 0; k < 4; ++k) e[mt][nt][k] = 0.f;
#pragma unroll
    for (int kk = 0; kk < KS; ++kk) {
      const int q0 = kk * 8 + tig, q1 = q0 + 4;
      uint32_t bh[NT][2], bl[NT][2];
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const int rr = nt * 8 + gid;
        const float v0 = (q0 < NP) ? Ts[q0 * RS + rr] : 0.f;
        const float v1 = (q1 < NP) ? Ts[q1 * RS + rr] : 0.f;
        tf32_split(v0, bh[nt][0], bl[nt][0]);
        tf32_split(v1, bh[nt][1], bl[nt][1]);
      }
#pragma unroll
      for (int mt = 0; mt < MT; ++mt) {
        const int row0 = mt * 16 + gid, row1 = row0 + 8;
        const float f0 = (row0 < NP && q0 < NP) ? Ds[row0 * NP + q0] : 0.f;
        const float f1 = (row1 < NP && q0 < NP) ? Ds[row1 * NP + q0] : 0.f;
        const float f2 = (row0 < NP && q1 < NP) ? Ds[row0 * NP + q1] : 0.f;
        const float f3 = (row1 < NP && q1 < NP) ? Ds[row1 * NP + q1] : 0.f;
        uint32_t ah[4], al[4];
        tf32_split(f0, ah[0], al[0]);
        tf32_split(f1, ah[1], al[1]);
        tf32_split(f2, ah[2], al[2]);
        tf32_split(f3, ah[3], al[3]);
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
          if (nt >= nt_used) break;
          if (x3) {
            mma_tf32(e[mt][nt], al, bh[nt]);
            mma_tf32(e[mt][nt], ah, bl[nt]);
          }
          mma_tf32(e[mt][nt], ah, bh[nt]);
        }
      }
    }
    // zn = (1 - om) zo + om E   (first sweep: om E); zo of cell K is its own iterate
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int row = mt * 16 + gid + ((k >> 1) << 3), col = nt * 8 + 2 * tig + (k & 1);
          if (row < NP && col < R) {
            const size_t o = ((size_t)K * NP + row) * R + col;
            const float v = first ? om * e[mt][nt][k] : fmaf(1.f - om, __ldg(zo + o), om * e[mt][nt][k]);
            zn[o] = (TOUT)v;
          }
        }
      }
    __syncwarp();
  }
}


}  // namespace

// ====================================================================== host engine
namespace {

struct Fail2 {
  kcmg_status st;
};

struct MLev {
  int n[3], C, N;
  const double* A64 = nullptr;   // natural FP64 blocks (owned by the context)
  const int* nbr = nullptr;
  double* D64 = nullptr;         // natural FP64 inverses (FP64 form)
  float* Acm = nullptr;          // cell-major FP32 blocks (mixed forms)
  float* D32 = nullptr;          // natural FP32 inverses
  __nv_bfloat16* D16 = nullptr;  // natural BF16 inverses
  double *x = nullptr, *r = nullptr, *b = nullptr, *z = nullptr, *w = nullptr, *wre = nullptr, *t = nullptr;
  double* zc = nullptr;          // level 0 of the task-parallel cycle: the coarse correction
  double *W = nullptr, *Z = nullptr;
  float *r32 = nullptr, *s0 = nullptr, *s1 = nullptr;
  int lcap = 0;
  MState* st = nullptr;
  // tuned launch shapes; sweep_kind: the FP32 sweep kernel (0: tensor cores, k_msweep_tc;
  // 1: tensor cores with bulk-copy staging, k_msweep_tcb; 2: CUDA cores, k_msweep_simt)
  int tc_wpb = 8, tc_grid = 0, sp_wpb = 8, sp_grid = 0, sweep_kind = 0;
  int tc_grid64 = 0;   // CUDA-core sweep: resident grid of its FP64-output form (last sweep)
};

}  // namespace

struct MrhsEngine {
  MrhsView v{};
  int R = 0, Ralloc = 0;
  int precision = 0;
  bool mixed = false;
  bool x3 = false;        // three-product TF32 smoother
  int nsm = 152;
  std::vector<MLev> lv;
  std::vector<void*> allocs;
  double *part = nullptr, *sums = nullptr, *cw = nullptr, *cz = nullptr;
  size_t part_len = 0;
  int* mask = nullptr;
  MState* hst = nullptr;  // pinned host copy of the flags
  long long launches = 0;
  std::vector<int> hist_act;   // active columns at each level-0 loop test
  std::string* err = nullptr;
  cudaStream_t s = nullptr;
  // autotuner record: per level 0 the chosen shapes and their times
  double tune[16] = {};
  int* tc_err = nullptr;  // set by the bulk-copy sweep when a copy did not complete in time
};

namespace {

#define MCK(call)                                                                     \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      if (E->err) {                                                                   \
        char b_[256];                                                                 \
        snprintf(b_, sizeof b_, "%s failed at %s:%d: %s", #call, __FILE__, __LINE__,  \
                 cudaGetErrorString(e_));                                             \
        *E->err = b_;                                                                 \
      }                                                                               \
      throw Fail2{e_ == cudaErrorMemoryAllocation ? KCMG_OOM : KCMG_CUDA_ERROR};      \
    }                                                                                 \
  } while (0)

template <typename T>
T* malloc_dev(MrhsEngine* E, size_t n) {
  void* p = nullptr;
  MCK(cudaMalloc(&p, n * sizeof(T) + 16));
  E->allocs.push_back(p);
  return static_cast<T*>(p);
}

int grid_for(size_t items, int per_block, int cap) {
  size_t g = (items + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if ((int)g > cap) g = cap;
  return (int)g;
}

#define MRHS_ND_SWITCH(np, dim, ...)                                      \
  switch ((np) * 10 + (dim)) {                                           \
    case 32: { constexpr int NP = 3, DIM = 2; __VA_ARGS__; break; }       \
    case 62: { constexpr int NP = 6, DIM = 2; __VA_ARGS__; break; }       \
    case 102: { constexpr int NP = 10, DIM = 2; __VA_ARGS__; break; }     \
    case 43: { constexpr int NP = 4, DIM = 3; __VA_ARGS__; break; }       \
    case 103: { constexpr int NP = 10, DIM = 3; __VA_ARGS__; break; }     \
    case 203: { constexpr int NP = 20, DIM = 3; __VA_ARGS__; break; }     \
    default: break;                                                      \
  }

// ---------------------------------------------------------------- launch wrappers
void spmm64(MrhsEngine* E, const MLev& L, const double* x, double* y, const double* b, int mode) {
  const int thr = L.sp_wpb * 32;
  const int grid = L.sp_grid > 0 ? L.sp_grid : grid_for(L.C, L.sp_wpb, 1 << 30);
  MRHS_ND_SWITCH(E->v.np, E->v.dim, {
    constexpr int S = 2 * DIM + 1;
    if (mode == 0) k_mspmm64<NP, S, 0><<<grid, thr, 0, E->s>>>(L.A64, L.nbr, L.C, E->R, x, y, b);
    else if (mode == 1) k_mspmm64<NP, S, 1><<<grid, thr, 0, E->s>>>(L.A64, L.nbr, L.C, E->R, x, y, b);
    else k_mspmm64<NP, S, 2><<<grid, thr, 0, E->s>>>(L.A64, L.nbr, L.C, E->R, x, y, b);
  });
  E->launches++;
}

template <typename TI, typename TOUT>
size_t tc_smem(int np, int dim, int wpb) {
  size_t ws = 0;
  MRHS_ND_SWITCH(np, dim, { ws = TcShape<NP, 2 * DIM + 1>::WS; });
  return ws * sizeof(float) * wpb;
}

template <typename TI, typename TOUT>
void sweep_tc(MrhsEngine* E, const MLev& L, const TI* D, const float* r32, const float* zo, TOUT* zn,
              int first, int wpb, int grid) {
  const size_t sm = tc_smem<TI, TOUT>(E->v.np, E->v.dim, wpb);
  MRHS_ND_SWITCH(E->v.np, E->v.dim, {
    constexpr int S = 2 * DIM + 1;
    auto kern = k_msweep_tc<NP, S, TI, TOUT>;
    kern<<<grid, wpb * 32, sm, E->s>>>(L.Acm, D, L.nbr, L.C, E->R, r32, zo, zn, (float)E->v.omega, first,
                                       E->x3 ? 1 : 0);
  });
  E->launches++;
}

// the bulk-copy sweep applies when every staged piece is a multiple of 16 bytes
bool tcb_ok(const MrhsEngine* E) {
  const int np = E->v.np;
  return (np * np * 4) % 16 == 0 && (np * E->R * 4) % 16 == 0;
}

size_t tcb_smem(int np, int dim, int R, int wpb) {
  size_t ws = 0;
  MRHS_ND_SWITCH(np, dim, { ws = TcbShape<NP, 2 * DIM + 1>::warp(R); });
  return ws * sizeof(float) * wpb;
}

template <typename TI, typename TOUT>
void sweep_tcb(MrhsEngine* E, const MLev& L, const TI* D, const float* r32, const float* zo, TOUT* zn,
               int first, int wpb, int grid) {
  const size_t sm = tcb_smem(E->v.np, E->v.dim, E->R, wpb);
  MRHS_ND_SWITCH(E->v.np, E->v.dim, {
    constexpr int S = 2 * DIM + 1;
    auto kern = k_msweep_tcb<NP, S, TI, TOUT>;
    kern<<<grid, wpb * 32, sm, E->s>>>(L.Acm, D, L.nbr, L.C, E->R, r32, zo, zn, (float)E->v.omega, first,
                                       E->x3 ? 1 : 0, E->tc_err);
  });
  E->launches++;
}

template <typename TI, typename TOUT>
void sweep_simt(MrhsEngine* E, const MLev& L, const TI* D, const float* r32, const float* zo, TOUT* zn,
                int first, int wpb, int grid) {
  launch_msweep_simt<TI, TOUT>(E->v.np, E->v.dim, L.Acm, D, L.nbr, L.C, E->R, r32, zo, zn, (float)E->v.omega,
                               first, wpb, grid, E->s);
  E->launches++;
}

// the resident grid of the CUDA-core sweep (blocks per SM from the occupancy of the
// instantiation: registers and shared memory), so that every warp starts at once
int simt_grid(const MrhsEngine* E, const MLev& L, int wpb, bool out64 = false) {
  const int per_sm = msweep_simt_blocks_per_sm(E->v.np, E->v.dim, L.D16 != nullptr, E->R, wpb, out64);
  return std::min(grid_for(msweep_simt_units(E->v.np, E->R, L.C), wpb, 1 << 30), E->nsm * per_sm);
}

// allow the tensor-core sweeps the device's opt-in shared memory
void tc_prepare(MrhsEngine* E) {
  int dev = 0, optin = 0;
  MCK(cudaGetDevice(&dev));
  MCK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  MRHS_ND_SWITCH(E->v.np, E->v.dim, {
    constexpr int S = 2 * DIM + 1;
    MCK(cudaFuncSetAttribute(k_msweep_tc<NP, S, float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    MCK(cudaFuncSetAttribute(k_msweep_tc<NP, S, float, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    MCK(cudaFuncSetAttribute(k_msweep_tc<NP, S, __nv_bfloat16, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    MCK(cudaFuncSetAttribute(k_msweep_tc<NP, S, __nv_bfloat16, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    MCK(cudaFuncSetAttribute(k_msweep_tcb<NP, S, float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    MCK(cudaFuncSetAttribute(k_msweep_tcb<NP, S, float, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    MCK(cudaFuncSetAttribute(k_msweep_tcb<NP, S, __nv_bfloat16, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    MCK(cudaFuncSetAttribute(k_msweep_tcb<NP, S, __nv_bfloat16, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
  });
  MCK(msweep_simt_prepare(E->v.np, E->v.dim, optin));
}

void sweep64(MrhsEngine* E, const MLev& L, const double* rv, const double* zo, double* zn, int first) {
  const int thr = L.sp_wpb * 32;
  const int grid = L.sp_grid > 0 ? L.sp_grid : grid_for(L.C, L.sp_wpb, 1 << 30);
  MRHS_ND_SWITCH(E->v.np, E->v.dim, {
    constexpr int S = 2 * DIM + 1;
    k_msweep64<NP, S><<<grid, thr, 0, E->s>>>(L.A64, L.D64, L.nbr, L.C, E->R, rv, zo, zn, E->v.omega, first);
  });
  E->launches++;
}

int gram_grid(const MLev& L) { return grid_for((size_t)L.N, kGramWarps, kGramBlocks); }

void ctl(MrhsEngine* E, int lev, int kind, const MState* parent = nullptr) {
  k_mctl<<<1, 32, 0, E->s>>>(E->lv[lev].st, parent, E->sums, E->cw, E->cz, kind);
  E->launches++;
}

void reduce(MrhsEngine* E, int nblk, int ncols, const MState* st, int limit) {
  k_mreduce<<<ncols, 256, 0, E->s>>>(E->part, nblk, ncols, st, limit, E->sums);
  E->launches++;
}

// per-RHS ||v||^2 -> sums[0..R)
void norms(MrhsEngine* E, const MLev& L, const double* vv) {
  const int g = gram_grid(L);
  k_mnorm<<<g, kGramWarps * 32, 0, E->s>>>(vv, L.N, E->R, E->part);
  E->launches++;
  reduce(E, g, 1, nullptr, 0);
}

void read_flags(MrhsEngine* E, int lev) {
  MCK(cudaMemcpyAsync(E->hst, E->lv[lev].st, 32, cudaMemcpyDeviceToHost, E->s));
  MCK(cudaStreamSynchronize(E->s));
}

// ---------------------------------------------------------------- cycle pieces
// z = BJ(r) on level lev (sweeps from z = 0); the result is L.z (FP64)
void smooth(MrhsEngine* E, int lev) {
  MLev& L = E->lv[lev];
  const int sw = E->v.sweeps;
  if (!E->mixed) {
    double* buf[2] = {L.t, L.wre};
    for (int k = 0; k < sw; ++k) {
      const double* zo = buf[(k + 1) & 1];
      double* zn = (k == sw - 1) ? L.z : buf[k & 1];
      sweep64(E, L, L.r, zo, zn, k == 0);
    }
    return;
  }
  const size_t n = (size_t)L.N * E->R;
  k_mto_f32<<<grid_for(n, 256, 4 * E->nsm * 8), 256, 0, E->s>>>(L.r, L.r32, n);
  E->launches++;
  float* buf[2] = {L.s0, L.s1};
  for (int k = 0; k < sw; ++k) {
    const float* zo = buf[(k + 1) & 1];
    const int grid = L.tc_grid > 0 ? L.tc_grid : grid_for(L.C, L.tc_wpb, 1 << 30);
    if (L.sweep_kind == 2) {
      if (k == sw - 1) {
        const int g64 = L.tc_grid64 > 0 ? L.tc_grid64 : grid;
        if (L.D16) sweep_simt<__nv_bfloat16, double>(E, L, L.D16, L.r32, zo, L.z, k == 0, L.tc_wpb, g64);
        else sweep_simt<float, double>(E, L, L.D32, L.r32, zo, L.z, k == 0, L.tc_wpb, g64);
      } else {
        if (L.D16) sweep_simt<__nv_bfloat16, float>(E, L, L.D16, L.r32, zo, buf[k & 1], k == 0, L.tc_wpb, grid);
        else sweep_simt<float, float>(E, L, L.D32, L.r32, zo, buf[k & 1], k == 0, L.tc_wpb, grid);
      }
      continue;
    }
    if (L.sweep_kind == 1) {
      if (k == sw - 1) {
        if (L.D16) sweep_tcb<__nv_bfloat16, double>(E, L, L.D16, L.r32, zo, L.z, k == 0, L.tc_wpb, grid);
        else sweep_tcb<float, double>(E, L, L.D32, L.r32, zo, L.z, k == 0, L.tc_wpb, grid);
      } else {
        if (L.D16) sweep_tcb<__nv_bfloat16, float>(E, L, L.D16, L.r32, zo, buf[k & 1], k == 0, L.tc_wpb, grid);
        else sweep_tcb<float, float>(E, L, L.D32, L.r32, zo, buf[k & 1], k == 0, L.tc_wpb, grid);
      }
      continue;
    }
    if (k == sw - 1) {
      if (L.D16) sweep_tc<__nv_bfloat16, double>(E, L, L.D16, L.r32, zo, L.z, k == 0, L.tc_wpb, grid);
      else sweep_tc<float, double>(E, L, L.D32, L.r32, zo, L.z, k == 0, L.tc_wpb, grid);
    } else {
      if (L.D16) sweep_tc<__nv_bfloat16, float>(E, L, L.D16, L.r32, zo, buf[k & 1], k == 0, L.tc_wpb, grid);
      else sweep_tc<float, float>(E, L, L.D32, L.r32, zo, buf[k & 1], k == 0, L.tc_wpb, grid);
    }
  }
}

// Alg. 1 for every right-hand side at once on the correction zcor (default: L.z)
void rm(MrhsEngine* E, int lev, const double* zcor = nullptr) {
  MLev& L = E->lv[lev];
  const int R = E->R, g = gram_grid(L), thr = kGramWarps * 32;
  const double* zz = zcor ? zcor : L.z;
  spmm64(E, L, zz, L.w, nullptr, 0);                                     // w = A z
  k_mdots<<<g, thr, 0, E->s>>>(L.W, L.w, L.N, R, L.lcap, L.st, E->part, 0);
  reduce(E, g, L.lcap + 1, L.st, 1);
  ctl(E, lev, CTL_GRAM1);
  k_mapply<<<g, thr, 0, E->s>>>(L.W, L.w, L.wre, L.N, R, L.st, E->sums);   // sums = h (pass 1)
  k_mdots<<<g, thr, 0, E->s>>>(L.W, L.wre, L.N, R, L.lcap, L.st, E->part, 1);
  E->launches += 3;
  // pass 2 results: the reduce reads only when some right-hand side reorthogonalised;
  // otherwise the partials are stale but CTL_GRAM2 ignores them (no REORTH flags)
  reduce(E, g, L.lcap + 1, L.st, 1);
  ctl(E, lev, CTL_GRAM2);
  k_mupdate<<<g, thr, 0, E->s>>>(L.W, L.Z, L.N, R, L.w, L.wre, zz, L.r, L.st, E->cw, E->cz, E->part);
  E->launches++;
  reduce(E, g, 2, nullptr, 0);
  ctl(E, lev, CTL_UPDATE);
  k_mfinish<<<g, thr, 0, E->s>>>(L.W, L.Z, L.N, R, L.x, L.r, L.st, E->part);
  E->launches++;
  reduce(E, g, 1, nullptr, 0);
  ctl(E, lev, CTL_FINISH);
}

void restrict_to(MrhsEngine* E, int lev, bool start) {
  MLev &F = E->lv[lev], &C = E->lv[lev + 1];
  const int g = grid_for(C.C, 8, 4096);
  MRHS_ND_SWITCH(E->v.np, E->v.dim, {
    k_mrestrict<NP, DIM><<<g, 256, 0, E->s>>>(F.r, F.n[0], F.n[1], C.n[0], C.n[1], C.C, E->v.P, E->R, C.b,
                                              start ? C.r : nullptr, start ? C.x : nullptr, start ? E->part : nullptr);
  });
  E->launches++;
  if (start) reduce(E, g, 1, nullptr, 0);
}

void prolong_from(MrhsEngine* E, int lev, double* target = nullptr) {
  MLev &F = E->lv[lev], &C = E->lv[lev + 1];
  const int g = grid_for(F.C, 8, 1 << 30);
  double* zf = target ? target : F.z;
  MRHS_ND_SWITCH(E->v.np, E->v.dim, {
    k_mprolong<NP, DIM><<<g, 256, 0, E->s>>>(C.x, F.n[0], F.n[1], F.C, C.n[0], C.n[1], E->v.P, E->R, zf);
  });
  E->launches++;
}

void coarse_solve(MrhsEngine* E) {
  MLev& C = E->lv[E->v.nlev - 1];
  k_mcoarse<<<grid_for(E->v.Nc, 8, 1 << 30), 256, 0, E->s>>>(E->v.Ainv, E->v.Nc, E->R, C.b, C.x);
  E->launches++;
}

// r = b - A x for the right-hand sides in the restart mask (level lev)
void restart(MrhsEngine* E, int lev, bool confirm) {
  MLev& L = E->lv[lev];
  spmm64(E, L, L.x, L.t, L.b, lev == 0 ? 2 : 1);
  if (confirm) k_claim_mask<<<1, 32, 0, E->s>>>(L.st, E->mask);
  else k_restart_mask<<<1, 32, 0, E->s>>>(L.st, E->mask);
  const size_t n = (size_t)L.N * E->R;
  k_mcopy_masked<<<grid_for(n, 256, E->nsm * 16), 256, 0, E->s>>>(L.t, L.r, L.N, E->R, E->mask);
  E->launches += 2;
  norms(E, L, L.t);
  ctl(E, lev, confirm ? CTL_CONFIRM : CTL_RESTART);
}

// MG(lev) of Alg. 2 for all right-hand sides; on entry b, r, x and the state are set
void mg(MrhsEngine* E, int lev) {
  MLev& L = E->lv[lev];
  const int nlev = E->v.nlev;
  for (;;) {
    ctl(E, lev, CTL_TEST);
    read_flags(E, lev);
    if (lev == 0) E->hist_act.push_back(E->hst->nact);
    if (E->hst->any_claim) { restart(E, lev, true); continue; }
    if (!E->hst->any) break;
    if (E->hst->any_restart) { restart(E, lev, false); continue; }
    smooth(E, lev);                                   // pre-smoother
    rm(E, lev);
    if (lev + 1 == nlev - 1) {                        // direct coarsest solve
      restrict_to(E, lev, false);
      coarse_solve(E);
    } else {
      restrict_to(E, lev, true);
      ctl(E, lev + 1, CTL_BEGIN, L.st);
      mg(E, lev + 1);
    }
    prolong_from(E, lev);                             // coarse correction
    rm(E, lev);
    smooth(E, lev);                                   // post-smoother
    rm(E, lev);
    ctl(E, lev, CTL_ITEND);
  }
}

// Level 0 as Alg. AsyncMG with a fixed smoother count m (v.async_smooth): per cycle the
// coarse path works on the cycle-start residual (restriction, MG on level 1 or the direct
// solve, prolongation into zc); the smoother path applies m smoother + RM steps; one RM
// with zc closes the cycle.  The batched engine runs on one stream, so the coarse path is
// issued first: it reads only the cycle-start residual and writes only level >= 1 buffers
// and zc, so the iterates are those of the concurrent form.
void mg_async0(MrhsEngine* E) {
  MLev& L = E->lv[0];
  const int nlev = E->v.nlev;
  for (;;) {
    ctl(E, 0, CTL_TEST);
    read_flags(E, 0);
    E->hist_act.push_back(E->hst->nact);
    if (E->hst->any_claim) { restart(E, 0, true); continue; }
    if (!E->hst->any) break;
    if (E->hst->any_restart) { restart(E, 0, false); continue; }
    if (nlev == 2) {                                  // coarse path
      restrict_to(E, 0, false);
      coarse_solve(E);
    } else {
      restrict_to(E, 0, true);
      ctl(E, 1, CTL_BEGIN, L.st);
      mg(E, 1);
    }
    prolong_from(E, 0, L.zc);
    for (int k = 0; k < E->v.async_smooth; ++k) {    // smoother path
      smooth(E, 0);
      rm(E, 0);
    }
    rm(E, 0, L.zc);                                   // the synchronisation
    ctl(E, 0, CTL_ITEND);
  }
}

// ---------------------------------------------------------------- setup of the engine
void init_state(MrhsEngine* E, int lev, double rtol, double atol, int maxit, long long guard_cap) {
  MState h;
  memset(&h, 0, sizeof h);
  h.R = E->R;
  h.level = lev;
  h.lcap = E->lv[lev].lcap;
  h.maxit = maxit;
  h.rtol = rtol;
  h.atol = atol;
  h.brk_tol = 1e-14;
  h.guard_cap = (int)std::min<long long>(guard_cap, 1LL << 30);
  h.per_cycle = (lev == 0 && E->v.async_smooth > 0) ? E->v.async_smooth + 1 : 3;
  // the restart length: lmax where it binds (as in the single-column solve), else capacity
  h.cap = (E->v.lmax > 0 && E->v.lmax < h.lcap) ? E->v.lmax : h.lcap;
  h.status = KCMG_OK;
  MCK(cudaMemcpyAsync(E->lv[lev].st, &h, sizeof h, cudaMemcpyHostToDevice, E->s));
}

// time a launch shape (CUDA events, best of reps)
template <typename F>
float time_it(MrhsEngine* E, F&& f, int reps) {
  cudaEvent_t a, b;
  MCK(cudaEventCreate(&a));
  MCK(cudaEventCreate(&b));
  f();   // warm-up
  float best = 1e30f;
  for (int i = 0; i < reps; ++i) {
    MCK(cudaEventRecord(a, E->s));
    f();
    MCK(cudaEventRecord(b, E->s));
    MCK(cudaEventSynchronize(b));
    float ms = 0;
    MCK(cudaEventElapsedTime(&ms, a, b));
    best = std::min(best, ms);
  }
  MCK(cudaGetLastError());
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return best;
}

// Autotuner: for every level with enough cells, time the candidate kernels and launch
// shapes of the FP32 smoother sweep (tensor cores: warps per block x grid; tensor cores
// with bulk-copy staging and the CUDA-core sweep: warps per block on a resident grid) and
// of the FP64 operator (warps per block) on the level's own buffers; keep the fastest.
void autotune(MrhsEngine* E) {
  int dev = 0, smem_optin = 0;
  MCK(cudaGetDevice(&dev));
  MCK(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  // KCMG_SWEEP = tc | tcb | simt runs every level's FP32 sweep with that kernel (tests,
  // tuning); unset, the tuner times all three and keeps the fastest
  const char* fk = getenv("KCMG_SWEEP");
  int force_kind = -1;
  if (fk && !strcmp(fk, "tc")) force_kind = 0;
  else if (fk && !strcmp(fk, "tcb")) force_kind = 1;
  else if (fk && !strcmp(fk, "simt")) force_kind = 2;
  for (int lev = 0; lev < E->v.nlev - 1; ++lev) {
    MLev& L = E->lv[lev];
    if (L.C < 256) continue;                        // small levels: defaults
    const int reps = lev == 0 ? 3 : 5;
    // FP64 operator: warps per block
    float best = 1e30f;
    int best_w = L.sp_wpb;
    for (int wpb : {4, 8}) {
      L.sp_wpb = wpb;
      L.sp_grid = 0;
      const float ms = time_it(E, [&] { spmm64(E, L, L.z, L.w, nullptr, 0); }, reps);
      if (ms < best) { best = ms; best_w = wpb; }
    }
    L.sp_wpb = best_w;
    if (lev == 0) { E->tune[0] = best_w; E->tune[1] = best; }
    if (!E->mixed) continue;
    // tensor-core sweep: warps per block and grid (one warp per cell, or a resident grid)
    float bt = 1e30f;
    int bw = L.tc_wpb, bg = 0, bk = 0;
    if (force_kind <= 0)
    for (int wpb : {2, 4, 8, 16}) {
      size_t sm = L.D16 ? tc_smem<__nv_bfloat16, float>(E->v.np, E->v.dim, wpb)
                        : tc_smem<float, float>(E->v.np, E->v.dim, wpb);
      if ((int)sm > smem_optin) continue;
      int per_sm = std::max(1, (int)(smem_optin / std::max<size_t>(sm, 1)));
      per_sm = std::min(per_sm, 64 / wpb);
      for (int gmode = 0; gmode < 2; ++gmode) {
        const int grid = gmode == 0 ? grid_for(L.C, wpb, 1 << 30) : std::min(grid_for(L.C, wpb, 1 << 30), E->nsm * per_sm);
        const float ms = time_it(E, [&] {
          if (L.D16) sweep_tc<__nv_bfloat16, float>(E, L, L.D16, L.r32, L.s0, L.s1, 0, wpb, grid);
          else sweep_tc<float, float>(E, L, L.D32, L.r32, L.s0, L.s1, 0, wpb, grid);
        }, reps);
        if (ms < bt) { bt = ms; bw = wpb; bg = gmode == 0 ? 0 : grid; }
      }
    }
    // the bulk-copy pipeline: warps per block, resident grid
    if (tcb_ok(E) && (force_kind == -1 || force_kind == 1))
      for (int wpb : {2, 4, 8}) {
        const size_t sm = tcb_smem(E->v.np, E->v.dim, E->R, wpb);
        if ((int)sm > smem_optin) continue;
        const int per_sm = std::max(1, std::min((int)(smem_optin / sm), 64 / wpb));
        const int grid = std::min(grid_for(L.C, wpb, 1 << 30), E->nsm * per_sm);
        const float ms = time_it(E, [&] {
          if (L.D16) sweep_tcb<__nv_bfloat16, float>(E, L, L.D16, L.r32, L.s0, L.s1, 0, wpb, grid);
          else sweep_tcb<float, float>(E, L, L.D32, L.r32, L.s0, L.s1, 0, wpb, grid);
        }, reps);
        if (ms < bt) { bt = ms; bw = wpb; bg = grid; bk = 1; }
      }
    // the CUDA-core sweep: warps per block, resident grid
    if (force_kind == -1 || force_kind == 2)
      for (int wpb : {1, 2, 4, 8}) {
        if ((int)msweep_simt_smem(E->v.np, E->v.dim, L.D16 != nullptr, E->R, wpb) > smem_optin) continue;
        const int grid = simt_grid(E, L, wpb);
        const float ms = time_it(E, [&] {
          if (L.D16) sweep_simt<__nv_bfloat16, float>(E, L, L.D16, L.r32, L.s0, L.s1, 0, wpb, grid);
          else sweep_simt<float, float>(E, L, L.D32, L.r32, L.s0, L.s1, 0, wpb, grid);
        }, reps);
        if (ms < bt) { bt = ms; bw = wpb; bg = grid; bk = 2; }
      }
    L.tc_wpb = bw;
    L.tc_grid = bg;
    L.sweep_kind = bk;
    L.tc_grid64 = bk == 2 ? simt_grid(E, L, bw, true) : 0;
    if (lev == 0) { E->tune[2] = bw; E->tune[3] = bg; E->tune[4] = bt; E->tune[8] = bk; }
  }
  // a forced kernel also runs on the small levels the tuner skips
  if (E->mixed && force_kind >= 1 && (force_kind == 2 || tcb_ok(E))) {
    for (int lev = 0; lev < E->v.nlev - 1; ++lev) {
      MLev& L = E->lv[lev];
      if (L.sweep_kind == force_kind) continue;
      int wpb = 4;   // the widest block (up to 4 warps) whose stages fit the opt-in shared memory
      if (force_kind == 1) {
        while (wpb > 1 && (int)tcb_smem(E->v.np, E->v.dim, E->R, wpb) > smem_optin) wpb /= 2;
        const size_t sm = tcb_smem(E->v.np, E->v.dim, E->R, wpb);
        if ((int)sm > smem_optin) continue;
        const int per_sm = std::max(1, std::min((int)(smem_optin / sm), 16));
        L.tc_grid = std::min(grid_for(L.C, wpb, 1 << 30), E->nsm * per_sm);
      } else {
        while (wpb > 1 && (int)msweep_simt_smem(E->v.np, E->v.dim, L.D16 != nullptr, E->R, wpb) > smem_optin) wpb /= 2;
        L.tc_grid = simt_grid(E, L, wpb);
        L.tc_grid64 = simt_grid(E, L, wpb, true);
      }
      L.sweep_kind = force_kind;
      L.tc_wpb = wpb;
      if (lev == 0) { E->tune[2] = wpb; E->tune[3] = L.tc_grid; E->tune[8] = force_kind; }
    }
  }
  E->launches = 0;
}

void build(MrhsEngine* E, const MrhsView& v, int R) {
  E->v = v;
  E->R = R;
  E->Ralloc = R;
  E->precision = v.precision;
  E->mixed = v.precision != KCMG_FP64;
  E->s = v.s;
  int dev = 0;
  MCK(cudaGetDevice(&dev));
  MCK(cudaDeviceGetAttribute(&E->nsm, cudaDevAttrMultiProcessorCount, dev));
  const int np = v.np, S = 2 * v.dim + 1;
  const size_t bs = (size_t)np * np;
  E->lv.resize(v.nlev);
  int* fail = malloc_dev<int>(E, 1);
  E->tc_err = malloc_dev<int>(E, 1);
  MCK(cudaMemsetAsync(E->tc_err, 0, sizeof(int), E->s));
  double* inv = nullptr;
  for (int l = 0; l < v.nlev; ++l) {
    MLev& L = E->lv[l];
    for (int j = 0; j < 3; ++j) L.n[j] = v.n[l][j];
    L.C = v.ncell[l];
    L.N = v.N[l];
    L.A64 = v.nat[l];
    L.nbr = v.nbr[l];
  }
  inv = malloc_dev<double>(E, (size_t)E->lv[0].C * bs);
  size_t free_b = 0, tot_b = 0;
  for (int l = 0; l < v.nlev - 1; ++l) {
    MLev& L = E->lv[l];
    const size_t NR = (size_t)L.N * R;
    MCK(cudaMemsetAsync(fail, 0, sizeof(int), E->s));
    launch_block_inverse(np, L.A64, L.C, inv, fail, E->s);
    MCK(cudaGetLastError());
    if (!E->mixed) {
      L.D64 = malloc_dev<double>(E, L.C * bs);
      MCK(cudaMemcpyAsync(L.D64, inv, L.C * bs * sizeof(double), cudaMemcpyDeviceToDevice, E->s));
    } else {
      L.Acm = malloc_dev<float>(E, (size_t)S * L.C * bs);
      k_cellmajor_f32<<<grid_for((size_t)S * L.C * bs, 256, 8192), 256, 0, E->s>>>(L.A64, S, L.C, (int)bs, L.Acm);
      if (v.precision == KCMG_MIXED_BF16INV) {
        L.D16 = malloc_dev<__nv_bfloat16>(E, L.C * bs);
        k_narrow<__nv_bfloat16><<<grid_for(L.C * bs, 256, 8192), 256, 0, E->s>>>(inv, L.D16, L.C * bs);
      } else {
        L.D32 = malloc_dev<float>(E, L.C * bs);
        k_narrow<float><<<grid_for(L.C * bs, 256, 8192), 256, 0, E->s>>>(inv, L.D32, L.C * bs);
      }
      L.r32 = malloc_dev<float>(E, NR);
      L.s0 = malloc_dev<float>(E, NR);
      L.s1 = malloc_dev<float>(E, NR);
    }
    MCK(cudaGetLastError());
    L.x = malloc_dev<double>(E, NR);
    L.r = malloc_dev<double>(E, NR);
    L.b = malloc_dev<double>(E, NR);
    L.z = malloc_dev<double>(E, NR);
    L.w = malloc_dev<double>(E, NR);
    L.wre = malloc_dev<double>(E, NR);
    L.t = malloc_dev<double>(E, NR);
    if (l == 0 && v.async_smooth > 0) L.zc = malloc_dev<double>(E, NR);
    L.st = malloc_dev<MState>(E, 1);
    // basis capacity: level 0 from lmax (default 60), coarse levels from their iteration
    // caps (3 corrections per cycle); level 0 shrinks to what the device can hold
    int cap;
    const int per_cycle0 = std::max(3, v.async_smooth + 1);   // corrections of one level-0 cycle
    if (l == 0) cap = (v.lmax > 0 ? v.lmax : 60) + per_cycle0;
    else cap = 3 * std::max(1, v.lvl_maxit[l]) + 3;
    if (v.lmax > 0 && l > 0) cap = std::min(cap, v.lmax + 3);
    if (l == 0) {
      // reserve the coarse levels' bases (an eighth per level) and a margin
      MCK(cudaMemGetInfo(&free_b, &tot_b));
      const size_t per = 2 * NR * sizeof(double);
      const size_t budget = free_b > ((size_t)4 << 30) ? (size_t)((free_b - ((size_t)4 << 30)) * 0.8) : free_b / 2;
      while (cap > 6 && (size_t)cap * per > budget) cap = cap * 3 / 4;
      if (cap < per_cycle0 + 3) cap = per_cycle0 + 3;   // one cycle must always fit
    }
    L.lcap = cap;
    L.W = malloc_dev<double>(E, (size_t)cap * NR);
    L.Z = malloc_dev<double>(E, (size_t)cap * NR);
    MCK(cudaMemsetAsync(L.z, 0, NR * sizeof(double), E->s));
    if (E->mixed) {
      MCK(cudaMemsetAsync(L.r32, 0, NR * sizeof(float), E->s));
      MCK(cudaMemsetAsync(L.s0, 0, NR * sizeof(float), E->s));
    }
  }
  {
    MLev& C = E->lv[v.nlev - 1];
    C.b = malloc_dev<double>(E, (size_t)C.N * R);
    C.x = malloc_dev<double>(E, (size_t)C.N * R);
  }
  int hostfail = 0;
  MCK(cudaMemcpyAsync(&hostfail, fail, sizeof(int), cudaMemcpyDeviceToHost, E->s));
  MCK(cudaStreamSynchronize(E->s));
  if (hostfail) {
    if (E->err) *E->err = "singular diagonal block";
    throw Fail2{KCMG_SINGULAR};
  }
  int maxcols = 2;
  for (int l = 0; l < v.nlev - 1; ++l) maxcols = std::max(maxcols, E->lv[l].lcap + 1);
  E->part_len = (size_t)kGramBlocks * maxcols * 32;
  const size_t rblocks = (size_t)grid_for(E->lv[1].C, 8, 4096);
  E->part_len = std::max(E->part_len, rblocks * 32);
  E->part = malloc_dev<double>(E, E->part_len);
  E->sums = malloc_dev<double>(E, (size_t)maxcols * 32);
  E->cw = malloc_dev<double>(E, (size_t)maxcols * 32);
  E->cz = malloc_dev<double>(E, (size_t)maxcols * 32);
  E->mask = malloc_dev<int>(E, kMaxRhs);
  MCK(cudaMallocHost(&E->hst, sizeof(MState)));
  if (E->mixed) tc_prepare(E);
  autotune(E);
}

}  // namespace

kcmg_status mrhs_ensure(MrhsEngine** peng, const MrhsView& v, int R, std::string* err) {
  MrhsEngine* E = *peng;
  if (E && (E->Ralloc != R || E->precision != v.precision || E->v.async_smooth != v.async_smooth)) {
    mrhs_destroy(E);
    E = *peng = nullptr;
  }
  try {
    if (!E) {
      E = new MrhsEngine();
      E->err = err;
      *peng = E;
      E->x3 = v.tc_tf32_only == 0;
      build(E, v, R);
    }
    E->err = err;
    E->x3 = v.tc_tf32_only == 0;
    E->v.tc_tf32_only = v.tc_tf32_only;
    return KCMG_OK;
  } catch (Fail2& f) {
    return f.st;
  }
}

kcmg_status mrhs_apply(MrhsEngine* E, int level, const double* x, double* y) {
  try {
    MLev& L = E->lv[level];
    const size_t NR = (size_t)L.N * E->R;
    MCK(cudaMemcpyAsync(L.z, x, NR * sizeof(double), cudaMemcpyDefault, E->s));
    spmm64(E, L, L.z, L.w, nullptr, 0);
    MCK(cudaGetLastError());
    MCK(cudaMemcpyAsync(y, L.w, NR * sizeof(double), cudaMemcpyDefault, E->s));
    MCK(cudaStreamSynchronize(E->s));
    return KCMG_OK;
  } catch (Fail2& f) {
    return f.st;
  }
}

kcmg_status mrhs_smooth(MrhsEngine* E, int level, const double* r, double* z) {
  try {
    MLev& L = E->lv[level];
    const size_t NR = (size_t)L.N * E->R;
    MCK(cudaMemcpyAsync(L.r, r, NR * sizeof(double), cudaMemcpyDefault, E->s));
    smooth(E, level);
    MCK(cudaGetLastError());
    MCK(cudaMemcpyAsync(z, L.z, NR * sizeof(double), cudaMemcpyDefault, E->s));
    MCK(cudaStreamSynchronize(E->s));
    return KCMG_OK;
  } catch (Fail2& f) {
    return f.st;
  }
}

kcmg_status mrhs_solve(MrhsEngine** peng, const MrhsView& v, const double* b, double* x, int R, double rtol,
                       double atol, int maxiter, kcmg_info* info, std::string* err) {
  kcmg_status es = mrhs_ensure(peng, v, R, err);
  if (es != KCMG_OK) return es;
  MrhsEngine* E = *peng;
  try {
    E->err = err;
    E->R = R;
    E->launches = 0;
    E->hist_act.clear();
    MLev& L = E->lv[0];
    const size_t NR = (size_t)L.N * R;
    MCK(cudaMemcpyAsync(L.b, b, NR * sizeof(double), cudaMemcpyDefault, E->s));
    MCK(cudaMemcpyAsync(L.x, x, NR * sizeof(double), cudaMemcpyDefault, E->s));
    long long cap = (long long)maxiter + 2;
    for (int l = 0; l < v.nlev - 1; ++l) {
      if (l > 0) cap = std::min<long long>(cap * std::max(1, v.lvl_maxit[l]) + 2, 1LL << 30);
      init_state(E, l, l == 0 ? rtol : v.lvl_rtol[l], l == 0 ? atol : 0.0, l == 0 ? maxiter : v.lvl_maxit[l], cap);
    }
    // r0 = b - A x0 (compensated), ||r0|| per right-hand side
    spmm64(E, L, L.x, L.r, L.b, 2);
    norms(E, L, L.r);
    ctl(E, 0, CTL_INIT0);
    if (v.async_smooth > 0) mg_async0(E);
    else mg(E, 0);
    // final true residual
    spmm64(E, L, L.x, L.t, L.b, 2);
    norms(E, L, L.t);
    std::vector<double> rn2(R);
    MCK(cudaMemcpyAsync(rn2.data(), E->sums, R * sizeof(double), cudaMemcpyDeviceToHost, E->s));
    std::vector<MState> hs(v.nlev - 1);
    for (int l = 0; l < v.nlev - 1; ++l)
      MCK(cudaMemcpyAsync(&hs[l], E->lv[l].st, sizeof(MState), cudaMemcpyDeviceToHost, E->s));
    MCK(cudaMemcpyAsync(x, L.x, NR * sizeof(double), cudaMemcpyDefault, E->s));
    int tc_err = 0;
    MCK(cudaMemcpyAsync(&tc_err, E->tc_err, sizeof(int), cudaMemcpyDeviceToHost, E->s));
    MCK(cudaStreamSynchronize(E->s));
    MCK(cudaGetLastError());
    if (tc_err) {   // a bulk copy of the tensor-core sweep did not complete within its wait bound
      MCK(cudaMemsetAsync(E->tc_err, 0, sizeof(int), E->s));
      if (err) *err = "tensor-core sweep: a bulk copy did not complete in time; the result is invalid";
      return KCMG_CUDA_ERROR;
    }
    double worst = 0.0, res0max = 0.0;
    bool all_ok = true, finite = true;
    for (int r = 0; r < R; ++r) {
      const double rn = sqrt(rn2[r]), r0 = hs[0].rnorm0[r];
      if (!std::isfinite(rn)) finite = false;
      const double rel = r0 > 0 ? rn / r0 : 0.0;
      worst = std::max(worst, rel);
      res0max = std::max(res0max, r0);
      if (!(rn <= fmax(rtol * r0, atol))) all_ok = false;
    }
    if (info) {
      info->iters = hs[0].iters_total;
      for (int l = 0; l < KCMG_MAX_LEVELS; ++l) info->level_iters[l] = (l < v.nlev - 1) ? hs[l].iters_total : 0;
      info->restarts = hs[0].nrestart;
      info->refinements = E->mixed ? hs[0].nrestart + 1 : 0;
      info->res0 = res0max;
      info->rel_res = worst;
      info->kernel_launches = E->launches;
      // history: active columns at every level-0 loop test (type 5)
      int m = 0;
      if (info->hist && info->hist_type && info->hist_cap > 0) {
        m = std::min<int>(info->hist_cap, (int)E->hist_act.size());
        std::vector<double> hv(m);
        std::vector<int> ht(m, 5);
        for (int i = 0; i < m; ++i) hv[i] = E->hist_act[i];
        MCK(cudaMemcpy(info->hist, hv.data(), m * sizeof(double), cudaMemcpyDefault));
        MCK(cudaMemcpy(info->hist_type, ht.data(), m * sizeof(int), cudaMemcpyDefault));
      }
      info->hist_len = m;
    }
    if (hs[0].status != KCMG_OK) return (kcmg_status)hs[0].status;
    if (!finite) return KCMG_NONFINITE;
    return all_ok ? KCMG_OK : KCMG_NOT_CONVERGED;
  } catch (Fail2& f) {
    return f.st;
  }
}

int mrhs_tuning(const MrhsEngine* E, double* out, int nout) {
  if (!E) return 0;
  const double vals[9] = {E->tune[0], E->tune[1], E->tune[2], E->tune[3], E->tune[4],
                          (double)E->lv[0].lcap, (double)E->R, E->x3 ? 1.0 : 0.0, E->tune[8]};
  const int n = std::min(nout, 9);
  for (int i = 0; i < n; ++i) out[i] = vals[i];
  return n;
}

void mrhs_destroy(MrhsEngine* E) {
  if (!E) return;
  if (E->s) cudaStreamSynchronize(E->s);
  for (void* p : E->allocs) cudaFree(p);
  if (E->hst) cudaFreeHost(E->hst);
  delete E;
}

}  // namespace kcmg
