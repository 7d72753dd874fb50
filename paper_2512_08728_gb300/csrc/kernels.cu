// Device kernels of the K-cycle orthonormalization multigrid solve (sm_103a).
//
// Operator application, block-Jacobi sweeps, transfers, the coarsest solve, the Gram /
// residual-minimisation kernels of Alg. 1, the device-side loop control of Alg. 2 and
// the setup kernels (Galerkin product, block inverses, dense coarsest inverse).
#include "kcmg_internal.h"
#include "reduce.cuh"

#include <cmath>

namespace kcmg {

// ------------------------------------------------------------------ small helpers
template <typename T> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float2; };

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename TI> struct InvPair;
template <> struct InvPair<double> {
  using type = double2;
  static __device__ __forceinline__ double2 load(const double* p, size_t i) {
    return __ldg(reinterpret_cast<const double2*>(p) + i);
  }
};
template <> struct InvPair<float> {
  using type = float2;
  static __device__ __forceinline__ float2 load(const float* p, size_t i) {
    return __ldg(reinterpret_cast<const float2*>(p) + i);
  }
};
template <> struct InvPair<__nv_bfloat16> {
  using type = float2;
  static __device__ __forceinline__ float2 load(const __nv_bfloat16* p, size_t i) {
    __nv_bfloat162 v = reinterpret_cast<const __nv_bfloat162*>(p)[i];
    return __bfloat1622float2(v);
  }
};

// Sum over the block with a fixed shuffle/shared-memory tree (deterministic).
// Result valid in thread 0.  sh: >= 32 doubles of shared memory.
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
  __syncthreads();
  if (ln == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    r = (ln < nw) ? sh[ln] : 0.0;
#pragma unroll
    for (int o = 16; o; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  }
  return r;
}

// True in every thread of the block that finished last (all partials visible).
__device__ __forceinline__ bool last_block(unsigned int* ticket) {
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0;
}

// Final reduction of few columns: out[c] = sum_b partial[b*ncol + c] (fixed order).
__device__ void reduce_few(const double* partial, int nblk, int ncol, double* out, double* sh) {
  for (int c = 0; c < ncol; ++c) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += __ldcg(partial + (size_t)b * ncol + c);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) out[c] = s;
  }
  __syncthreads();
}

__device__ __forceinline__ void set_cond(const EpiArgs& e, int c) {
  e.st->cond = c;
  if (e.use_handle) cudaGraphSetConditional(e.handle, c ? 1u : 0u);
}

// Loop condition of Alg. 2 on a level.  The guard (loop bodies executed in this solve,
// counted outside the reductions) bounds every while loop independently of the rest.
__device__ __forceinline__ int more_cycles(const LevelState* st) {
  return (st->rnorm > st->eps) && (st->it < st->maxit) && (st->status == KCMG_OK) &&
         (st->guard < st->guard_cap);
}

__device__ __forceinline__ void record(const EpiArgs& e, int type) {
  LevelState* st = e.st;
  if (st->level == 0 && e.hist && st->hist_len < st->hist_cap) {
    e.hist[st->hist_len] = st->rnorm;
    e.hist_type_buf[st->hist_len] = type;
    st->hist_len++;
  }
}

// Epilogues run by thread 0 of the last block with the reduced sums.
__device__ void epilogue(const EpiArgs& e, const double* sums) {
  LevelState* st = e.st;
  switch (e.kind) {
    case EPI_MG_BEGIN: {
      st->rnorm0 = st->rnorm = sqrt(sums[0]);
      st->eps = fmax(st->rtol * st->rnorm0, st->atol);
      st->l = 0; st->it = 0; st->flags = 0; st->breakdowns = 0; st->restart_req = 0;
      if (!isfinite(st->rnorm)) st->status = KCMG_NONFINITE;
      record(e, 0);
      set_cond(e, more_cycles(st));
    } break;
    case EPI_GRAM1: {
      const int l = st->l;
      double hh = 0.0;
      for (int i = 0; i < l; ++i) { e.h[i] = sums[i]; hh += sums[i] * sums[i]; }
      const double naz2 = sums[l];
      st->naz2 = naz2;
      int f = 0;
      // Pythagoras estimate of ||w - W h||^2; reorthogonalise when it fell below a
      // quarter of ||w||^2 (a second Gram-Schmidt pass, "twice is enough")
      if (l > 0 && naz2 - hh < 0.25 * naz2) f |= F_REORTH;
      if (!isfinite(naz2) || !(naz2 > 0.0)) f |= F_DISCARD;
      st->flags = f;
    } break;
    case EPI_GRAM2: {
      for (int i = 0; i < st->l; ++i) e.h2[i] = sums[i];
    } break;
    case EPI_UPDATE: {
      const double nw = sqrt(sums[0]), naz = sqrt(st->naz2);
      if ((st->flags & F_DISCARD) || !isfinite(nw) || !(nw > st->brk * naz)) {
        st->flags |= F_DISCARD;
        if (!isfinite(nw) && st->level == 0) st->status = KCMG_NONFINITE;
      } else {
        st->gamma = 1.0 / nw;
        st->alpha = st->gamma * sums[1];   // alpha = (gamma w_hat) . r
      }
    } break;
    case EPI_FINISH: {
      if (!(st->flags & F_DISCARD)) {
        st->l++;
        st->breakdowns = 0;
      } else if (st->level == 0) {
        if (++st->breakdowns >= 2 && st->status == KCMG_OK) st->status = KCMG_BREAKDOWN;
      }
      st->rnorm = sqrt(sums[0]);
      if (!isfinite(st->rnorm) && st->status == KCMG_OK) st->status = KCMG_NONFINITE;
      record(e, e.hist_type);
      if (e.end_iter) {
        st->it++;
        st->iters_total++;
        const int cap = (st->lmax > 0 && st->lmax < st->lcap) ? st->lmax : st->lcap;
        if (st->level == 0 && !(st->rnorm > st->eps) && st->l > 0) st->restart_req = 1;
        if (st->l + st->per_cycle > cap) st->restart_req = 1;
      }
    } break;
    case EPI_RESTART: {
      st->rnorm = sqrt(sums[0]);
      st->l = 0;
      st->restart_req = 0;
      st->nrestart++;
      if (!isfinite(st->rnorm) && st->status == KCMG_OK) st->status = KCMG_NONFINITE;
      record(e, 4);
      set_cond(e, more_cycles(st));
    } break;
    case EPI_NORM: {
      if (e.out) *e.out = sqrt(sums[0]);
    } break;
    default: break;
  }
}

// Write this block's partial sums, and if last, reduce and run the epilogue.
template <int NC>
__device__ __forceinline__ void finish_reduction(double (&v)[NC], double* partial, const EpiArgs& e,
                                                 double* sh) {
  bsum_n<NC>(v, sh);
  if (threadIdx.x == 0)
#pragma unroll
    for (int c = 0; c < NC; ++c) partial[(size_t)blockIdx.x * NC + c] = v[c];
  if (last_block(&e.st->ticket)) {
    __shared__ double sums[NC];
    reduce_few(partial, gridDim.x, NC, sums, sh);
    if (threadIdx.x == 0) {
      epilogue(e, sums);
      e.st->ticket = 0u;
    }
  }
}

// ------------------------------------------------------------------ operator kernels
// y = A x (or y = b - A x), one thread per DOF row, optional ||y||^2 with an epilogue.
// conditional: run only if the level requested a restart; otherwise thread 0 of block 0
// re-evaluates the loop condition and every block returns.
// Error-free transformations for the compensated residual (Knuth's two-sum; the product
// error from a fused multiply-add).
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  s = a + b;
  const double bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// r = b - A x with the products and sums of each row carried in double-double and rounded
// once: the correctly rounded residual of the FP64 iterate, so that convergence tests near
// the attainable accuracy are not decided by summation noise.  ||r||^2 with an epilogue.
template <int NP, int S>
__device__ __forceinline__ double residual_dd_row(const double* __restrict__ A, const int* __restrict__ nbr,
                                                  int G, int row, const double* __restrict__ x,
                                                  double bv) {
  constexpr int JP = (NP + 1) / 2;
  constexpr int NF = S - 1;
  const int g = row >> 5, lane = row & 31, K = row / NP;
  double hi = 0.0, lo = 0.0;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int J = (s == 0) ? K : __ldg(nbr + (size_t)K * NF + s - 1);
    if (J < 0) continue;
    const double2* Ap = reinterpret_cast<const double2*>(A) + ((size_t)(s * G + g) * JP) * 32 + lane;
    const double* xp = x + (size_t)J * NP;
#pragma unroll
    for (int jp = 0; jp < JP; ++jp) {
      const double2 a = __ldg(Ap + jp * 32);
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (2 * jp + q >= NP) continue;
        const double av = q ? a.y : a.x, xv = __ldg(xp + 2 * jp + q);
        const double p = av * xv, pe = fma(av, xv, -p);
        double sh, se;
        two_sum(hi, p, sh, se);
        hi = sh;
        lo += se + pe;
      }
    }
  }
  double t, te;
  two_sum(bv, -hi, t, te);
  return t + (te - lo);
}

template <int NP, int S>
__global__ void __launch_bounds__(320)
k_residual_dd(const double* __restrict__ A, const int* __restrict__ nbr, int N, int G,
              const double* __restrict__ x, double* __restrict__ r, const double* __restrict__ b,
              double* partial, EpiArgs e, int conditional) {
  if (conditional) {   // end of a loop body: count it, then restart or set the condition
    if (!e.st->restart_req) {
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        e.st->guard++;
        set_cond(e, more_cycles(e.st));
      }
      return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&e.st->guard, 1);
  }
  __shared__ double sh[32 * 8];   // bsum_n<NC> needs 32 * NC
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  double out = 0.0;
  if (row < N) {
    out = residual_dd_row<NP, S>(A, nbr, G, row, x, b[row]);
    r[row] = out;
  }
  double v[1] = {out * out};
  finish_reduction<1>(v, partial, e, sh);
}

template <typename T, int NP, int S, bool RESID, bool NORM>
__global__ void __launch_bounds__(320)
k_spmv(const T* __restrict__ A, const int* __restrict__ nbr, int N, int G,
       const T* __restrict__ x, T* __restrict__ y, const T* __restrict__ b, double* partial,
       EpiArgs e, int conditional) {
  using V2 = typename Vec2<T>::type;
  constexpr int JP = (NP + 1) / 2;
  constexpr int NF = S - 1;
  if (conditional) {
    // end of a loop body: count it, then either restart (below) or set the condition
    if (!e.st->restart_req) {
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        e.st->guard++;
        set_cond(e, more_cycles(e.st));
      }
      return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&e.st->guard, 1);
  }
  __shared__ double sh[32 * 8];   // bsum_n<NC> needs 32 * NC
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  const int g = row >> 5, lane = row & 31;
  T acc = T(0);
  if (row < N) {
    const int K = row / NP;
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const int J = (s == 0) ? K : __ldg(nbr + (size_t)K * NF + s - 1);
      if (J < 0) continue;
      const V2* Ap = reinterpret_cast<const V2*>(A) + ((size_t)(s * G + g) * JP) * 32 + lane;
      const T* xp = x + (size_t)J * NP;
#pragma unroll
      for (int jp = 0; jp < JP; ++jp) {
        const V2 a = __ldg(Ap + jp * 32);
        acc = fma(a.x, __ldg(xp + 2 * jp), acc);
        if (2 * jp + 1 < NP) acc = fma(a.y, __ldg(xp + 2 * jp + 1), acc);
      }
    }
    const T out = RESID ? (b[row] - acc) : acc;
    y[row] = out;
    acc = out;
  }
  if (NORM) {
    double v[1] = {row < N ? (double)acc * (double)acc : 0.0};
    finish_reduction<1>(v, partial, e, sh);
  }
}

// One damped block-Jacobi sweep (Alg. BJ): t = r - A_off z_old (skipped on the first
// sweep from z = 0), z_new = (1 - omega) z_old + omega D^{-1} t.  A block holds whole
// cells; t is exchanged through shared memory for the inverse-block product.
template <typename T, typename TI, int NP, int S, bool FIRST>
__global__ void __launch_bounds__(320)
k_bj_sweep(const T* __restrict__ A, const TI* __restrict__ Dinv, const int* __restrict__ nbr,
           int N, int G, const T* __restrict__ r, const T* __restrict__ zold,
           T* __restrict__ znew, double omega) {
  using V2 = typename Vec2<T>::type;
  constexpr int JP = (NP + 1) / 2;
  constexpr int NF = S - 1;
  extern __shared__ unsigned char smem_raw[];
  T* ts = reinterpret_cast<T*>(smem_raw);
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  const int g = row >> 5, lane = row & 31;
  T tv = T(0);
  if (row < N) {
    tv = r[row];
    if (!FIRST) {
      const int K = row / NP;
      T acc = T(0);
#pragma unroll
      for (int s = 1; s < S; ++s) {
        const int J = __ldg(nbr + (size_t)K * NF + s - 1);
        if (J < 0) continue;
        const V2* Ap = reinterpret_cast<const V2*>(A) + ((size_t)(s * G + g) * JP) * 32 + lane;
        const T* zp = zold + (size_t)J * NP;
#pragma unroll
        for (int jp = 0; jp < JP; ++jp) {
          const V2 a = __ldg(Ap + jp * 32);
          acc = fma(a.x, zp[2 * jp], acc);
          if (2 * jp + 1 < NP) acc = fma(a.y, zp[2 * jp + 1], acc);
        }
      }
      tv -= acc;
    }
  }
  ts[threadIdx.x] = tv;
  __syncthreads();
  if (row < N) {
    const int base = (row / NP) * NP - blockIdx.x * blockDim.x;
    T dz = T(0);
#pragma unroll
    for (int jp = 0; jp < JP; ++jp) {
      const auto d = InvPair<TI>::load(Dinv, ((size_t)g * JP + jp) * 32 + lane);
      dz = fma((T)d.x, ts[base + 2 * jp], dz);
      if (2 * jp + 1 < NP) dz = fma((T)d.y, ts[base + 2 * jp + 1], dz);
    }
    const T om = (T)omega;
    znew[row] = FIRST ? om * dz : fma(T(1) - om, zold[row], om * dz);
  }
}

// ------------------------------------------------------------------ transfers
struct Dims { int n[3]; };

// r_c[J][i] = sum_k sum_a P_k[a][i] r_f[child_k(J)][a]  (R = P^T).  With b/r/x given this
// also starts the next level's MG call: b = r = r_c, x = 0, ||r_c||^2 -> MG_BEGIN.
template <typename T, typename TIN, int NP, int DIM>
__global__ void __launch_bounds__(256)
k_restrict(Dims nf, Dims nc, const T* __restrict__ P, const TIN* __restrict__ rf, T* bout,
           T* rout, T* xout, int Nc, double* partial, EpiArgs e) {
  constexpr int NCH = 1 << DIM;
  __shared__ T Ps[NCH * NP * NP];
  __shared__ double sh[32 * 8];   // bsum_n<NC> needs 32 * NC
  for (int i = threadIdx.x; i < NCH * NP * NP; i += blockDim.x) Ps[i] = P[i];
  __syncthreads();
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  T s = T(0);
  if (row < Nc) {
    const int J = row / NP, i = row - J * NP;
    const int jx = J % nc.n[0], jy = (J / nc.n[0]) % nc.n[1], jz = DIM == 3 ? J / (nc.n[0] * nc.n[1]) : 0;
#pragma unroll
    for (int k = 0; k < NCH; ++k) {
      const int fx = 2 * jx + (k & 1), fy = 2 * jy + ((k >> 1) & 1), fz = DIM == 3 ? 2 * jz + ((k >> 2) & 1) : 0;
      const int K = fx + nf.n[0] * (fy + nf.n[1] * fz);
      const TIN* rp = rf + (size_t)K * NP;
#pragma unroll
      for (int a = 0; a < NP; ++a) s = fma(Ps[(k * NP + a) * NP + i], (T)rp[a], s);
    }
    bout[row] = s;
    if (rout) { rout[row] = s; xout[row] = T(0); }
  }
  if (e.kind != EPI_NONE) {
    double v[1] = {row < Nc ? (double)s * (double)s : 0.0};
    finish_reduction<1>(v, partial, e, sh);
  }
}

// z_f[child_k(J)][a] = sum_i P_k[a][i] z_c[J][i]
template <typename T, typename TOUT, int NP, int DIM>
__global__ void __launch_bounds__(256)
k_prolong(Dims nf, Dims nc, const T* __restrict__ P, const T* __restrict__ zc, TOUT* __restrict__ zf,
          int Nf) {
  constexpr int NCH = 1 << DIM;
  __shared__ T Ps[NCH * NP * NP];
  for (int i = threadIdx.x; i < NCH * NP * NP; i += blockDim.x) Ps[i] = P[i];
  __syncthreads();
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= Nf) return;
  const int K = row / NP, a = row - K * NP;
  const int ix = K % nf.n[0], iy = (K / nf.n[0]) % nf.n[1], iz = DIM == 3 ? K / (nf.n[0] * nf.n[1]) : 0;
  const int k = (ix & 1) | ((iy & 1) << 1) | (DIM == 3 ? ((iz & 1) << 2) : 0);
  const int J = (ix >> 1) + nc.n[0] * ((iy >> 1) + nc.n[1] * (iz >> 1));
  const T* zp = zc + (size_t)J * NP;
  T s = T(0);
#pragma unroll
  for (int i = 0; i < NP; ++i) s = fma(Ps[(k * NP + a) * NP + i], zp[i], s);
  zf[row] = (TOUT)s;
}

// x = A_c^{-1} b with the dense FP64 inverse; one warp per row.
template <typename T>
__global__ void k_coarse_gemv(const double* __restrict__ Ainv, int n, const T* __restrict__ b,
                              T* __restrict__ x) {
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), ln = threadIdx.x & 31;
  if (row >= n) return;
  double s = 0.0;
  for (int j = ln; j < n; j += 32) s = fma(__ldg(Ainv + (size_t)row * n + j), (double)b[j], s);
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (ln == 0) x[row] = (T)s;
}

// ------------------------------------------------------------------ Gram / RM (Alg. 1)
// partial[k][c] = sum over element chunk k of W_c . w for c < l, and ||w||^2 at c = l.
// Work items are (group of kDotCols columns) x (element chunk); the fixed grid takes them
// round-robin with K = grid / groups chunks per group, so a block reduces its sums once
// per item and the reduction order depends only on N, l and the grid.  With PAIR (N even)
// a thread takes two consecutive elements per step with one 16-byte (FP64) or 8-byte
// (FP32) load per column.  The last partial column group reads a valid column in place of
// the missing ones and drops those sums, so every step issues the same FMAs (no
// predicated arithmetic).  ||w||^2 rides with group 0 as a separate accumulator.
constexpr int kDotCols = 8;

template <typename T> struct Pair;
template <> struct Pair<double> { using type = double2; };
template <> struct Pair<float> { using type = float2; };

template <typename T, bool PAIR, bool NORM>
__device__ __forceinline__ void dots_item(const T* __restrict__ W, int N, const T* __restrict__ w, int l, int c0,
                                          int u0, int u1, T (&acc)[kDotCols], T& ww) {
  using T2 = typename Pair<T>::type;
  const T* Wc[kDotCols];
#pragma unroll
  for (int c = 0; c < kDotCols; ++c) Wc[c] = W + (size_t)min(c0 + c, l - 1) * N;
  for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) {
    if (PAIR) {
      const T2 wv = __ldg(reinterpret_cast<const T2*>(w) + u);
#pragma unroll
      for (int c = 0; c < kDotCols; ++c) {
        const T2 a = __ldg(reinterpret_cast<const T2*>(Wc[c]) + u);
        acc[c] = fma(a.x, wv.x, acc[c]);
        acc[c] = fma(a.y, wv.y, acc[c]);
      }
      if (NORM) {
        ww = fma(wv.x, wv.x, ww);
        ww = fma(wv.y, wv.y, ww);
      }
    } else {
      const T wv = __ldg(w + u);
#pragma unroll
      for (int c = 0; c < kDotCols; ++c) acc[c] = fma(__ldg(Wc[c] + u), wv, acc[c]);
      if (NORM) ww = fma(wv, wv, ww);
    }
  }
}

template <typename T, bool PAIR>
__global__ void __launch_bounds__(kVecThreads)
k_gram_dots(const T* __restrict__ W, int N, const T* __restrict__ w, double* partial,
            EpiArgs e, int conditional) {
  LevelState* st = e.st;
  if (conditional && !(st->flags & F_REORTH)) return;
  __shared__ double sh[32 * 8];   // bsum_n<NC> needs 32 * NC
  const int l = st->l;
  const int ncol = l + 1;
  const int groups = l > 0 ? (l + kDotCols - 1) / kDotCols : 1;   // l = 0: the norm only
  const int K = max(1, (int)gridDim.x / groups);
  const int units = PAIR ? N / 2 : N;
  const int chunk = (units + K - 1) / K;
  for (int item = blockIdx.x; item < groups * K; item += gridDim.x) {
    const int g = item / K, k = item - g * K;
    const int c0 = g * kDotCols;
    const int u0 = min(units, k * chunk), u1 = min(units, u0 + chunk);
    T acct[kDotCols];
#pragma unroll
    for (int c = 0; c < kDotCols; ++c) acct[c] = T(0);
    T ww = T(0);
    if (l == 0) {
      for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) {
        if (PAIR) {
          const typename Pair<T>::type wv = __ldg(reinterpret_cast<const typename Pair<T>::type*>(w) + u);
          ww = fma(wv.x, wv.x, ww);
          ww = fma(wv.y, wv.y, ww);
        } else {
          const T wv = __ldg(w + u);
          ww = fma(wv, wv, ww);
        }
      }
    } else if (g == 0) {
      dots_item<T, PAIR, true>(W, N, w, l, c0, u0, u1, acct, ww);
    } else {
      dots_item<T, PAIR, false>(W, N, w, l, c0, u0, u1, acct, ww);
    }
    // the block's sums in FP64 (FP32 vectors: FP32 products and per-thread sums)
    double acc[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = (double)acct[c];
    bsum_n<8>(acc, sh);
    if (threadIdx.x == 0)
#pragma unroll
      for (int c = 0; c < kDotCols; ++c)
        if (c0 + c < l) partial[(size_t)k * ncol + c0 + c] = acc[c];
    if (g == 0) {
      double v[1] = {(double)ww};
      bsum_n<1>(v, sh);
      if (threadIdx.x == 0) partial[(size_t)k * ncol + l] = v[0];
    }
  }
  if (last_block(&st->ticket)) {
    // one warp per column: lanes read independent partials, then a fixed shuffle tree
    extern __shared__ double sums[];  // [ncol]
    const int wid = threadIdx.x >> 5, ln = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int c = wid; c < ncol; c += nw) {
      double s = 0.0;
      for (int b = ln; b < K; b += 32) s += __ldcg(partial + (size_t)b * ncol + c);
#pragma unroll
      for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (ln == 0) sums[c] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      epilogue(e, sums);
      st->ticket = 0u;
    }
  }
}

// w_out = w - W h (first pass of the reorthogonalisation; runs only when requested)
template <typename T>
__global__ void __launch_bounds__(kVecThreads)
k_gram_apply(const T* __restrict__ W, int N, const T* __restrict__ w, T* __restrict__ wout,
             const LevelState* st, const double* __restrict__ h) {
  if (!(st->flags & F_REORTH)) return;
  extern __shared__ double hs[];
  const int l = st->l;
  for (int i = threadIdx.x; i < l; i += blockDim.x) hs[i] = h[i];
  __syncthreads();
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
    T s = w[j];
#pragma unroll 4
    for (int i = 0; i < l; ++i) s = fma((T)(-hs[i]), __ldg(W + (size_t)i * N + j), s);
    wout[j] = s;
  }
}

// w_hat = w_src - W c_w, z_hat = z - Z c_z written to column l of W and Z; partial sums
// ||w_hat||^2 and w_hat . r.  Without reorthogonalisation w_src = w, c_w = c_z = h; with it
// w_src = w' = w - W h, c_w = h2, c_z = h + h2.  With PAIR (N even) a thread updates two
// consecutive elements with one 16-byte (FP64) / 8-byte (FP32) load per column of W and Z.
template <typename T, bool PAIR>
__global__ void __launch_bounds__(kVecThreads)
k_gram_update(T* W, T* Z, int N, const T* __restrict__ w, const T* __restrict__ wre,
              const T* __restrict__ z, const T* __restrict__ r, double* partial, EpiArgs e) {
  using T2 = typename Pair<T>::type;
  LevelState* st = e.st;
  extern __shared__ double cs[];  // [2][l]
  __shared__ double sh[32 * 8];   // bsum_n<NC> needs 32 * NC
  const int l = st->l;
  const bool re = (st->flags & F_REORTH) != 0;
  for (int i = threadIdx.x; i < l; i += blockDim.x) {
    cs[i] = re ? e.h2[i] : e.h[i];
    cs[l + i] = re ? e.h[i] + e.h2[i] : e.h[i];
  }
  __syncthreads();
  const T* ws = re ? wre : w;
  T* Wl = W + (size_t)l * N;
  T* Zl = Z + (size_t)l * N;
  T nw2 = T(0), wr = T(0);   // per-thread sums in T, reduced in FP64
  if (PAIR) {
    const int units = N / 2;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < units; u += gridDim.x * blockDim.x) {
      T2 a = reinterpret_cast<const T2*>(ws)[u], c = reinterpret_cast<const T2*>(z)[u];
#pragma unroll 4
      for (int i = 0; i < l; ++i) {
        const T2 wi = __ldg(reinterpret_cast<const T2*>(W + (size_t)i * N) + u);
        const T2 zi = __ldg(reinterpret_cast<const T2*>(Z + (size_t)i * N) + u);
        const T cw = (T)(-cs[i]), cz = (T)(-cs[l + i]);
        a.x = fma(cw, wi.x, a.x);
        a.y = fma(cw, wi.y, a.y);
        c.x = fma(cz, zi.x, c.x);
        c.y = fma(cz, zi.y, c.y);
      }
      reinterpret_cast<T2*>(Wl)[u] = a;
      reinterpret_cast<T2*>(Zl)[u] = c;
      const T2 rv = reinterpret_cast<const T2*>(r)[u];
      nw2 = fma(a.x, a.x, nw2);
      nw2 = fma(a.y, a.y, nw2);
      wr = fma(a.x, rv.x, wr);
      wr = fma(a.y, rv.y, wr);
    }
  } else {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
      T a = ws[j], c = z[j];
#pragma unroll 4
      for (int i = 0; i < l; ++i) {
        a = fma((T)(-cs[i]), __ldg(W + (size_t)i * N + j), a);
        c = fma((T)(-cs[l + i]), __ldg(Z + (size_t)i * N + j), c);
      }
      Wl[j] = a;
      Zl[j] = c;
      nw2 = fma(a, a, nw2);
      wr = fma(a, r[j], wr);
    }
  }
  double v[2] = {(double)nw2, (double)wr};
  finish_reduction<2>(v, partial, e, sh);
}

// Normalise the new column (gamma) and update x += alpha z_{l+1}, r -= alpha w_{l+1};
// ||r||^2 -> EPI_FINISH.  A discarded correction leaves W, Z, x, r unchanged.
template <typename T>
__global__ void __launch_bounds__(kVecThreads)
k_rm_finish(T* W, T* Z, int N, T* x, T* r, double* partial, EpiArgs e) {
  LevelState* st = e.st;
  __shared__ double sh[32 * 8];   // bsum_n<NC> needs 32 * NC
  const bool keep = !(st->flags & F_DISCARD);
  const int l = st->l;
  const T gam = (T)st->gamma, al = (T)st->alpha;
  T* Wl = W + (size_t)l * N;
  T* Zl = Z + (size_t)l * N;
  double r2 = 0.0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
    T rv = r[j];
    if (keep) {
      const T wv = Wl[j] * gam, zv = Zl[j] * gam;
      Wl[j] = wv;
      Zl[j] = zv;
      x[j] = fma(al, zv, x[j]);
      rv = fma(-al, wv, rv);
      r[j] = rv;
    }
    r2 = fma((double)rv, (double)rv, r2);
  }
  double v[1] = {r2};
  finish_reduction<1>(v, partial, e, sh);
}

template <typename T>
__global__ void __launch_bounds__(kVecThreads)
k_norm(const T* __restrict__ v, int N, double* partial, EpiArgs e) {
  __shared__ double sh[32 * 8];   // bsum_n<NC> needs 32 * NC
  double s = 0.0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
    const double a = (double)v[j];
    s = fma(a, a, s);
  }
  double vv[1] = {s};
  finish_reduction<1>(vv, partial, e, sh);
}

__global__ void k_control(EpiArgs e) { set_cond(e, more_cycles(e.st)); }

template <typename Ts, typename Td>
__global__ void k_convert(const Ts* __restrict__ a, Td* __restrict__ b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = (Td)a[i];
}
__global__ void k_scale_to_float(const double* __restrict__ a, float* __restrict__ b, double s, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = (float)(s * a[i]);
}
__global__ void k_axpy_scaled_to_double(const float* __restrict__ e, double* __restrict__ x, double s,
                                        size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    x[i] = fma(s, (double)e[i], x[i]);
}
template <typename T>
__global__ void k_axpy_to_double(const T* __restrict__ e, double* __restrict__ x, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    x[i] += (double)e[i];
}

// ------------------------------------------------------------------ setup kernels
__global__ void k_build_nbr(int dim, Dims n, int* nbr) {
  const int C = n.n[0] * n.n[1] * (dim == 3 ? n.n[2] : 1);
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= C) return;
  const int c[3] = {K % n.n[0], (K / n.n[0]) % n.n[1], dim == 3 ? K / (n.n[0] * n.n[1]) : 0};
  const int stride[3] = {1, n.n[0], n.n[0] * n.n[1]};
  for (int j = 0; j < dim; ++j) {
    nbr[K * 2 * dim + 2 * j] = c[j] > 0 ? K - stride[j] : -1;
    nbr[K * 2 * dim + 2 * j + 1] = c[j] < n.n[j] - 1 ? K + stride[j] : -1;
  }
}

// Galerkin product A_c = P^T A P, one block per (coarse cell, coarse slot), np*np threads.
// Contributions: every child K of J and fine slot s whose neighbour K2 lies in the coarse
// cell addressed by the coarse slot: C += P_k^T A[s][K] P_k2.
template <int NP, int DIM>
__global__ void k_galerkin(const double* __restrict__ Af, const int* __restrict__ nbrf, Dims nf,
                           Dims nc, const double* __restrict__ P, double* __restrict__ Ac) {
  constexpr int S = 2 * DIM + 1, NCH = 1 << DIM;
  __shared__ double Ps[NCH * NP * NP];
  __shared__ double Ts[NP * NP];
  const int J = blockIdx.x, cs = blockIdx.y;
  const int Cc = nc.n[0] * nc.n[1] * (DIM == 3 ? nc.n[2] : 1);
  const int Cf = nf.n[0] * nf.n[1] * (DIM == 3 ? nf.n[2] : 1);
  for (int i = threadIdx.x; i < NCH * NP * NP; i += blockDim.x) Ps[i] = P[i];
  const int ti = threadIdx.x / NP, tj = threadIdx.x % NP;
  const bool act = threadIdx.x < NP * NP;
  const int jx = J % nc.n[0], jy = (J / nc.n[0]) % nc.n[1], jz = DIM == 3 ? J / (nc.n[0] * nc.n[1]) : 0;
  double acc = 0.0;
  __syncthreads();
  for (int k = 0; k < NCH; ++k) {
    const int fx = 2 * jx + (k & 1), fy = 2 * jy + ((k >> 1) & 1), fz = DIM == 3 ? 2 * jz + ((k >> 2) & 1) : 0;
    const int K = fx + nf.n[0] * (fy + nf.n[1] * fz);
    for (int s = 0; s < S; ++s) {
      const int K2 = (s == 0) ? K : nbrf[K * (S - 1) + s - 1];
      if (K2 < 0) continue;
      const int x2 = K2 % nf.n[0], y2 = (K2 / nf.n[0]) % nf.n[1], z2 = DIM == 3 ? K2 / (nf.n[0] * nf.n[1]) : 0;
      const int J2 = (x2 >> 1) + nc.n[0] * ((y2 >> 1) + nc.n[1] * (z2 >> 1));
      const int target = (J2 == J) ? 0 : s;  // crossing a coarse face keeps the direction
      if (target != cs) continue;
      const int k2 = (x2 & 1) | ((y2 & 1) << 1) | (DIM == 3 ? ((z2 & 1) << 2) : 0);
      const double* Ab = Af + ((size_t)s * Cf + K) * NP * NP;
      // T = A_b P_k2 : T[a][j] = sum_m A[a][m] P_k2[m][j]
      if (act) {
        double t = 0.0;
        for (int m = 0; m < NP; ++m) t = fma(Ab[ti * NP + m], Ps[(k2 * NP + m) * NP + tj], t);
        Ts[ti * NP + tj] = t;
      }
      __syncthreads();
      if (act)
        for (int a = 0; a < NP; ++a) acc = fma(Ps[(k * NP + a) * NP + ti], Ts[a * NP + tj], acc);
      __syncthreads();
    }
  }
  if (act) Ac[((size_t)cs * Cc + J) * NP * NP + threadIdx.x] = acc;
}

// Gauss-Jordan inverse with partial pivoting of every diagonal block; one warp per cell,
// lane j holds columns j and j + 32 of the augmented matrix [A | I].
template <int NP>
__global__ void k_block_inverse(const double* __restrict__ diag, int ncell, double* __restrict__ inv,
                                int* fail) {
  const int K = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), ln = threadIdx.x & 31;
  if (K >= ncell) return;
  double c0[NP], c1[NP];  // column ln and column ln+32 of [A | I]
  const double* A = diag + (size_t)K * NP * NP;
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    const int j0 = ln, j1 = ln + 32;
    c0[i] = j0 < NP ? A[i * NP + j0] : (j0 - NP == i ? 1.0 : 0.0);
    c1[i] = j1 < NP ? A[i * NP + j1] : (j1 - NP == i ? 1.0 : 0.0);
  }
  bool bad = false;
#pragma unroll
  for (int c = 0; c < NP; ++c) {
    // pivot search in column c (held by lane c in c0)
    int p = c;
    double best = -1.0;
#pragma unroll
    for (int i = 0; i < NP; ++i)
      if (i >= c && fabs(c0[i]) > best) { best = fabs(c0[i]); p = i; }
    p = __shfl_sync(0xffffffffu, p, c);
    best = __shfl_sync(0xffffffffu, best, c);
    if (!(best > 0.0)) bad = true;
    // swap rows c and p
    double a0 = 0, a1 = 0, b0 = 0, b1 = 0;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      if (i == c) { a0 = c0[i]; a1 = c1[i]; }
      if (i == p) { b0 = c0[i]; b1 = c1[i]; }
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      if (i == c) { c0[i] = b0; c1[i] = b1; }
      else if (i == p) { c0[i] = a0; c1[i] = a1; }
    }
    double d = 0.0;
#pragma unroll
    for (int i = 0; i < NP; ++i) if (i == c) d = c0[i];
    d = __shfl_sync(0xffffffffu, d, c);
    const double inv_d = bad ? 0.0 : 1.0 / d;
    double pr0 = 0, pr1 = 0;
#pragma unroll
    for (int i = 0; i < NP; ++i)
      if (i == c) { c0[i] *= inv_d; c1[i] *= inv_d; pr0 = c0[i]; pr1 = c1[i]; }
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      const double f = __shfl_sync(0xffffffffu, c0[i], c);
      if (i != c) { c0[i] = fma(-f, pr0, c0[i]); c1[i] = fma(-f, pr1, c1[i]); }
    }
  }
  if (bad && ln == 0) atomicExch(fail, 1);
  double* out = inv + (size_t)K * NP * NP;
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    if (ln >= NP && ln < 2 * NP) out[i * NP + ln - NP] = c0[i];
    if (ln + 32 >= NP && ln + 32 < 2 * NP) out[i * NP + ln + 32 - NP] = c1[i];
  }
}

// dense augmented matrix M = [A_c | I] (n x 2n) of the coarsest operator
__global__ void k_assemble_dense(int np, int dim, const double* __restrict__ blk,
                                 const int* __restrict__ nbr, int ncell, double* M) {
  const int n = ncell * np, S = 2 * dim + 1;
  const size_t tot = (size_t)n * 2 * n;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < tot; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / (2 * n)), j = (int)(idx % (2 * n));
    double v = 0.0;
    if (j >= n) {
      v = (j - n == i) ? 1.0 : 0.0;
    } else {
      const int K = i / np, a = i % np, J = j / np, m = j % np;
      for (int s = 0; s < S; ++s) {
        const int K2 = s == 0 ? K : nbr[K * (S - 1) + s - 1];
        if (K2 == J) v += blk[((size_t)s * ncell + K) * np * np + a * np + m];
      }
    }
    M[idx] = v;
  }
}

// Gauss-Jordan step c on M (n x 2n): pick the pivot, swap, scale (single block)
__global__ void k_gj_pivot(double* M, int n, int c, double* fcol, int* fail) {
  __shared__ double bv[1024];
  __shared__ int bi[1024];
  double best = -1.0;
  int p = c;
  for (int i = c + threadIdx.x; i < n; i += blockDim.x) {
    const double v = fabs(M[(size_t)i * 2 * n + c]);
    if (v > best) { best = v; p = i; }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = p;
  __syncthreads();
  for (int o = blockDim.x / 2; o; o >>= 1) {
    if (threadIdx.x < o) {
      const double v2 = bv[threadIdx.x + o];
      const int i2 = bi[threadIdx.x + o];
      if (v2 > bv[threadIdx.x] || (v2 == bv[threadIdx.x] && i2 < bi[threadIdx.x])) {
        bv[threadIdx.x] = v2;
        bi[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  p = bi[0];
  if (!(bv[0] > 0.0)) {
    if (threadIdx.x == 0) atomicExch(fail, 1);
    return;
  }
  for (int j = threadIdx.x; j < 2 * n; j += blockDim.x) {
    const double a = M[(size_t)c * 2 * n + j], b = M[(size_t)p * 2 * n + j];
    M[(size_t)c * 2 * n + j] = b;
    M[(size_t)p * 2 * n + j] = a;
  }
  __syncthreads();
  const double d = M[(size_t)c * 2 * n + c];
  __syncthreads();
  for (int j = threadIdx.x; j < 2 * n; j += blockDim.x) M[(size_t)c * 2 * n + j] /= d;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) fcol[i] = (i == c) ? 0.0 : M[(size_t)i * 2 * n + c];
}

// elimination of column c from every other row: M[i][j] -= f_i M[c][j]
__global__ void k_gj_elim(double* M, int n, int c, const double* __restrict__ fcol, const int* fail) {
  if (*fail) return;
  const size_t tot = (size_t)n * 2 * n;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < tot; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / (2 * n)), j = (int)(idx % (2 * n));
    if (i == c) continue;
    M[idx] = fma(-fcol[i], M[(size_t)c * 2 * n + j], M[idx]);
  }
}

__global__ void k_extract_inverse(const double* __restrict__ M, int n, double* Ainv) {
  const size_t tot = (size_t)n * n;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < tot; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / n), j = (int)(idx % n);
    Ainv[idx] = M[(size_t)i * 2 * n + n + j];
  }
}

// natural [nslot][C][np][np] FP64 -> row-interleaved T
template <typename T>
__global__ void k_interleave(int np, int nslot, const double* __restrict__ nat, int ncell, int G,
                             T* __restrict__ out) {
  const int JP = (np + 1) / 2;
  const size_t tot = (size_t)nslot * G * JP * 64;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < tot; idx += (size_t)gridDim.x * blockDim.x) {
    const int e = (int)(idx & 1);
    const int lane = (int)((idx >> 1) & 31);
    size_t q = idx >> 6;
    const int jp = (int)(q % JP);
    q /= JP;
    const int g = (int)(q % G);
    const int s = (int)(q / G);
    const int row = g * 32 + lane, j = 2 * jp + e;
    double v = 0.0;
    if (row < ncell * np && j < np) {
      const int K = row / np, i = row % np;
      v = nat[((size_t)s * ncell + K) * np * np + i * np + j];
    }
    out[idx] = (T)v;
  }
}

// transposed operator: out[s][K] = (in[opp(s)][nbr(K, s)])^T
__global__ void k_transpose_blocks(int np, int dim, const double* __restrict__ in,
                                   const int* __restrict__ nbr, int ncell, double* __restrict__ out) {
  const int S = 2 * dim + 1;
  const size_t tot = (size_t)S * ncell * np * np;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < tot; idx += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(idx % np), i = (int)((idx / np) % np);
    const int K = (int)((idx / ((size_t)np * np)) % ncell), s = (int)(idx / ((size_t)np * np * ncell));
    const int J = s == 0 ? K : nbr[K * (S - 1) + s - 1];
    const int opp = s == 0 ? 0 : (((s - 1) ^ 1) + 1);
    out[idx] = J < 0 ? 0.0 : in[((size_t)opp * ncell + J) * np * np + j * np + i];
  }
}

__global__ void k_count_diff(const double* __restrict__ a, const double* __restrict__ b, size_t n,
                             unsigned int* cnt) {
  unsigned int c = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    c += (a[i] != b[i]);
  if (c) atomicAdd(cnt, c);
}

// g_K = -lambda^T (dA/d log nu_K) u (SWIP operator with harmonic face coefficients)
template <int NP>
__device__ double bil(const double* M, const double* l, const double* u) {
  double s = 0.0;
  for (int i = 0; i < NP; ++i) {
    double t = 0.0;
    for (int j = 0; j < NP; ++j) t = fma(M[i * NP + j], u[j], t);
    s = fma(l[i], t, s);
  }
  return s;
}
template <int NP>
__global__ void k_grad_lognu(int dim, Dims n, const double* __restrict__ nu, const double* __restrict__ V,
                             const double* __restrict__ F, const double* __restrict__ B,
                             const double* __restrict__ lam, const double* __restrict__ u, double* g) {
  const int C = n.n[0] * n.n[1] * (dim == 3 ? n.n[2] : 1);
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= C) return;
  constexpr int BS = NP * NP;
  const int c[3] = {K % n.n[0], (K / n.n[0]) % n.n[1], dim == 3 ? K / (n.n[0] * n.n[1]) : 0};
  const int stride[3] = {1, n.n[0], n.n[0] * n.n[1]};
  const double* lK = lam + (size_t)K * NP;
  const double* uK = u + (size_t)K * NP;
  double s = bil<NP>(V, lK, uK);
  for (int k = 0; k < dim; ++k) {
    const double* Fk = F + (size_t)k * 4 * BS;
    const double* Bk = B + (size_t)k * 2 * BS;
    if (c[k] < n.n[k] - 1) {
      const int R = K + stride[k];
      const double a = nu[K], b = nu[R], dg = 2.0 * b * b / ((a + b) * (a + b));
      const double* lR = lam + (size_t)R * NP;
      const double* uR = u + (size_t)R * NP;
      s += dg * (bil<NP>(Fk, lK, uK) + bil<NP>(Fk + BS, lK, uR) + bil<NP>(Fk + 2 * BS, lR, uK) +
                 bil<NP>(Fk + 3 * BS, lR, uR));
    } else {
      s += bil<NP>(Bk + BS, lK, uK);
    }
    if (c[k] > 0) {
      const int L = K - stride[k];
      const double a = nu[K], b = nu[L], dg = 2.0 * b * b / ((a + b) * (a + b));
      const double* lL = lam + (size_t)L * NP;
      const double* uL = u + (size_t)L * NP;
      s += dg * (bil<NP>(Fk, lL, uL) + bil<NP>(Fk + BS, lL, uK) + bil<NP>(Fk + 2 * BS, lK, uL) +
                 bil<NP>(Fk + 3 * BS, lK, uK));
    } else {
      s += bil<NP>(Bk, lK, uK);
    }
  }
  g[K] = -nu[K] * s;
}

// ------------------------------------------------------------------ launchers
// total-degree DG spaces: 2-D p = 1, 2, 3 (3, 6, 10 modes); 3-D p = 1, 2, 3 (4, 10, 20)
bool np_supported(int np, int dim) {
  return dim == 2 ? (np == 3 || np == 6 || np == 10) : dim == 3 ? (np == 4 || np == 10 || np == 20) : false;
}

int block_rows_for(int np) {
  switch (np) {
    case 3: return 288;   // 3 * 96
    case 4: return 256;
    case 6: return 288;
    case 10: return 320;  // 2 * lcm(32, 10)
    case 20: return 320;
    default: return 0;
  }
}

static inline int nblocks(size_t n, int t, int cap = 4096) {
  size_t b = (n + t - 1) / t;
  if (b < 1) b = 1;
  return (int)(b > (size_t)cap ? cap : b);
}

static Dims mkdims(const int* n) { Dims d; d.n[0] = n[0]; d.n[1] = n[1]; d.n[2] = n[2]; return d; }

// dispatch over the supported (np, dim) pairs; the body sees NP, DIM and S = 2 DIM + 1
#define KCMG_ND_SWITCH(np, dim, ...)                                                      \
  switch (np * 10 + dim) {                                                                \
    case 32: { constexpr int NP = 3, DIM = 2, S = 5; (void)S; (void)DIM; __VA_ARGS__; } break;       \
    case 62: { constexpr int NP = 6, DIM = 2, S = 5; (void)S; (void)DIM; __VA_ARGS__; } break;       \
    case 102: { constexpr int NP = 10, DIM = 2, S = 5; (void)S; (void)DIM; __VA_ARGS__; } break;     \
    case 43: { constexpr int NP = 4, DIM = 3, S = 7; (void)S; (void)DIM; __VA_ARGS__; } break;       \
    case 103: { constexpr int NP = 10, DIM = 3, S = 7; (void)S; (void)DIM; __VA_ARGS__; } break;     \
    case 203: { constexpr int NP = 20, DIM = 3, S = 7; (void)S; (void)DIM; __VA_ARGS__; } break;     \
    default: break;                                                                       \
  }
#define KCMG_NP_SWITCH(np, ...)                               \
  switch (np) {                                               \
    case 3: { constexpr int NP = 3; __VA_ARGS__; } break;     \
    case 4: { constexpr int NP = 4; __VA_ARGS__; } break;     \
    case 6: { constexpr int NP = 6; __VA_ARGS__; } break;     \
    case 10: { constexpr int NP = 10; __VA_ARGS__; } break;   \
    case 20: { constexpr int NP = 20; __VA_ARGS__; } break;   \
    default: break;                                           \
  }

template <typename T>
void launch_spmv(int np, int dim, const T* A, const int* nbr, int N, int G, int rows_pad,
                 int block_rows, const T* x, T* y, const T* b, double* partial,
                 const EpiArgs& e, int conditional, cudaStream_t s) {
  const int grid = rows_pad / block_rows;
  const bool resid = b != nullptr, norm = e.kind != EPI_NONE;
  KCMG_ND_SWITCH(np, dim, {
    if (resid && norm) k_spmv<T, NP, S, true, true><<<grid, block_rows, 0, s>>>(A, nbr, N, G, x, y, b, partial, e, conditional);
    else if (resid) k_spmv<T, NP, S, true, false><<<grid, block_rows, 0, s>>>(A, nbr, N, G, x, y, b, partial, e, conditional);
    else if (norm) k_spmv<T, NP, S, false, true><<<grid, block_rows, 0, s>>>(A, nbr, N, G, x, y, b, partial, e, conditional);
    else k_spmv<T, NP, S, false, false><<<grid, block_rows, 0, s>>>(A, nbr, N, G, x, y, b, partial, e, conditional);
  });
}

void launch_residual_dd(int np, int dim, const double* A, const int* nbr, int N, int G, int rows_pad,
                        int block_rows, const double* x, double* r, const double* b, double* partial,
                        const EpiArgs& e, int conditional, cudaStream_t s) {
  const int grid = rows_pad / block_rows;
  KCMG_ND_SWITCH(np, dim, {
    k_residual_dd<NP, S><<<grid, block_rows, 0, s>>>(A, nbr, N, G, x, r, b, partial, e, conditional);
  });
}

template <typename T, typename TI>
void launch_bj_sweep(int np, int dim, const T* A, const TI* Dinv, const int* nbr, int N, int G,
                     int rows_pad, int block_rows, const T* r, const T* zold, T* znew,
                     double omega, int first, cudaStream_t s) {
  const int grid = rows_pad / block_rows;
  const size_t sm = (size_t)block_rows * sizeof(T);
  KCMG_ND_SWITCH(np, dim, {
    if (first) k_bj_sweep<T, TI, NP, S, true><<<grid, block_rows, sm, s>>>(A, Dinv, nbr, N, G, r, zold, znew, omega);
    else k_bj_sweep<T, TI, NP, S, false><<<grid, block_rows, sm, s>>>(A, Dinv, nbr, N, G, r, zold, znew, omega);
  });
}

template <typename T, typename TIN>
void launch_restrict(int np, int dim, const int* nf, const int* nc, const T* P, const TIN* rf,
                     T* b, T* r, T* x, double* partial, const EpiArgs& e, cudaStream_t s) {
  const int Nc = nc[0] * nc[1] * (dim == 3 ? nc[2] : 1) * np;
  const int grid = nblocks(Nc, 256, 1 << 30);
  KCMG_ND_SWITCH(np, dim, {
    k_restrict<T, TIN, NP, DIM><<<grid, 256, 0, s>>>(mkdims(nf), mkdims(nc), P, rf, b, r, x, Nc, partial, e);
  });
}

template <typename T, typename TOUT>
void launch_prolong(int np, int dim, const int* nf, const int* nc, const T* P, const T* zc,
                    TOUT* zf, cudaStream_t s) {
  const int Nf = nf[0] * nf[1] * (dim == 3 ? nf[2] : 1) * np;
  const int grid = nblocks(Nf, 256, 1 << 30);
  KCMG_ND_SWITCH(np, dim, {
    k_prolong<T, TOUT, NP, DIM><<<grid, 256, 0, s>>>(mkdims(nf), mkdims(nc), P, zc, zf, Nf);
  });
}

template <typename T>
void launch_coarse_gemv(const double* Ainv, int n, const T* b, T* x, cudaStream_t s) {
  const int rows_per_block = 8;
  k_coarse_gemv<T><<<(n + rows_per_block - 1) / rows_per_block, 32 * rows_per_block, 0, s>>>(Ainv, n, b, x);
}

// dynamic shared memory: the final sums (lcap + 1 doubles) or the coefficients
// (lcap or 2 lcap doubles); lcap <= kLcapMax keeps it within the default 48 KB
template <typename T>
void launch_gram_dots(const T* W, int N, const T* w, int lcap, int nblk, double* partial,
                      const EpiArgs& e, int conditional, cudaStream_t s) {
  if (N % 2 == 0)   // pairs of elements: every column base is 16-byte (FP64) / 8-byte (FP32) aligned
    k_gram_dots<T, true><<<nblk, kVecThreads, (lcap + 1) * sizeof(double), s>>>(W, N, w, partial, e, conditional);
  else
    k_gram_dots<T, false><<<nblk, kVecThreads, (lcap + 1) * sizeof(double), s>>>(W, N, w, partial, e, conditional);
}

template <typename T>
void launch_gram_apply(const T* W, int N, const T* w, T* wout, int lcap, int nblk, LevelState* st,
                       const double* h, cudaStream_t s) {
  k_gram_apply<T><<<nblk, kVecThreads, lcap * sizeof(double), s>>>(W, N, w, wout, st, h);
}

template <typename T>
void launch_gram_update(const T* W, const T* Z, int N, const T* w, const T* wre, const T* z,
                        const T* r, int lcap, int nblk, double* partial, const EpiArgs& e,
                        cudaStream_t s) {
  if (N % 2 == 0)   // pairs of elements (aligned column bases), half the grid
    k_gram_update<T, true><<<(nblk + 1) / 2, kVecThreads, 2 * lcap * sizeof(double), s>>>(
        const_cast<T*>(W), const_cast<T*>(Z), N, w, wre, z, r, partial, e);
  else
    k_gram_update<T, false><<<nblk, kVecThreads, 2 * lcap * sizeof(double), s>>>(
        const_cast<T*>(W), const_cast<T*>(Z), N, w, wre, z, r, partial, e);
}

template <typename T>
void launch_rm_finish(T* W, T* Z, int N, T* x, T* r, int nblk, double* partial, const EpiArgs& e,
                      cudaStream_t s) {
  k_rm_finish<T><<<nblk, kVecThreads, 0, s>>>(W, Z, N, x, r, partial, e);
}

template <typename T>
void launch_norm(const T* v, int N, int nblk, double* partial, const EpiArgs& e, cudaStream_t s) {
  k_norm<T><<<nblk, kVecThreads, 0, s>>>(v, N, partial, e);
}

void launch_control(const EpiArgs& e, cudaStream_t s) { k_control<<<1, 1, 0, s>>>(e); }

template <typename Ts, typename Td>
void launch_convert(const Ts* src, Td* dst, size_t n, cudaStream_t s) {
  k_convert<Ts, Td><<<nblocks(n, 256), 256, 0, s>>>(src, dst, n);
}
template <typename T>
void launch_axpy_to_double(const T* e, double* x, size_t n, cudaStream_t s) {
  k_axpy_to_double<T><<<nblocks(n, 256), 256, 0, s>>>(e, x, n);
}
void launch_scale_to_float(const double* src, float* dst, double a, size_t n, cudaStream_t s) {
  k_scale_to_float<<<nblocks(n, 256), 256, 0, s>>>(src, dst, a, n);
}
void launch_axpy_scaled_to_double(const float* e, double* x, double a, size_t n, cudaStream_t s) {
  k_axpy_scaled_to_double<<<nblocks(n, 256), 256, 0, s>>>(e, x, a, n);
}

int launch_galerkin(int np, int dim, const double* Af, const int* nbrf, const int* nf,
                    const int* nc, const double* P, double* Ac, cudaStream_t s) {
  const int Cc = nc[0] * nc[1] * (dim == 3 ? nc[2] : 1);
  dim3 grid(Cc, 2 * dim + 1);
  const int threads = ((np * np + 31) / 32) * 32;
  int ok = 0;
  KCMG_ND_SWITCH(np, dim, {
    ok = 1;
    k_galerkin<NP, DIM><<<grid, threads, 0, s>>>(Af, nbrf, mkdims(nf), mkdims(nc), P, Ac);
  });
  return ok;
}

int launch_block_inverse(int np, const double* diag, int ncell, double* inv, int* fail,
                         cudaStream_t s) {
  const int wpb = 4;
  int ok = 0;
  KCMG_NP_SWITCH(np, {
    ok = 1;
    k_block_inverse<NP><<<(ncell + wpb - 1) / wpb, 32 * wpb, 0, s>>>(diag, ncell, inv, fail);
  });
  return ok;
}

void launch_dense_gj_step(double* M, int n, int c, double* fcol, int* fail, cudaStream_t s) {
  k_gj_pivot<<<1, 1024, 0, s>>>(M, n, c, fcol, fail);
  k_gj_elim<<<nblocks((size_t)n * 2 * n, 256, 2048), 256, 0, s>>>(M, n, c, fcol, fail);
}

void launch_assemble_dense(int np, int dim, const double* blk, const int* nbr, int ncell,
                           double* M, cudaStream_t s) {
  const size_t n = (size_t)ncell * np;
  k_assemble_dense<<<nblocks(n * 2 * n, 256), 256, 0, s>>>(np, dim, blk, nbr, ncell, M);
}

void launch_extract_inverse(const double* M, int n, double* Ainv, cudaStream_t s) {
  k_extract_inverse<<<nblocks((size_t)n * n, 256), 256, 0, s>>>(M, n, Ainv);
}

template <typename T>
void launch_interleave(int np, int nslot, const double* nat, int ncell, int G, T* out,
                       cudaStream_t s) {
  const size_t tot = (size_t)nslot * G * ((np + 1) / 2) * 64;
  k_interleave<T><<<nblocks(tot, 256, 1 << 16), 256, 0, s>>>(np, nslot, nat, ncell, G, out);
}

void launch_transpose_blocks(int np, int dim, const double* in, const int* nbr, int ncell,
                             double* out, cudaStream_t s) {
  const size_t tot = (size_t)(2 * dim + 1) * ncell * np * np;
  k_transpose_blocks<<<nblocks(tot, 256, 1 << 16), 256, 0, s>>>(np, dim, in, nbr, ncell, out);
}

void launch_count_diff(const double* a, const double* b, size_t n, unsigned int* cnt,
                       cudaStream_t s) {
  k_count_diff<<<nblocks(n, 256, 1 << 14), 256, 0, s>>>(a, b, n, cnt);
}

void launch_build_nbr(int dim, const int* n, int* nbr, cudaStream_t s) {
  const int C = n[0] * n[1] * (dim == 3 ? n[2] : 1);
  k_build_nbr<<<nblocks(C, 256, 1 << 30), 256, 0, s>>>(dim, mkdims(n), nbr);
}

void launch_grad_lognu(int np, int dim, const int* n, const double* nu, const double* V,
                       const double* F, const double* B, const double* lam, const double* u,
                       double* g, cudaStream_t s) {
  const int C = n[0] * n[1] * (dim == 3 ? n[2] : 1);
  KCMG_NP_SWITCH(np, {
    k_grad_lognu<NP><<<nblocks(C, 128, 1 << 30), 128, 0, s>>>(dim, mkdims(n), nu, V, F, B, lam, u, g);
  });
}

// explicit instantiations
#define KCMG_INST_T(T)                                                                        \
  template void launch_spmv<T>(int, int, const T*, const int*, int, int, int, int, const T*, T*, \
                               const T*, double*, const EpiArgs&, int, cudaStream_t);            \
  template void launch_restrict<T, T>(int, int, const int*, const int*, const T*, const T*, T*,   \
                                      T*, T*, double*, const EpiArgs&, cudaStream_t);            \
  template void launch_prolong<T, T>(int, int, const int*, const int*, const T*, const T*, T*,    \
                                     cudaStream_t);                                              \
  template void launch_coarse_gemv<T>(const double*, int, const T*, T*, cudaStream_t);           \
  template void launch_gram_dots<T>(const T*, int, const T*, int, int, double*, const EpiArgs&,   \
                                    int, cudaStream_t);                                          \
  template void launch_gram_apply<T>(const T*, int, const T*, T*, int, int, LevelState*,         \
                                     const double*, cudaStream_t);                               \
  template void launch_gram_update<T>(const T*, const T*, int, const T*, const T*, const T*,     \
                                      const T*, int, int, double*, const EpiArgs&, cudaStream_t); \
  template void launch_rm_finish<T>(T*, T*, int, T*, T*, int, double*, const EpiArgs&,           \
                                    cudaStream_t);                                               \
  template void launch_norm<T>(const T*, int, int, double*, const EpiArgs&, cudaStream_t);       \
  template void launch_interleave<T>(int, int, const double*, int, int, T*, cudaStream_t);       \
  template void launch_axpy_to_double<T>(const T*, double*, size_t, cudaStream_t);

KCMG_INST_T(double)
KCMG_INST_T(float)
template void launch_bj_sweep<double, double>(int, int, const double*, const double*, const int*, int,
                                              int, int, int, const double*, const double*, double*,
                                              double, int, cudaStream_t);
template void launch_bj_sweep<float, float>(int, int, const float*, const float*, const int*, int, int,
                                            int, int, const float*, const float*, float*, double, int,
                                            cudaStream_t);
template void launch_bj_sweep<float, __nv_bfloat16>(int, int, const float*, const __nv_bfloat16*,
                                                    const int*, int, int, int, int, const float*,
                                                    const float*, float*, double, int, cudaStream_t);
template void launch_interleave<__nv_bfloat16>(int, int, const double*, int, int, __nv_bfloat16*,
                                               cudaStream_t);
template void launch_restrict<float, double>(int, int, const int*, const int*, const float*,
                                             const double*, float*, float*, float*, double*,
                                             const EpiArgs&, cudaStream_t);
template void launch_prolong<float, double>(int, int, const int*, const int*, const float*,
                                            const float*, double*, cudaStream_t);
template void launch_convert<double, float>(const double*, float*, size_t, cudaStream_t);
template void launch_convert<double, __nv_bfloat16>(const double*, __nv_bfloat16*, size_t, cudaStream_t);
template void launch_convert<float, double>(const float*, double*, size_t, cudaStream_t);

}  // namespace kcmg
