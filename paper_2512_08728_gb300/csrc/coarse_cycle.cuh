// Persistent cooperative kernel for the coarse part of the K-cycle: MG(lambda) of Alg. 2
// on every level below the finest, with the block-Jacobi smoother (Alg. BJ), residual
// minimisation (Alg. 1), transfers, the level-local criteria of Sec. 4.2 and the dense
// coarsest solve, all in one launch per finest-level cycle.
//
// Coarse levels are small (here 5K-330K unknowns) and a kernel per step would be bound
// by launch and reduction latency; one resident grid separated by grid barriers keeps
// every SM busy instead.  Every control decision is taken by all blocks from the same
// reduced values (fixed reduction order), so all blocks follow the same path.  The grid
// barrier spins with a bound: if it ever times out it raises an error flag and every
// block leaves the kernel, so a fault becomes a status, not a hang.
#pragma once
#include "kcmg_internal.h"
#include "reduce.cuh"
#include "schwarz.cuh"

#include <cuda/atomic>

#include <cmath>

namespace kcmg {

namespace {

template <typename T> struct V2T;
template <> struct V2T<double> { using type = double2; };
template <> struct V2T<float> { using type = float2; };

template <typename TI> __device__ __forceinline__ float2 inv_pair_f(const TI* p, size_t i);
template <> __device__ __forceinline__ float2 inv_pair_f<float>(const float* p, size_t i) {
  return __ldg(reinterpret_cast<const float2*>(p) + i);
}
template <> __device__ __forceinline__ float2 inv_pair_f<__nv_bfloat16>(const __nv_bfloat16* p, size_t i) {
  return __bfloat1622float2(reinterpret_cast<const __nv_bfloat162*>(p)[i]);
}
template <typename T, typename TI> struct InvLoad {
  static __device__ __forceinline__ void get(const TI* p, size_t i, T& a, T& b) {
    const float2 v = inv_pair_f<TI>(p, i);
    a = (T)v.x;
    b = (T)v.y;
  }
};
template <> struct InvLoad<double, double> {
  static __device__ __forceinline__ void get(const double* p, size_t i, double& a, double& b) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p) + i);
    a = v.x;
    b = v.y;
  }
};

__device__ __forceinline__ double bsum(double v, double* sh) {
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
  return r;  // valid in thread 0
}

template <typename T> __device__ __forceinline__ T ldv(const T* p) { return __ldcg(p); }

}  // namespace

// Grid barrier with a bounded wait.  Every block adds one to a counter (acquire-release,
// which publishes the block's writes) and waits until the counter reaches the total for
// this generation; the host zeroes the counter before every launch.  gen: this block's
// barrier count so far.  Returns false (in every thread of the block) once the error flag
// is set; callers then leave the kernel.
static __device__ __forceinline__ bool cc_barrier(const CoarseArgs& a, unsigned int& gen) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    cuda::atomic_ref<unsigned int, cuda::thread_scope_device> cnt(*a.bar_count);
    cuda::atomic_ref<int, cuda::thread_scope_device> err(*a.err);
    int ok = err.load(cuda::memory_order_relaxed) == 0;
    if (ok) {
      const unsigned int target = (gen + 1) * gridDim.x;
      const unsigned int old = cnt.fetch_add(1u, cuda::memory_order_acq_rel);
      if (old + 1 != target) {
        long long spins = 0;
        while (cnt.load(cuda::memory_order_acquire) < target) {
          if ((++spins & 1023) == 0) {
            if (err.load(cuda::memory_order_relaxed)) break;
            if (spins > (1LL << 23)) {   // seconds: far beyond any legitimate wait
              err.store(1, cuda::memory_order_relaxed);
              break;
            }
          }
        }
      }
      ok = err.load(cuda::memory_order_relaxed) == 0;
    }
    s_ok = ok;
  }
  ++gen;
  __syncthreads();
  return s_ok != 0;
}

namespace {

// Per-level scalars, held identically by every block.
struct LvScal {
  int l, it;
  double rnorm, rnorm0, eps;
};

// Vectors, basis W, Z, the Alg. 1 operator and the transfers are in TV (FP64, or FP32 in
// the inner solve of the iterative-refinement forms); the smoother sweeps run in TS with
// inverses stored as TI.  Reductions and Gram coefficients are FP64 in every form.
template <typename TV, typename TS, typename TI, int NP, int DIM>
struct CoarseCycle {
  using T = TV;
  using V2 = typename V2T<TV>::type;
  using VS2 = typename V2T<TS>::type;
  static constexpr int S = 2 * DIM + 1;
  static constexpr int NF = S - 1;
  static constexpr int JP = (NP + 1) / 2;
  static constexpr int NCH = 1 << DIM;

  const CoarseArgs& a;
  double* sh;      // 32 doubles
  double* red_s;   // reduced sums (shared), >= kCoarseMaxCols
  TS* tile;        // blockDim TS (smoother exchange)
  TS* as_rs;       // (blockDim / 32) x 2^d np TS: a warp's gathered patch residual (Alg. AS)
  T* Ps;           // NCH*NP*NP (prolongation matrices)
  double* cw;      // coefficient vectors in shared memory: 2 * kCoarseMaxCols
  int rcount = 0;  // reductions done (selects the partial buffer)
  unsigned int gen = 0;  // grid barriers passed (identical in every block)
  bool ok = true;
  __device__ bool bar() { return cc_barrier(a, gen); }
  double bytes = 0.0;  // algorithmic bytes of this launch (kept by thread 0 of block 0)

  __device__ void count(double b) {
    if (blockIdx.x == 0 && threadIdx.x == 0) bytes += b;
  }
  // unique operator bytes of n slots on a level with this element size
  __device__ double opbytes(const CoarseLevel& C, int slots, int elem) const {
    return (double)slots * C.N * NP * elem;
  }

  __device__ const CoarseLevel& L(int lev) const { return a.lv[lev]; }
  __device__ T* vec(void* p) const { return static_cast<T*>(p); }

  // ---------------------------------------------------------------- reductions
  // every block: v (this thread's contributions) -> red_s[0..nc) (grid totals)
  template <int NC>
  __device__ bool reduce_few(const double (&v)[NC]) {
    double* part = a.partial + (size_t)(rcount & 1) * a.partial_stride;
    rcount++;
    double t[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) t[c] = v[c];
    bsum_n<NC>(t, sh);
    if (threadIdx.x == 0)
#pragma unroll
      for (int c = 0; c < NC; ++c) part[(size_t)blockIdx.x * NC + c] = t[c];
    if (!bar()) return false;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      double s = 0.0;
      for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s += __ldcg(part + (size_t)b * NC + c);
      t[c] = s;
    }
    bsum_n<NC>(t, sh);
    if (threadIdx.x == 0)
#pragma unroll
      for (int c = 0; c < NC; ++c) red_s[c] = t[c];
    __syncthreads();
    return true;
  }

  // many columns: partial[b][c] already written by every block for c < nc; owners
  // reduce one column each, then all blocks read the totals into red_s
  __device__ bool reduce_cols(double* part, int nc) {
    if (nc * (int)gridDim.x <= 4096) {   // few columns: every block sums all of them
      if (!bar()) return false;
      for (int c0 = 0; c0 < nc; c0 += 8) {
        double t[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          t[c] = 0.0;
          if (c0 + c < nc)
            for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t[c] += __ldcg(part + (size_t)b * nc + c0 + c);
        }
        bsum_n<8>(t, sh);
        if (threadIdx.x == 0)
#pragma unroll
          for (int c = 0; c < 8; ++c)
            if (c0 + c < nc) red_s[c0 + c] = t[c];
      }
      __syncthreads();
      return true;
    }
    if (!bar()) return false;
    for (int c = blockIdx.x; c < nc; c += gridDim.x) {
      double s = 0.0;
      for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s += __ldcg(part + (size_t)b * nc + c);
      s = bsum(s, sh);
      if (threadIdx.x == 0) a.red[c] = s;
    }
    if (!bar()) return false;
    for (int c = threadIdx.x; c < nc; c += blockDim.x) red_s[c] = __ldcg(a.red + c);
    __syncthreads();
    return true;
  }

  // ---------------------------------------------------------------- operator phases
  // y = A x (or b - A x) on level lev; returns this thread's sum of y^2
  __device__ double spmv(int lev, const T* x, T* y, const T* b) {
    const CoarseLevel& C = L(lev);
    const T* A = static_cast<const T*>(C.A);
    count(opbytes(C, S, sizeof(T)) + (double)C.N * sizeof(T) * (b ? 3 : 2));
    double nrm = 0.0;
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < C.rows_pad; row += gridDim.x * blockDim.x) {
      if (row >= C.N) continue;
      const int g = row >> 5, lane = row & 31, K = row / NP;
      T acc[4] = {T(0), T(0), T(0), T(0)};   // independent FMA chains (latency)
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const int J = (s == 0) ? K : __ldg(C.nbr + (size_t)K * NF + s - 1);
        if (J < 0) continue;
        const V2* Ap = reinterpret_cast<const V2*>(A) + ((size_t)(s * C.G + g) * JP) * 32 + lane;
        const T* xp = x + (size_t)J * NP;
        const int c = (s & 1) << 1;
#pragma unroll
        for (int jp = 0; jp < JP; ++jp) {
          const V2 av = __ldg(Ap + jp * 32);
          acc[c] = fma(av.x, ldv(xp + 2 * jp), acc[c]);
          if (2 * jp + 1 < NP) acc[c + 1] = fma(av.y, ldv(xp + 2 * jp + 1), acc[c + 1]);
        }
      }
      const T sum = (acc[0] + acc[1]) + (acc[2] + acc[3]);
      const T out = b ? (ldv(b + row) - sum) : sum;
      y[row] = out;
      nrm = fma((double)out, (double)out, nrm);
    }
    return nrm;
  }

  // One sweep of Alg. BJ in TS over tiles of blockDim rows (whole cells): t = r - A_off zo
  // (skipped on the first sweep from z = 0), zn = (1 - omega) zo + omega D^{-1} t.
  // The last sweep writes the FP64 correction.
  template <typename TO>
  __device__ void sweep(const CoarseLevel& C, const T* r, const TS* zo, TO* zn, bool first) {
    count(opbytes(C, first ? 0 : S - 1, a.smoother_bytes) + opbytes(C, 1, a.inverse_bytes) +
          (double)C.N * (sizeof(T) + sizeof(TO) + (first ? 0 : sizeof(TS))));
    const TS* A = static_cast<const TS*>(C.As);
    const TI* D = static_cast<const TI*>(C.Dinv);
    const TS om = (TS)a.omega;
    const int ntile = C.rows_pad / blockDim.x;
    for (int tl = blockIdx.x; tl < ntile; tl += gridDim.x) {
      const int row = tl * blockDim.x + threadIdx.x;
      const int g = row >> 5, lane = row & 31;
      TS tv = TS(0);
      if (row < C.N) {
        tv = (TS)ldv(r + row);
        if (!first) {
          const int K = row / NP;
          TS acc[4] = {TS(0), TS(0), TS(0), TS(0)};
#pragma unroll
          for (int s = 1; s < S; ++s) {
            const int J = __ldg(C.nbr + (size_t)K * NF + s - 1);
            if (J < 0) continue;
            const VS2* Ap = reinterpret_cast<const VS2*>(A) + ((size_t)(s * C.G + g) * JP) * 32 + lane;
            const TS* zp = zo + (size_t)J * NP;
            const int c = (s & 1) << 1;
#pragma unroll
            for (int jp = 0; jp < JP; ++jp) {
              const VS2 av = __ldg(Ap + jp * 32);
              acc[c] = fma(av.x, ldv(zp + 2 * jp), acc[c]);
              if (2 * jp + 1 < NP) acc[c + 1] = fma(av.y, ldv(zp + 2 * jp + 1), acc[c + 1]);
            }
          }
          tv -= (acc[0] + acc[1]) + (acc[2] + acc[3]);
        }
      }
      __syncthreads();
      tile[threadIdx.x] = tv;
      __syncthreads();
      if (row < C.N) {
        const int base = (row / NP) * NP - tl * blockDim.x;
        TS d0s = TS(0), d1s = TS(0);
#pragma unroll
        for (int jp = 0; jp < JP; ++jp) {
          TS d0, d1;
          InvLoad<TS, TI>::get(D, ((size_t)g * JP + jp) * 32 + lane, d0, d1);
          d0s = fma(d0, tile[base + 2 * jp], d0s);
          if (2 * jp + 1 < NP) d1s = fma(d1, tile[base + 2 * jp + 1], d1s);
        }
        const TS dz = d0s + d1s;
        const TS v = first ? om * dz : fma(TS(1) - om, ldv(zo + row), om * dz);
        zn[row] = (TO)v;
      }
    }
  }

  // Alg. AS phases on a level (schwarz.cuh): the sweep's residual in TS, both partitions'
  // patch solves (one warp per patch), and the combination z_new = z_old + omega (z_0 + z_1)
  __device__ void as_residual(const CoarseLevel& C, const T* r, const TS* zo, bool first) {
    count((double)C.N * (sizeof(T) + sizeof(TS)) + (first ? 0.0 : opbytes(C, S, a.smoother_bytes) + (double)C.N * sizeof(TS)));
    const TS* A = static_cast<const TS*>(C.As);
    TS* res = static_cast<TS*>(C.as_r);
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < C.N; row += gridDim.x * blockDim.x) {
      TS v = (TS)ldv(r + row);
      if (!first) {
        const int g = row >> 5, lane = row & 31, K = row / NP;
        TS acc[4] = {TS(0), TS(0), TS(0), TS(0)};
#pragma unroll
        for (int s = 0; s < S; ++s) {
          const int J = (s == 0) ? K : __ldg(C.nbr + (size_t)K * NF + s - 1);
          if (J < 0) continue;
          const VS2* Ap = reinterpret_cast<const VS2*>(A) + ((size_t)(s * C.G + g) * JP) * 32 + lane;
          const TS* zp = zo + (size_t)J * NP;
          const int c = (s & 1) << 1;
#pragma unroll
          for (int jp = 0; jp < JP; ++jp) {
            const VS2 av = __ldg(Ap + jp * 32);
            acc[c] = fma(av.x, ldv(zp + 2 * jp), acc[c]);
            if (2 * jp + 1 < NP) acc[c + 1] = fma(av.y, ldv(zp + 2 * jp + 1), acc[c + 1]);
          }
        }
        v -= (acc[0] + acc[1]) + (acc[2] + acc[3]);
      }
      res[row] = v;
    }
  }
  __device__ void as_patches(const CoarseLevel& C) {
    constexpr int M = NCH * NP;
    const int np0 = as_npatch(C.n, DIM, 0), np1 = as_npatch(C.n, DIM, 1);
    count((double)(np0 + np1) * M * M * a.inverse_bytes + (double)(np0 + np1) * M * 2 * sizeof(TS));
    const TI* inv0 = static_cast<const TI*>(C.as_inv0);
    const TI* inv1 = static_cast<const TI*>(C.as_inv1);
    const TS* res = static_cast<const TS*>(C.as_r);
    TS* zP = static_cast<TS*>(C.as_z);
    const int warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    TS* rs = as_rs + (size_t)warp * M;
    for (int w = blockIdx.x * wpb + warp; w < np0 + np1; w += gridDim.x * wpb) {
      if (w < np0) as_patch_solve_warp<TS, TI, NP, DIM>(C.n, 0, w, inv0, res, zP, rs);
      else as_patch_solve_warp<TS, TI, NP, DIM>(C.n, 1, w - np0, inv1, res, zP + (size_t)np0 * M, rs);
    }
  }
  template <typename TO>
  __device__ void as_combine(const CoarseLevel& C, const TS* zo, TO* zn, bool first) {
    count((double)C.N * (2 * sizeof(TS) + sizeof(TO)));
    const int np0 = as_npatch(C.n, DIM, 0);
    const TS* zP = static_cast<const TS*>(C.as_z);
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < C.N; row += gridDim.x * blockDim.x)
      zn[row] = (TO)as_combine_row<TS, NP, DIM>(C.n, row, zP, np0, zo, (TS)a.omega, first);
  }

  // z = BJ(r) or AS(r) from z = 0 (a.sweeps sweeps); returns the correction C.z (type T)
  __device__ T* smooth(int lev, const T* r) {
    const CoarseLevel& C = L(lev);
    if (a.smoother == 1) {
      TS* sb[2] = {static_cast<TS*>(C.s0), static_cast<TS*>(C.s1)};
      T* out = vec(C.z);
      for (int k = 0; k < a.sweeps && ok; ++k) {
        const TS* zo = sb[(k + 1) & 1];
        as_residual(C, r, zo, k == 0);
        if (!(ok = bar())) break;
        as_patches(C);
        if (!(ok = bar())) break;
        if (k == a.sweeps - 1) as_combine<T>(C, zo, out, k == 0);
        else as_combine<TS>(C, zo, sb[k & 1], k == 0);
        ok = bar();
        ph(PH_SWEEP);
      }
      return out;
    }
    TS* sb[2] = {static_cast<TS*>(C.s0), static_cast<TS*>(C.s1)};
    T* out = vec(C.z);
    for (int k = 0; k < a.sweeps && ok; ++k) {
      const TS* zo = sb[(k + 1) & 1];
      if (k == a.sweeps - 1) sweep<T>(C, r, zo, out, k == 0);
      else sweep<TS>(C, r, zo, sb[k & 1], k == 0);
      ok = bar();
      ph(PH_SWEEP);
    }
    return out;
  }

  // ---------------------------------------------------------------- Alg. 1
  // returns false on a barrier error
  __device__ bool rm(int lev, const T* z, LvScal& sc) {
    const CoarseLevel& C = L(lev);
    const int N = C.N, l = sc.l;
    T* W = vec(C.W);
    T* Z = vec(C.Z);
    T* w = vec(C.w);
    T* wre = vec(C.wre);
    const T* r = vec(C.r);
    // w = A z.  No grid barrier before the dots: both phases give each thread the same
    // rows (grid-stride), so every w[j] a thread reads it wrote itself.
    spmv(lev, z, w, nullptr);
    // h = W^T w, ||w||^2  (columns in groups of 8)
    const int nc = l + 1;
    double* part = a.partial + (size_t)(rcount & 1) * a.partial_stride;
    rcount++;
    dots(W, N, w, l, part);
    count((double)(l + 1) * N * sizeof(T));
    if (!reduce_cols(part, nc)) return false;
    ph(PH_RM_GRAM1);
    double hh = 0.0;
    for (int i = 0; i < l; ++i) hh += red_s[i] * red_s[i];
    const double naz2 = red_s[l];
    const bool reorth = l > 0 && (naz2 - hh < 0.25 * naz2);
    bool discard = !isfinite(naz2) || !(naz2 > 0.0);
    // coefficients into shared memory: cw (for w), cw + lcap (for z)
    for (int i = threadIdx.x; i < l; i += blockDim.x) { cw[i] = red_s[i]; cw[kCoarseMaxCols + i] = red_s[i]; }
    __syncthreads();
    const T* wsrc = w;
    if (reorth) {
      // w' = w - W h, then h2 = W^T w'
      for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
        T s = ldv(w + j);
        for (int i = 0; i < l; ++i) s = fma((T)(-cw[i]), ldv(W + (size_t)i * N + j), s);
        wre[j] = s;
      }
      if (!bar()) return false;
      double* part2 = a.partial + (size_t)(rcount & 1) * a.partial_stride;
      rcount++;
      dots(W, N, wre, l, part2);
      count((double)(l + 2) * N * sizeof(T) + (double)(l + 1) * N * sizeof(T));   // apply + second dots
      if (!reduce_cols(part2, nc)) return false;
      for (int i = threadIdx.x; i < l; i += blockDim.x) {
        cw[kCoarseMaxCols + i] += red_s[i];   // z gets h + h2
        cw[i] = red_s[i];                     // w' gets h2
      }
      __syncthreads();
      wsrc = wre;
      ph(PH_RM_REORTH);
    }
    // w_hat = wsrc - W cw, z_hat = z - Z cz into column l; ||w_hat||^2, w_hat . r
    T* Wl = W + (size_t)l * N;
    T* Zl = Z + (size_t)l * N;
    double nw2 = 0.0, wr = 0.0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
      T av = ldv(wsrc + j), zv = ldv(z + j), av1 = T(0), zv1 = T(0);
      int i = 0;
      for (; i + 1 < l; i += 2) {
        av = fma((T)(-cw[i]), ldv(W + (size_t)i * N + j), av);
        zv = fma((T)(-cw[kCoarseMaxCols + i]), ldv(Z + (size_t)i * N + j), zv);
        av1 = fma((T)(-cw[i + 1]), ldv(W + (size_t)(i + 1) * N + j), av1);
        zv1 = fma((T)(-cw[kCoarseMaxCols + i + 1]), ldv(Z + (size_t)(i + 1) * N + j), zv1);
      }
      if (i < l) {
        av = fma((T)(-cw[i]), ldv(W + (size_t)i * N + j), av);
        zv = fma((T)(-cw[kCoarseMaxCols + i]), ldv(Z + (size_t)i * N + j), zv);
      }
      av += av1;
      zv += zv1;
      Wl[j] = av;
      Zl[j] = zv;
      nw2 = fma((double)av, (double)av, nw2);
      wr = fma((double)av, (double)ldv(r + j), wr);
    }
    count((double)(2 * l + 5) * N * sizeof(T));   // W, Z columns; w, z, r in; new columns out
    {
      double v[2] = {nw2, wr};
      if (!reduce_few<2>(v)) return false;
    }
    ph(PH_RM_UPDATE);
    const double nw = sqrt(red_s[0]);
    if (!isfinite(nw) || !(nw > a.brk * sqrt(naz2))) discard = true;
    const double gam = discard ? 0.0 : 1.0 / nw;
    const double alp = discard ? 0.0 : gam * red_s[1];
    // normalise and update x, r; ||r||^2
    double r2 = 0.0;
    T* x = vec(C.x);
    T* rr = vec(C.r);
    const T g = (T)gam, al = (T)alp;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
      T rv = ldv(rr + j);
      if (!discard) {
        const T wv = ldv(Wl + j) * g, zv = ldv(Zl + j) * g;
        Wl[j] = wv;
        Zl[j] = zv;
        x[j] = fma(al, zv, ldv(x + j));
        rv = fma(-al, wv, rv);
        rr[j] = rv;
      }
      r2 = fma((double)rv, (double)rv, r2);
    }
    count(discard ? 0.0 : (double)N * 8 * sizeof(T));
    // ||r - alpha w||^2 = ||r||^2 - alpha^2 for unit w with alpha = w . r; reduce the
    // updated vector explicitly only if that cancels more than four digits
    const double r2old = sc.rnorm * sc.rnorm;
    const double r2new = r2old - alp * alp;
    if (discard) {
      // x, r unchanged
    } else if (r2new > 1e-4 * r2old) {
      sc.rnorm = sqrt(r2new);
    } else {
      double v[1] = {r2};
      if (!reduce_few<1>(v)) return false;
      sc.rnorm = sqrt(red_s[0]);
    }
    if (!discard) sc.l++;
    ph(PH_RM_FINISH);
    return true;
  }

  // partial[blk][c] for c < l: W_c . w ; c = l: ||w||^2.  Groups of 8 columns; the last
  // group reads a valid column in place of the missing ones and drops those sums, and the
  // norm is a separate sum of group 0, so every step issues the same FMAs.  Per-thread
  // sums in T, block and grid sums in FP64.
  __device__ void dots(const T* W, int N, const T* w, int l, double* part) {
    const int nc = l + 1;
    const int groups = l > 0 ? (l + 7) / 8 : 1;
    for (int g = 0; g < groups; ++g) {
      const int c0 = 8 * g;
      T acc[8];
      T ww = T(0);
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[c] = T(0);
      for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
        const T wv = ldv(w + j);
        if (l > 0)
#pragma unroll
          for (int c = 0; c < 8; ++c)
            acc[c] = fma(ldv(W + (size_t)min(c0 + c, l - 1) * N + j), wv, acc[c]);
        if (g == 0) ww = fma(wv, wv, ww);
      }
      double v[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) v[c] = (double)acc[c];
      bsum_n<8>(v, sh);
      if (threadIdx.x == 0)
#pragma unroll
        for (int c = 0; c < 8; ++c)
          if (c0 + c < l) part[(size_t)blockIdx.x * nc + c0 + c] = v[c];
      if (g == 0) {
        double n[1] = {(double)ww};
        bsum_n<1>(n, sh);
        if (threadIdx.x == 0) part[(size_t)blockIdx.x * nc + l] = n[0];
      }
    }
  }

  // ---------------------------------------------------------------- transfers
  // b_{lev+1} = R r_lev; with start: r_{lev+1} = b_{lev+1}, x_{lev+1} = 0; returns ||b||^2 part
  __device__ double restrict_(int lev, bool start) {
    const CoarseLevel &F = L(lev), &C = L(lev + 1);
    count((double)F.N * sizeof(T) + (double)C.N * sizeof(T) * (start ? 3 : 1));
    const T* rf = vec(F.r);
    T* bc = vec(C.b);
    double nrm = 0.0;
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < C.N; row += gridDim.x * blockDim.x) {
      const int J = row / NP, i = row - J * NP;
      const int jx = J % C.n[0], jy = (J / C.n[0]) % C.n[1], jz = DIM == 3 ? J / (C.n[0] * C.n[1]) : 0;
      T s = T(0);
#pragma unroll
      for (int k = 0; k < NCH; ++k) {
        const int fx = 2 * jx + (k & 1), fy = 2 * jy + ((k >> 1) & 1), fz = DIM == 3 ? 2 * jz + ((k >> 2) & 1) : 0;
        const int K = fx + F.n[0] * (fy + F.n[1] * fz);
#pragma unroll
        for (int q = 0; q < NP; ++q) s = fma(Ps[(k * NP + q) * NP + i], ldv(rf + (size_t)K * NP + q), s);
      }
      bc[row] = s;
      if (start) {
        vec(C.r)[row] = s;
        vec(C.x)[row] = T(0);
      }
      nrm = fma((double)s, (double)s, nrm);
    }
    return nrm;
  }

  // z_lev = P x_{lev+1}
  __device__ void prolong(int lev) {
    const CoarseLevel &F = L(lev), &C = L(lev + 1);
    count((double)F.N * sizeof(T) + (double)C.N * sizeof(T));
    const T* xc = vec(C.x);
    T* zf = vec(F.z);
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < F.N; row += gridDim.x * blockDim.x) {
      const int K = row / NP, q = row - K * NP;
      const int ix = K % F.n[0], iy = (K / F.n[0]) % F.n[1], iz = DIM == 3 ? K / (F.n[0] * F.n[1]) : 0;
      const int k = (ix & 1) | ((iy & 1) << 1) | (DIM == 3 ? ((iz & 1) << 2) : 0);
      const int J = (ix >> 1) + C.n[0] * ((iy >> 1) + C.n[1] * (iz >> 1));
      T s = T(0);
#pragma unroll
      for (int i = 0; i < NP; ++i) s = fma(Ps[(k * NP + q) * NP + i], ldv(xc + (size_t)J * NP + i), s);
      zf[row] = s;
    }
  }

  // x_c = A_c^{-1} b_c (FP64 dense inverse), one warp per row
  __device__ void coarse_solve(int lev) {
    const CoarseLevel& C = L(lev);
    count((double)a.Nc * a.Nc * 8 + (double)a.Nc * 2 * sizeof(T));
    const T* bc = vec(C.b);
    T* xc = vec(C.x);
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, ln = threadIdx.x & 31;
    for (int row = wid; row < a.Nc; row += warps) {
      double s = 0.0;
      for (int j = ln; j < a.Nc; j += 32) s = fma(__ldg(a.Ainv + (size_t)row * a.Nc + j), (double)ldv(bc + j), s);
#pragma unroll
      for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (ln == 0) xc[row] = (T)s;
    }
  }

  // ---------------------------------------------------------------- Alg. 2 on lev >= 1
  // The recursion MG(lev) -> MG(lev + 1) of Alg. 2 runs as a loop over an explicit
  // per-level state (the levels form a chain, so a phase per level suffices).
  // On entry b, r = b and x = 0 of level lev0 are set and sc[lev0].rnorm0 = ||b||.
  enum Phase { TEST, AFTER_COARSE };

  __device__ void start(int lev, LvScal& sc) {
    sc.l = 0;
    sc.it = 0;
    sc.rnorm = sc.rnorm0;
    sc.eps = L(lev).rtol * sc.rnorm0;
  }

  // time attribution per phase kind (thread 0 of block 0; the interval since the previous
  // phase boundary, closing barrier included)
  unsigned long long t_ph = 0;
  __device__ void ph(int kind) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      unsigned long long t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (t_ph) atomicAdd(a.stat_phase_ns + kind, t - t_ph);
      t_ph = t;
    }
  }

  // time attribution per level (thread 0 of block 0)
  unsigned long long t_mark = 0;
  __device__ void mark(int lev) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      unsigned long long t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (t_mark) atomicAdd(a.stat_level_ns + lev, t - t_mark);
      t_mark = t;
    }
  }

  __device__ void run(int lev0) {
    LvScal sc[KCMG_MAX_LEVELS];
    int phase[KCMG_MAX_LEVELS];
    int restarts[KCMG_MAX_LEVELS];
    int guard[KCMG_MAX_LEVELS];
    for (int i = 0; i < KCMG_MAX_LEVELS; ++i) { phase[i] = TEST; restarts[i] = 0; guard[i] = 0; }
    int lev = lev0;
    mark(lev);
    ph(PH_CONTROL);
    sc[lev].rnorm0 = red_s[0];
    sc[lev].rnorm0 = sqrt(sc[lev].rnorm0);
    start(lev, sc[lev]);
    while (ok) {
      const CoarseLevel& C = L(lev);
      LvScal& s = sc[lev];
      if (phase[lev] == TEST) {
        // while ||r|| > eps (level-local criteria of Sec. 4.2)
        if (!(s.rnorm > s.eps && s.it < C.maxit && guard[lev] < (1 << 24))) {
          if (blockIdx.x == 0 && threadIdx.x == 0 && C.st) {
            C.st->iters_total += s.it;
            C.st->nrestart += restarts[lev];
          }
          mark(lev);
          if (lev == lev0) break;
          --lev;                                                   // return to the caller
          if (!(ok = bar())) break;
          ph(PH_CONTROL);
          continue;
        }
        ++guard[lev];
        T* z = smooth(lev, vec(C.r));                              // pre-smoother
        if (!ok || !(ok = rm(lev, z, s))) break;
        if (!(ok = bar())) break;                                  // r complete everywhere
        const bool direct = (lev + 1 == a.nlev - 1);
        const double nb = restrict_(lev, !direct);                 // r_c = R r
        phase[lev] = AFTER_COARSE;
        if (direct) {
          if (!(ok = bar())) break;
          ph(PH_TRANSFER);
          mark(lev);
          coarse_solve(lev + 1);                                   // z_c = A_c \ r_c
          if (!(ok = bar())) break;
          ph(PH_COARSEST);
          mark(lev + 1);
        } else {
          double v[1] = {nb};
          if (!(ok = reduce_few<1>(v))) break;
          ph(PH_TRANSFER);
          mark(lev);
          ++lev;                                                   // z_c = MG(A_c, r_c, 0)
          sc[lev].rnorm0 = sqrt(red_s[0]);
          start(lev, sc[lev]);
          phase[lev] = TEST;
        }
        continue;
      }
      // AFTER_COARSE: prolongate, minimise, post-smooth, minimise
      prolong(lev);                                                // z = P z_c
      if (!(ok = bar())) break;
      ph(PH_TRANSFER);
      if (!(ok = rm(lev, vec(C.z), s))) break;
      T* z = smooth(lev, vec(C.r));                                // post-smoother
      if (!ok || !(ok = rm(lev, z, s))) break;
      s.it++;
      const int cap = (a.lmax > 0 && a.lmax < C.lcap) ? a.lmax : C.lcap;
      if (s.l + 3 > cap) {                                         // restart: r = b - A x
        if (!(ok = bar())) break;
        double v[1] = {spmv(lev, vec(C.x), vec(C.r), vec(C.b))};
        if (!(ok = reduce_few<1>(v))) break;
        ph(PH_RESTART);
        s.rnorm = sqrt(red_s[0]);
        s.l = 0;
        ++restarts[lev];
      }
      phase[lev] = TEST;
    }
  }
};

// Resident blocks per SM the register allocation must allow.  With 2 the kernel fits in
// 94 registers without spills (158 with 1), so level-0 kernels of the task-parallel cycle
// can run on its SMs beside it: measured 75.8 against 77.5 ms per 64^3 cycle, with the
// coarse kernel itself slower (1.00 against 0.78 ms per launch) as it shares the SMs.
#ifndef KCMG_CC_MINBLOCKS
#define KCMG_CC_MINBLOCKS 2
#endif
template <typename TV, typename TS, typename TI, int NP, int DIM>
__global__ void __launch_bounds__(320, KCMG_CC_MINBLOCKS) k_coarse_cycle(CoarseArgs a) {
  using T = TV;
  extern __shared__ unsigned char smem_raw[];
  __shared__ double sh[32 * 8];
  __shared__ double red_s[kCoarseMaxCols];
  __shared__ double cw[2 * kCoarseMaxCols];
  constexpr int NCH = 1 << DIM;
  T* Ps = reinterpret_cast<T*>(smem_raw);   // prolongation matrices first (8-byte aligned)
  TS* tile = reinterpret_cast<TS*>(Ps + NCH * NP * NP);
  const double* P = static_cast<const double*>(a.P);   // FP64 prolongation matrices
  for (int i = threadIdx.x; i < NCH * NP * NP; i += blockDim.x) Ps[i] = (T)P[i];
  __syncthreads();
  constexpr int M_AS = NCH * NP;
  TS* as_rs = tile + blockDim.x;            // (blockDim / 32) warps x M_AS
  CoarseCycle<TV, TS, TI, NP, DIM> cc{a, sh, red_s, tile, as_rs, Ps, cw};
  unsigned long long t0 = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  // start of MG on the first coarse level: b, r, x were set by the restriction kernel
  const CoarseLevel& C = a.lv[a.lev0];
  double nb = 0.0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < C.N; j += gridDim.x * blockDim.x) {
    const double v = (double)ldv(static_cast<const T*>(C.b) + j);
    nb += v * v;
  }
  double v[1] = {nb};
  if (!cc.reduce_few<1>(v)) return;
  cc.count((double)C.N * sizeof(T));
  cc.run(a.lev0);   // reads ||b||^2 from red_s[0]
  // device time of this launch: every block has passed the last barrier of the cycle
  if (cc.ok) cc.ok = cc.bar();
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    unsigned long long t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    atomicAdd(a.stat_ns, t1 - t0);
    atomicAdd(a.stat_launches, 1ull);
    atomicAdd(a.stat_bytes, cc.bytes);
  }
}

}  // namespace

}  // namespace kcmg
