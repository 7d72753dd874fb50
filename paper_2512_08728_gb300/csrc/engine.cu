// Host engine and C interface of libkcmg: device setup of the agglomeration hierarchy,
// the K-cycle driver (Alg. 2 with Alg. 1 after every correction), FP64 iterative
// refinement around an FP32 cycle, and the CUDA-graph form of the cycle in which every
// level's while loop is a conditional while node driven by device-side state.
#include "kcmg_internal.h"
#include "schwarz.cuh"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

using namespace kcmg;

namespace {

struct Level {
  int n[3] = {1, 1, 1};
  int ncell = 0, N = 0, G = 0, rows_pad = 0, block_rows = 0;
  int* nbr = nullptr;
  double* nat = nullptr;            // natural FP64 blocks [S][C][np][np]
  double* A64 = nullptr;            // row-interleaved FP64 operator
  double* D64 = nullptr;            // row-interleaved FP64 block inverses
  float* A32 = nullptr;             // mixed precision copies
  float* D32 = nullptr;
  __nv_bfloat16* D16 = nullptr;
  void *x = nullptr, *r = nullptr, *b = nullptr, *z = nullptr, *t = nullptr, *w = nullptr,
       *wre = nullptr, *W = nullptr, *Z = nullptr;
  // mixed forms: FP32 buffers of the smoother sweeps (the level's vectors are FP64)
  float *r_lo = nullptr, *z_lo = nullptr, *t_lo = nullptr;
  // additive Schwarz smoother (Alg. AS): transposed patch inverses of partitions 0 and 1,
  // patch solutions and the sweep's residual, all in the smoother's precision
  void *as_inv0 = nullptr, *as_inv1 = nullptr, *as_z = nullptr, *as_r = nullptr;
  // matrix-free level-0 coupling (FP32 sweeps): coefficient per cell, face matrices
  float *mf_nu = nullptr, *mf_F = nullptr;
  int lcap = 0;
  int nblk = 1;                     // blocks of the multi-column dot kernels
  int nblk2 = 1;                    // blocks of the update / finish / norm kernels
  double *h = nullptr, *h2 = nullptr, *partial = nullptr;
  LevelState* st = nullptr;
};

}  // namespace

struct kcmg_ctx {
  kcmg_params p{};
  int dim = 0, np = 0, S = 0, nlev = 0, nch = 0;
  int dev = 0;                        // the device the context was built on
  bool ir = false;                    // FP64 iterative refinement around an FP32 inner solve
  double *xo = nullptr, *bo = nullptr, *xt = nullptr;   // its FP64 outer x, b and trial x
  double* na_scratch = nullptr;       // static scratch of kcmg_residual_noalloc on dev
  bool mixed = false;
  cudaStream_t user = nullptr, s = nullptr;
  cudaStream_t cap[KCMG_MAX_LEVELS + 2] = {};
  cudaEvent_t ev = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;   // task-parallel level-0 cycle
  double* zc = nullptr;                               // its coarse correction (level 0)
  std::vector<Level> lv;
  double* P64 = nullptr;
  float* P32 = nullptr;
  double* Ainv = nullptr;
  int Nc = 0;
  double *ro = nullptr, *scal = nullptr;
  double* hist = nullptr;
  int* hist_type = nullptr;
  int hist_cap = 4096;
  double *stage_in = nullptr, *stage_out = nullptr, *stage_big = nullptr;
  size_t stage_big_len = 0;
  int* dflag = nullptr;
  cudaGraphExec_t gexec = nullptr;
  bool graph_ready = false;
  // persistent coarse cycle (levels >= 1 in one cooperative launch per level-0 cycle)
  bool coarse_kernel = false;
  int cc_lev0 = 0;   // first level run by the persistent kernel
  int cc_grid = 0;
  CoarseArgs cc{};
  long long graph_body_launches = 0;  // kernels per level-0 loop body of the graph
  long long graph_body_kernels[KCMG_MAX_LEVELS] = {};
  long long last_launches = 0;        // kernels of the last cycle run
  // coarse-cycle counters (launches, ns, algorithmic bytes) and report scratch
  unsigned long long* stat_ns = nullptr;
  unsigned long long* stat_launches = nullptr;
  double* stat_bytes = nullptr;
  unsigned long long* stat_level_ns = nullptr;
  unsigned long long* stat_phase_ns = nullptr;
  kcmg_ctx* adj = nullptr;       // transposed hierarchy (may be this)
  MrhsEngine* mrhs = nullptr;    // batched multi-right-hand-side solver (built on demand)
  bool adj_built = false;
  std::vector<void*> allocs;
  std::string err;
};

namespace {

struct Fail {
  kcmg_status st;
};

void set_err(kcmg_ctx* c, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
}

#define CK(call)                                                                     \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      set_err(ctx, "%s failed at %s:%d: %s", #call, __FILE__, __LINE__,              \
              cudaGetErrorString(e_));                                               \
      throw Fail{e_ == cudaErrorMemoryAllocation ? KCMG_OOM : KCMG_CUDA_ERROR};      \
    }                                                                                \
  } while (0)

#define REQUIRE(cond, ...)               \
  do {                                   \
    if (!(cond)) {                       \
      set_err(ctx, __VA_ARGS__);         \
      throw Fail{KCMG_INVALID_ARG};      \
    }                                    \
  } while (0)

template <typename T>
T* dalloc(kcmg_ctx* ctx, size_t n) {
  void* p = nullptr;
  CK(cudaMalloc(&p, n * sizeof(T) + 16));
  ctx->allocs.push_back(p);
  return static_cast<T*>(p);
}

// copy n doubles from a host or device pointer into device memory dst (unified
// addressing lets cudaMemcpyDefault tell host from device pointers)
void copy_in(kcmg_ctx* ctx, double* dst, const double* src, size_t n) {
  CK(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDefault, ctx->s));
}
void copy_out(kcmg_ctx* ctx, double* dst, const double* src, size_t n) {
  CK(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDefault, ctx->s));
}

int level_cells(const int* n, int dim) { return n[0] * n[1] * (dim == 3 ? n[2] : 1); }

// operator of a level's residual minimisation and the prolongation matrices, in the
// level's vector type (FP64; FP32 in the inner solve of the iterative-refinement forms)
template <typename V> const V* level_op(const Level& L);
template <> const double* level_op<double>(const Level& L) { return L.A64; }
template <> const float* level_op<float>(const Level& L) { return L.A32; }
template <typename V> const V* prolong_mats(const kcmg_ctx* c);
template <> const double* prolong_mats<double>(const kcmg_ctx* c) { return c->P64; }
template <> const float* prolong_mats<float>(const kcmg_ctx* c) { return c->P32; }

// ------------------------------------------------------------------ setup
void setup_level_geometry(kcmg_ctx* ctx, Level& L, int l) {
  for (int j = 0; j < 3; ++j) L.n[j] = (j < ctx->dim) ? (ctx->p.n[j] >> l) : 1;
  L.ncell = level_cells(L.n, ctx->dim);
  L.N = L.ncell * ctx->np;
  L.block_rows = block_rows_for(ctx->np);
  L.rows_pad = ((L.N + L.block_rows - 1) / L.block_rows) * L.block_rows;
  L.G = L.rows_pad / 32;
  L.nblk = (L.N + kVecThreads * 4 - 1) / (kVecThreads * 4);
  if (L.nblk > kDotBlocksMax) L.nblk = kDotBlocksMax;
  if (L.nblk < 1) L.nblk = 1;
  L.nblk2 = (L.N + kVecThreads - 1) / kVecThreads;   // one element per thread
  if (L.nblk2 > 2048) L.nblk2 = 2048;
  if (L.nblk2 < 1) L.nblk2 = 1;
  L.nbr = dalloc<int>(ctx, (size_t)L.ncell * 2 * ctx->dim);
  launch_build_nbr(ctx->dim, L.n, L.nbr, ctx->s);
}

template <typename T>
void alloc_cycle_vectors(kcmg_ctx* ctx, Level& L, int lcap) {
  const size_t N = L.N;
  L.lcap = lcap;
  L.x = dalloc<T>(ctx, N);
  L.r = dalloc<T>(ctx, N);
  L.b = dalloc<T>(ctx, N);
  L.z = dalloc<T>(ctx, N);
  L.t = dalloc<T>(ctx, N);
  L.w = dalloc<T>(ctx, N);
  L.wre = dalloc<T>(ctx, N);
  L.W = dalloc<T>(ctx, N * lcap);
  L.Z = dalloc<T>(ctx, N * lcap);
  L.h = dalloc<double>(ctx, lcap);
  L.h2 = dalloc<double>(ctx, lcap);
  const size_t spmv_blocks = L.rows_pad / L.block_rows;
  size_t plen = (size_t)kDotBlocksMax * (lcap + 1);
  if (spmv_blocks > plen) plen = spmv_blocks;
  if ((size_t)4 * 65536 > plen) plen = 4 * 65536;
  L.partial = dalloc<double>(ctx, plen);
  L.st = dalloc<LevelState>(ctx, 1);
  CK(cudaMemsetAsync(L.st, 0, sizeof(LevelState), ctx->s));
}

void build_hierarchy(kcmg_ctx* ctx, const double* blocks_src) {
  const int np = ctx->np, dim = ctx->dim, S = ctx->S;
  const size_t bs = (size_t)np * np;
  for (int l = 0; l < ctx->nlev; ++l) setup_level_geometry(ctx, ctx->lv[l], l);
  // fine natural blocks
  Level& F = ctx->lv[0];
  F.nat = dalloc<double>(ctx, (size_t)S * F.ncell * bs);
  copy_in(ctx, F.nat, blocks_src, (size_t)S * F.ncell * bs);
  for (int l = 0; l + 1 < ctx->nlev; ++l) {
    Level &A = ctx->lv[l], &C = ctx->lv[l + 1];
    C.nat = dalloc<double>(ctx, (size_t)S * C.ncell * bs);
    if (!launch_galerkin(np, dim, A.nat, A.nbr, A.n, C.n, ctx->P64, C.nat, ctx->s))
      REQUIRE(false, "unsupported np %d", np);
    CK(cudaGetLastError());
  }
  // block inverses and interleaved copies
  double* inv_nat = dalloc<double>(ctx, (size_t)F.ncell * bs);
  for (int l = 0; l < ctx->nlev; ++l) {
    Level& L = ctx->lv[l];
    CK(cudaMemsetAsync(ctx->dflag, 0, sizeof(int), ctx->s));
    launch_block_inverse(np, L.nat, L.ncell, inv_nat, ctx->dflag, ctx->s);
    CK(cudaGetLastError());
    int fail = 0;
    CK(cudaMemcpyAsync(&fail, ctx->dflag, sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    if (fail) {
      set_err(ctx, "diagonal block of level %d is singular", l);
      throw Fail{KCMG_SINGULAR};
    }
    const size_t opsz = (size_t)S * L.G * ((np + 1) / 2) * 64;
    const size_t invsz = (size_t)L.G * ((np + 1) / 2) * 64;
    L.A64 = dalloc<double>(ctx, opsz);
    L.D64 = dalloc<double>(ctx, invsz);
    launch_interleave<double>(np, S, L.nat, L.ncell, L.G, L.A64, ctx->s);
    launch_interleave<double>(np, 1, inv_nat, L.ncell, L.G, L.D64, ctx->s);
    if (ctx->mixed) {
      L.A32 = dalloc<float>(ctx, opsz);
      launch_interleave<float>(np, S, L.nat, L.ncell, L.G, L.A32, ctx->s);
      if (ctx->p.precision == KCMG_MIXED_BF16INV || ctx->p.precision == KCMG_IR32_BF16INV) {
        L.D16 = dalloc<__nv_bfloat16>(ctx, invsz);
        launch_interleave<__nv_bfloat16>(np, 1, inv_nat, L.ncell, L.G, L.D16, ctx->s);
      } else {
        L.D32 = dalloc<float>(ctx, invsz);
        launch_interleave<float>(np, 1, inv_nat, L.ncell, L.G, L.D32, ctx->s);
      }
    }
    CK(cudaGetLastError());
  }
  // additive Schwarz smoother: patch inverses of every iterated level (FP64 Gauss-Jordan,
  // then stored in the smoother's precision)
  if (ctx->p.smoother == 1) {
    const int m = (1 << dim) * np;
    const bool bf16 = ctx->p.precision == KCMG_MIXED_BF16INV || ctx->p.precision == KCMG_IR32_BF16INV;
    size_t maxp = 0;
    for (int l = 0; l + 1 < ctx->nlev; ++l)
      for (int part = 0; part < 2; ++part) {
        const size_t c = (size_t)as_npatch(ctx->lv[l].n, dim, part);
        if (c > maxp) maxp = c;
      }
    double* tmp = nullptr;   // FP64 inverses of one partition before conversion
    if (ctx->mixed) CK(cudaMalloc(&tmp, maxp * m * m * sizeof(double)));
    try {
      for (int l = 0; l + 1 < ctx->nlev; ++l) {
        Level& L = ctx->lv[l];
        for (int part = 0; part < 2; ++part) {
          const size_t cnt = (size_t)as_npatch(L.n, dim, part) * m * m;
          double* inv64 = ctx->mixed ? tmp : dalloc<double>(ctx, cnt);
          CK(cudaMemsetAsync(ctx->dflag, 0, sizeof(int), ctx->s));
          CK(launch_patch_inverse(np, dim, L.nat, L.nbr, L.n, part, inv64, ctx->dflag, ctx->s));
          int fail = 0;
          CK(cudaMemcpyAsync(&fail, ctx->dflag, sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
          CK(cudaStreamSynchronize(ctx->s));
          if (fail) {
            set_err(ctx, "a Schwarz patch matrix of level %d is singular", l);
            throw Fail{KCMG_SINGULAR};
          }
          void* dst = inv64;
          if (ctx->mixed && bf16) {
            __nv_bfloat16* b16 = dalloc<__nv_bfloat16>(ctx, cnt);
            launch_convert<double, __nv_bfloat16>(inv64, b16, cnt, ctx->s);
            dst = b16;
          } else if (ctx->mixed) {
            float* f32 = dalloc<float>(ctx, cnt);
            launch_convert<double, float>(inv64, f32, cnt, ctx->s);
            dst = f32;
          }
          CK(cudaGetLastError());
          CK(cudaStreamSynchronize(ctx->s));   // tmp is reused by the next partition
          (part == 0 ? L.as_inv0 : L.as_inv1) = dst;
        }
        const size_t nz = ((size_t)as_npatch(L.n, dim, 0) + as_npatch(L.n, dim, 1)) * m;
        const size_t es = ctx->mixed ? sizeof(float) : sizeof(double);
        L.as_z = dalloc<char>(ctx, nz * es);
        L.as_r = dalloc<char>(ctx, (size_t)L.N * es);
      }
    } catch (...) {
      if (tmp) cudaFree(tmp);
      throw;
    }
    if (tmp) cudaFree(tmp);
  }
  // dense inverse of the coarsest operator (Gauss-Jordan with partial pivoting)
  Level& C = ctx->lv[ctx->nlev - 1];
  const int n = C.N;
  ctx->Nc = n;
  double* M = dalloc<double>(ctx, (size_t)n * 2 * n);
  double* fcol = dalloc<double>(ctx, n);
  launch_assemble_dense(np, dim, C.nat, C.nbr, C.ncell, M, ctx->s);
  CK(cudaMemsetAsync(ctx->dflag, 0, sizeof(int), ctx->s));
  for (int c = 0; c < n; ++c) launch_dense_gj_step(M, n, c, fcol, ctx->dflag, ctx->s);
  CK(cudaGetLastError());
  ctx->Ainv = dalloc<double>(ctx, (size_t)n * n);
  launch_extract_inverse(M, n, ctx->Ainv, ctx->s);
  int fail = 0;
  CK(cudaMemcpyAsync(&fail, ctx->dflag, sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaStreamSynchronize(ctx->s));
  if (fail) {
    set_err(ctx, "coarsest operator (%d DOFs) is singular", n);
    throw Fail{KCMG_SINGULAR};
  }
}

// ------------------------------------------------------------------ the cycle
// Every level keeps its vectors, basis W, Z and residual minimisation (Alg. 1, with the
// FP64 operator) in T0 = FP64, as do the transfers and the coarsest solve; the smoother
// sweeps run in T.  T = double is the FP64 form; T = float the mixed form, in which the
// FP64 residual minimisation over FP32-smoothed corrections acts as the iterative
// refinement (the attainable residual is FP64's).
void launch_coarse(kcmg_ctx* ctx, cudaStream_t s) {
  CK(cudaMemsetAsync(ctx->cc.bar_count, 0, sizeof(unsigned int), s));   // barrier counter
  cudaError_t err;
  const int thr = ctx->lv[ctx->cc_lev0].block_rows;
  const bool bf16 = ctx->p.precision == KCMG_MIXED_BF16INV || ctx->p.precision == KCMG_IR32_BF16INV;
  if (!ctx->mixed) err = launch_coarse_cycle<double, double, double>(ctx->cc, ctx->cc_grid, thr, s);
  else if (ctx->ir && bf16) err = launch_coarse_cycle<float, float, __nv_bfloat16>(ctx->cc, ctx->cc_grid, thr, s);
  else if (ctx->ir) err = launch_coarse_cycle<float, float, float>(ctx->cc, ctx->cc_grid, thr, s);
  else if (bf16) err = launch_coarse_cycle<double, float, __nv_bfloat16>(ctx->cc, ctx->cc_grid, thr, s);
  else err = launch_coarse_cycle<double, float, float>(ctx->cc, ctx->cc_grid, thr, s);
  CK(err);
}

template <typename T0, typename T>
struct Cycle {
  kcmg_ctx* ctx;
  bool capture = false;
  cudaGraphConditionalHandle handle[KCMG_MAX_LEVELS] = {};
  long long launches = 0;   // kernels issued (eager) or recorded (capture)

  static constexpr bool kMixed = !std::is_same<T0, T>::value;

  const T* Ainner(const Level& L) const;   // operator in T
  const T* Pm() const;

  EpiArgs epi(int lev, int kind) const {
    Level& L = ctx->lv[lev];
    EpiArgs e;
    e.st = L.st;
    e.kind = kind;
    e.h = L.h;
    e.h2 = L.h2;
    if (lev == 0) {
      e.hist = ctx->hist;
      e.hist_type_buf = ctx->hist_type;
    }
    if (capture) {
      e.use_handle = 1;
      e.handle = handle[lev];
    }
    return e;
  }

  // Alg. AS in T on buffers z/t: per sweep the residual r - A z_old (skipped on the first
  // sweep from z = 0), both partitions' patch solves, and z_new = z_old + omega (z_0 + z_1)
  T* as_sweeps(const Level& L, const T* r, T* z, T* t, cudaStream_t s) {
    T* buf[2] = {z, t};
    T* res = static_cast<T*>(L.as_r);
    T* zp = static_cast<T*>(L.as_z);
    const double om = ctx->p.omega;
    const int sw = ctx->p.sweeps;
    const bool bf16 = ctx->p.precision == KCMG_MIXED_BF16INV || ctx->p.precision == KCMG_IR32_BF16INV;
    for (int k = 0; k < sw; ++k) {
      T* out = buf[k & 1];
      const T* old = buf[(k + 1) & 1];
      const T* rk = r;
      if (k > 0) {
        launches += 1;
        launch_spmv<T>(ctx->np, ctx->dim, Ainner(L), L.nbr, L.N, L.G, L.rows_pad, L.block_rows, old, res, r,
                       nullptr, EpiArgs{}, 0, s);
        rk = res;
      }
      launches += 2;
      if (std::is_same<T, double>::value)
        launch_as_patch<double, double>(ctx->np, ctx->dim, L.n, (const double*)L.as_inv0, (const double*)L.as_inv1,
                                        (const double*)rk, (double*)zp, s);
      else if (bf16)
        launch_as_patch<float, __nv_bfloat16>(ctx->np, ctx->dim, L.n, (const __nv_bfloat16*)L.as_inv0,
                                              (const __nv_bfloat16*)L.as_inv1, (const float*)rk, (float*)zp, s);
      else
        launch_as_patch<float, float>(ctx->np, ctx->dim, L.n, (const float*)L.as_inv0, (const float*)L.as_inv1,
                                      (const float*)rk, (float*)zp, s);
      launch_as_combine<T>(ctx->np, ctx->dim, L.n, L.N, zp, old, out, om, k == 0, s);
    }
    return buf[(sw - 1) & 1];
  }

  // the smoother sweeps in T on buffers z/t; returns the buffer holding the result
  T* sweeps(const Level& L, const T* r, T* z, T* t, cudaStream_t s) {
    if (ctx->p.smoother == 1) return as_sweeps(L, r, z, t, s);
    T* buf[2] = {z, t};
    const double om = ctx->p.omega;
    const int sw = ctx->p.sweeps;
    launches += sw;
    for (int k = 0; k < sw; ++k) {
      T* out = buf[k & 1];
      const T* old = buf[(k + 1) & 1];
      if (!std::is_same<T, double>::value && L.mf_nu) {   // level 0, coupling matrix-free
        if (L.D16)
          launch_bj_sweep_mf<__nv_bfloat16>(ctx->np, ctx->dim, L.n, L.mf_nu, L.mf_F, L.D16, L.N, L.rows_pad,
                                            L.block_rows, (const float*)r, (const float*)old, (float*)out, om,
                                            k == 0, s);
        else
          launch_bj_sweep_mf<float>(ctx->np, ctx->dim, L.n, L.mf_nu, L.mf_F, L.D32, L.N, L.rows_pad,
                                    L.block_rows, (const float*)r, (const float*)old, (float*)out, om, k == 0, s);
      } else if (std::is_same<T, double>::value) {
        launch_bj_sweep<double, double>(ctx->np, ctx->dim, (const double*)Ainner(L), L.D64, L.nbr, L.N,
                                        L.G, L.rows_pad, L.block_rows, (const double*)r,
                                        (const double*)old, (double*)out, om, k == 0, s);
      } else if (L.D16) {
        launch_bj_sweep<float, __nv_bfloat16>(ctx->np, ctx->dim, (const float*)Ainner(L), L.D16, L.nbr,
                                              L.N, L.G, L.rows_pad, L.block_rows, (const float*)r,
                                              (const float*)old, (float*)out, om, k == 0, s);
      } else {
        launch_bj_sweep<float, float>(ctx->np, ctx->dim, (const float*)Ainner(L), L.D32, L.nbr, L.N,
                                      L.G, L.rows_pad, L.block_rows, (const float*)r,
                                      (const float*)old, (float*)out, om, k == 0, s);
      }
    }
    return buf[(sw - 1) & 1];
  }

  // z = BJ(r) from z = 0 on level lev (Alg. BJ); V is the level's vector type
  template <typename V>
  V* smooth(int lev, const V* r, cudaStream_t s) {
    Level& L = ctx->lv[lev];
    if (kMixed) {
      launches += 2;
      launch_convert<double, float>((const double*)r, L.r_lo, L.N, s);
      const float* out = (const float*)sweeps(L, (const T*)L.r_lo, (T*)L.z_lo, (T*)L.t_lo, s);
      launch_convert<float, double>(out, (double*)L.z, L.N, s);
      return static_cast<V*>(L.z);
    }
    return (V*)sweeps(L, (const T*)r, static_cast<T*>(L.z), static_cast<T*>(L.t), s);
  }

  // Alg. 1 on level lev with correction z (vectors in V, operator Aop)
  template <typename V>
  void rm(int lev, const V* Aop, const V* z, int end_iter, int htype, cudaStream_t s) {
    Level& L = ctx->lv[lev];
    V* W = static_cast<V*>(L.W);
    V* Z = static_cast<V*>(L.Z);
    V* w = static_cast<V*>(L.w);
    V* wre = static_cast<V*>(L.wre);
    EpiArgs none = epi(lev, EPI_NONE);
    launches += 6;
    launch_spmv<V>(ctx->np, ctx->dim, Aop, L.nbr, L.N, L.G, L.rows_pad, L.block_rows, z, w,
                   nullptr, L.partial, none, 0, s);
    launch_gram_dots<V>(W, L.N, w, L.lcap, L.nblk, L.partial, epi(lev, EPI_GRAM1), 0, s);
    launch_gram_apply<V>(W, L.N, w, wre, L.lcap, L.nblk2, L.st, L.h, s);
    launch_gram_dots<V>(W, L.N, wre, L.lcap, L.nblk, L.partial, epi(lev, EPI_GRAM2), 1, s);
    launch_gram_update<V>(W, Z, L.N, w, wre, z, static_cast<V*>(L.r), L.lcap, L.nblk2, L.partial,
                          epi(lev, EPI_UPDATE), s);
    EpiArgs fin = epi(lev, EPI_FINISH);
    fin.end_iter = end_iter;
    fin.hist_type = htype;
    launch_rm_finish<V>(W, Z, L.N, static_cast<V*>(L.x), static_cast<V*>(L.r), L.nblk2, L.partial,
                        fin, s);
  }

  // one pass of the while body of Alg. 2 on level lev; V is the level's vector type
  template <typename V>
  void body(int lev, const V* Aop, cudaStream_t s) {
    Level& L = ctx->lv[lev];
    Level& C = ctx->lv[lev + 1];
    V* z = smooth<V>(lev, static_cast<V*>(L.r), s);                       // pre-smoother
    rm<V>(lev, Aop, z, 0, 1, s);
    launches += 3;                                                         // transfers, restart check
    if (lev + 1 == ctx->nlev - 1) {                                        // direct solve
      launches += 1;
      launch_restrict<V, V>(ctx->np, ctx->dim, L.n, C.n, prolong_mats<V>(ctx), static_cast<V*>(L.r),
                            static_cast<V*>(C.b), nullptr, nullptr, nullptr, EpiArgs{}, s);
      launch_coarse_gemv<V>(ctx->Ainv, ctx->Nc, static_cast<V*>(C.b), static_cast<V*>(C.x), s);
    } else if (ctx->coarse_kernel && lev + 1 == ctx->cc_lev0) {            // small levels in
      launch_restrict<V, V>(ctx->np, ctx->dim, L.n, C.n, prolong_mats<V>(ctx), static_cast<V*>(L.r),  // one
                            static_cast<V*>(C.b), static_cast<V*>(C.r), static_cast<V*>(C.x),  // launch
                            nullptr, EpiArgs{}, s);
      launches += 1;
      launch_coarse(ctx, s);
    } else {                                                               // recursion
      if (capture) {
        cudaGraph_t g;
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t* deps;
        const cudaGraphEdgeData* ed;
        size_t nd;
        unsigned long long id;
        CK(cudaStreamGetCaptureInfo(s, &cs, &id, &g, &deps, &ed, &nd));
        CK(cudaGraphConditionalHandleCreate(&handle[lev + 1], g, 0, 0));
      }
      launch_restrict<V, V>(ctx->np, ctx->dim, L.n, C.n, prolong_mats<V>(ctx), static_cast<V*>(L.r),
                            static_cast<V*>(C.b), static_cast<V*>(C.r), static_cast<V*>(C.x),
                            C.partial, epi(lev + 1, EPI_MG_BEGIN), s);
      loop<V>(lev + 1, level_op<V>(C), s);
    }
    launch_prolong<V, V>(ctx->np, ctx->dim, L.n, C.n, prolong_mats<V>(ctx), static_cast<V*>(C.x),
                         static_cast<V*>(L.z), s);                         // z = P z_c
    rm<V>(lev, Aop, static_cast<V*>(L.z), 0, 2, s);
    z = smooth<V>(lev, static_cast<V*>(L.r), s);                           // post-smoother
    rm<V>(lev, Aop, z, 1, 3, s);
    // restart check: r = b - A x on request, then the loop condition of this level
    // (compensated on level 0, where the tolerance can sit near the attainable accuracy)
    if (lev == 0 && std::is_same<V, double>::value)
      launch_residual_dd(ctx->np, ctx->dim, (const double*)Aop, L.nbr, L.N, L.G, L.rows_pad, L.block_rows,
                         (const double*)L.x, (double*)L.r, (const double*)L.b, L.partial,
                         epi(lev, EPI_RESTART), 1, s);
    else
      launch_spmv<V>(ctx->np, ctx->dim, Aop, L.nbr, L.N, L.G, L.rows_pad, L.block_rows,
                     static_cast<V*>(L.x), static_cast<V*>(L.r), static_cast<V*>(L.b), L.partial,
                     epi(lev, EPI_RESTART), 1, s);
  }

  // One cycle of Alg. AsyncMG on level 0 with a fixed smoother count m.  The coarse path
  // (restriction of the cycle-start residual, MG on level 1 or the direct solve,
  // prolongation into zc) runs on its own stream, forked after the restriction; the
  // smoother path applies m smoother + RM steps on s meanwhile; after the join one RM
  // with zc closes the cycle.  The two paths share no buffer: the smoother path writes the
  // level-0 z, t, w, W, Z, x, r and state, the coarse path level >= 1 buffers and zc.
  template <typename V>
  void body_async(const V* Aop, cudaStream_t s) {
    Level& L = ctx->lv[0];
    Level& C = ctx->lv[1];
    cudaStream_t cs = ctx->cap[KCMG_MAX_LEVELS + 1];
    const bool direct = ctx->nlev == 2;
    const bool persistent = !direct && ctx->coarse_kernel && ctx->cc_lev0 == 1;
    if (!direct && !persistent && capture) {
      cudaGraph_t g;
      cudaStreamCaptureStatus cst;
      const cudaGraphNode_t* deps;
      const cudaGraphEdgeData* ed;
      size_t nd;
      unsigned long long id;
      CK(cudaStreamGetCaptureInfo(s, &cst, &id, &g, &deps, &ed, &nd));
      CK(cudaGraphConditionalHandleCreate(&handle[1], g, 0, 0));
    }
    launches += 1;                                                      // r_c = R r
    if (direct)
      launch_restrict<V, V>(ctx->np, ctx->dim, L.n, C.n, prolong_mats<V>(ctx), static_cast<V*>(L.r),
                            static_cast<V*>(C.b), nullptr, nullptr, nullptr, EpiArgs{}, s);
    else if (persistent)
      launch_restrict<V, V>(ctx->np, ctx->dim, L.n, C.n, prolong_mats<V>(ctx), static_cast<V*>(L.r),
                            static_cast<V*>(C.b), static_cast<V*>(C.r), static_cast<V*>(C.x),
                            nullptr, EpiArgs{}, s);
    else
      launch_restrict<V, V>(ctx->np, ctx->dim, L.n, C.n, prolong_mats<V>(ctx), static_cast<V*>(L.r),
                            static_cast<V*>(C.b), static_cast<V*>(C.r), static_cast<V*>(C.x),
                            C.partial, epi(1, EPI_MG_BEGIN), s);
    CK(cudaEventRecord(ctx->fork_ev, s));                                // fork
    CK(cudaStreamWaitEvent(cs, ctx->fork_ev, 0));
    // smoother path first, so that host-driven coarse control overlaps it
    for (int k = 0; k < ctx->p.async_smooth; ++k) {
      V* z = smooth<V>(0, static_cast<V*>(L.r), s);
      rm<V>(0, Aop, z, 0, 1, s);
    }
    // coarse path
    if (direct) {
      launches += 1;
      launch_coarse_gemv<V>(ctx->Ainv, ctx->Nc, static_cast<V*>(C.b), static_cast<V*>(C.x), cs);
    } else if (persistent) {
      launches += 1;
      launch_coarse(ctx, cs);
    } else {
      loop<V>(1, level_op<V>(C), cs);
    }
    launches += 1;
    launch_prolong<V, V>(ctx->np, ctx->dim, L.n, C.n, prolong_mats<V>(ctx), static_cast<V*>(C.x),
                         reinterpret_cast<V*>(ctx->zc), cs);                // z_cor = P z_c
    CK(cudaEventRecord(ctx->join_ev, cs));                               // join
    CK(cudaStreamWaitEvent(s, ctx->join_ev, 0));
    rm<V>(0, Aop, reinterpret_cast<const V*>(ctx->zc), 1, 2, s);
    launches += 1;                                                       // restart check
    if (std::is_same<V, double>::value)
      launch_residual_dd(ctx->np, ctx->dim, (const double*)Aop, L.nbr, L.N, L.G, L.rows_pad, L.block_rows,
                         (const double*)L.x, (double*)L.r, (const double*)L.b, L.partial,
                         epi(0, EPI_RESTART), 1, s);
    else
      launch_spmv<V>(ctx->np, ctx->dim, Aop, L.nbr, L.N, L.G, L.rows_pad, L.block_rows,
                     static_cast<V*>(L.x), static_cast<V*>(L.r), static_cast<V*>(L.b), L.partial,
                     epi(0, EPI_RESTART), 1, s);
  }

  long long body_launches = 0;                        // level-0 loop body (capture)
  long long body_kernels[KCMG_MAX_LEVELS] = {};       // kernels of one body per level,
  long long loop_total[KCMG_MAX_LEVELS + 1] = {};     // excluding nested loops

  // host-driven control: the loop condition, read on the stream that runs the level
  bool read_cond(int lev, cudaStream_t s) {
    int c = 0;
    CK(cudaMemcpyAsync(&c, &ctx->lv[lev].st->cond, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return c != 0;
  }

  // while (cond_lev) body(lev): host-driven, or a conditional while node when capturing
  template <typename V>
  void loop(int lev, const V* Aop, cudaStream_t s) {
    const bool task_parallel = lev == 0 && ctx->p.async_smooth > 0;
    if (!capture) {
      while (read_cond(lev, s)) {
        if (task_parallel) body_async<V>(Aop, s);
        else body<V>(lev, Aop, s);
      }
      return;
    }
    cudaGraph_t g;
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t* deps;
    const cudaGraphEdgeData* ed;
    size_t nd;
    unsigned long long id;
    CK(cudaStreamGetCaptureInfo(s, &cs, &id, &g, &deps, &ed, &nd));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle[lev];
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, g, deps, ed, nd, &cp));
    CK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    cudaStream_t bs = ctx->cap[lev + 1];
    CK(cudaStreamBeginCaptureToGraph(bs, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                     cudaStreamCaptureModeRelaxed));
    const long long before = launches;
    loop_total[lev + 1] = 0;
    if (task_parallel) body_async<V>(Aop, bs);
    else body<V>(lev, Aop, bs);
    loop_total[lev] = launches - before;
    body_kernels[lev] = loop_total[lev] - loop_total[lev + 1];
    if (lev == 0) body_launches = launches - before;
    CK(cudaStreamEndCapture(bs, nullptr));
  }

  // level 0: r0 = b - A x0 (compensated FP64; FP32 in the inner solve of the
  // iterative-refinement forms), then the level-0 loop
  void run(cudaStream_t s) {
    Level& L = ctx->lv[0];
    if (capture) {
      cudaGraph_t g;
      cudaStreamCaptureStatus cs;
      const cudaGraphNode_t* deps;
      const cudaGraphEdgeData* ed;
      size_t nd;
      unsigned long long id;
      CK(cudaStreamGetCaptureInfo(s, &cs, &id, &g, &deps, &ed, &nd));
      CK(cudaGraphConditionalHandleCreate(&handle[0], g, 0, 0));
    }
    if (std::is_same<T0, double>::value)
      launch_residual_dd(ctx->np, ctx->dim, L.A64, L.nbr, L.N, L.G, L.rows_pad, L.block_rows,
                         static_cast<double*>(L.x), static_cast<double*>(L.r), static_cast<double*>(L.b),
                         L.partial, epi(0, EPI_MG_BEGIN), 0, s);
    else
      launch_spmv<T0>(ctx->np, ctx->dim, level_op<T0>(L), L.nbr, L.N, L.G, L.rows_pad, L.block_rows,
                      static_cast<T0*>(L.x), static_cast<T0*>(L.r), static_cast<T0*>(L.b), L.partial,
                      epi(0, EPI_MG_BEGIN), 0, s);
    loop<T0>(0, level_op<T0>(L), s);
  }
};

template <> const double* Cycle<double, double>::Ainner(const Level& L) const { return L.A64; }
template <> const float* Cycle<double, float>::Ainner(const Level& L) const { return L.A32; }
template <> const double* Cycle<double, double>::Pm() const { return ctx->P64; }
template <> const float* Cycle<double, float>::Pm() const { return ctx->P32; }
template <> const float* Cycle<float, float>::Ainner(const Level& L) const { return L.A32; }
template <> const float* Cycle<float, float>::Pm() const { return ctx->P32; }

// host copy of the level states before a cycle
void init_states(kcmg_ctx* ctx, double rtol0, double atol0, int maxit0) {
  long long cap = (long long)maxit0 + 2;
  for (int l = 0; l < ctx->nlev; ++l) {
    if (l > 0) cap = cap * (ctx->p.lvl_maxit[l] > 0 ? ctx->p.lvl_maxit[l] : 1) + 2;
    if (cap > (1LL << 30)) cap = 1LL << 30;
    LevelState h;
    memset(&h, 0, sizeof h);
    h.level = l;
    h.lcap = ctx->lv[l].lcap;
    h.lmax = ctx->p.lmax;
    h.maxit = (l == 0) ? maxit0 : ctx->p.lvl_maxit[l];
    h.rtol = (l == 0) ? rtol0 : ctx->p.lvl_rtol[l];
    h.atol = (l == 0) ? atol0 : 0.0;
    h.status = KCMG_OK;
    h.hist_cap = (l == 0) ? ctx->hist_cap : 0;
    // breakdown threshold of Alg. 1 relative to ||A z|| (the minimisation is FP64)
    h.brk = 1e-14;
    h.guard = 0;
    h.guard_cap = (int)cap;
    h.per_cycle = (l == 0 && ctx->p.async_smooth > 0) ? ctx->p.async_smooth + 1 : 3;
    if (!ctx->lv[l].st) continue;   // the coarsest level is solved directly: no state
    CK(cudaMemcpyAsync(ctx->lv[l].st, &h, sizeof h, cudaMemcpyHostToDevice, ctx->s));
  }
  if (ctx->coarse_kernel) {   // grid-barrier counter and error flag of the coarse cycle
    CK(cudaMemsetAsync(ctx->cc.bar_count, 0, sizeof(unsigned int), ctx->s));
    CK(cudaMemsetAsync(ctx->cc.err, 0, sizeof(int), ctx->s));
  }
  CK(cudaStreamSynchronize(ctx->s));
}

template <typename T0, typename T>
void run_cycle(kcmg_ctx* ctx) {
  if (ctx->p.use_graph) {
    if (!ctx->graph_ready) {
      Cycle<T0, T> cy{ctx};
      cy.capture = true;
      ctx->graph_body_launches = 0;
      cudaGraph_t g;
      CK(cudaStreamBeginCapture(ctx->s, cudaStreamCaptureModeRelaxed));
      try {
        cy.run(ctx->s);
      } catch (...) {
        cudaStreamEndCapture(ctx->s, &g);
        cudaGetLastError();
        throw;
      }
      CK(cudaStreamEndCapture(ctx->s, &g));
      // kernels per execution of each level's loop body (nested loops excluded)
      ctx->graph_body_launches = 0;
      for (int l = 0; l < KCMG_MAX_LEVELS; ++l) ctx->graph_body_kernels[l] = cy.body_kernels[l];
      CK(cudaGraphInstantiate(&ctx->gexec, g, 0));
      CK(cudaGraphDestroy(g));
      ctx->graph_ready = true;
    }
    CK(cudaGraphLaunch(ctx->gexec, ctx->s));
    ctx->last_launches = -2;   // filled from the cycle count after the solve
  } else {
    Cycle<T0, T> cy{ctx};
    cy.launches = 1;           // the initial residual
    cy.run(ctx->s);
    ctx->last_launches = cy.launches;
  }
  CK(cudaGetLastError());
}

// true FP64 residual r = b - A x with the FP64 operator; returns ||r||
double fp64_residual(kcmg_ctx* ctx, const double* x, const double* b, double* r) {
  Level& L = ctx->lv[0];
  EpiArgs e;
  e.st = L.st;  // only its reduction ticket is used
  e.kind = EPI_NORM;
  e.out = ctx->scal;
  launch_residual_dd(ctx->np, ctx->dim, L.A64, L.nbr, L.N, L.G, L.rows_pad, L.block_rows, x, r, b,
                     L.partial, e, 0, ctx->s);
  CK(cudaGetLastError());
  double v = 0;
  CK(cudaMemcpyAsync(&v, ctx->scal, sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaStreamSynchronize(ctx->s));
  return v;
}

struct StateReport {
  LevelState st[KCMG_MAX_LEVELS];
};

void read_states(kcmg_ctx* ctx, StateReport& rep) {
  memset(&rep, 0, sizeof rep);
  for (int l = 0; l < ctx->nlev; ++l)
    if (ctx->lv[l].st)
      CK(cudaMemcpyAsync(&rep.st[l], ctx->lv[l].st, sizeof(LevelState), cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaStreamSynchronize(ctx->s));
}

// kernels of one run of the cycle, from the loop-body counts and the executed bodies
long long cycle_launches(const kcmg_ctx* ctx, const StateReport& rep) {
  if (ctx->last_launches != -2) return ctx->last_launches + 1;
  long long n = 2;                  // initial and final residual
  for (int l = 0; l < ctx->nlev; ++l) n += (long long)rep.st[l].guard * ctx->graph_body_kernels[l];
  return n;
}

void fill_info(kcmg_ctx* ctx, kcmg_info* info, const StateReport& rep, double res0, double rel) {
  if (!info) return;
  info->iters = rep.st[0].iters_total;
  for (int l = 0; l < KCMG_MAX_LEVELS; ++l) info->level_iters[l] = l < ctx->nlev ? rep.st[l].iters_total : 0;
  info->restarts = rep.st[0].nrestart;
  // each level-0 restart replaces the recursive residual by the FP64 true residual:
  // in the mixed form these are the refinement steps (plus the initial residual)
  info->refinements = ctx->mixed ? rep.st[0].nrestart + 1 : 0;
  info->res0 = res0;
  info->rel_res = rel;
  info->kernel_launches = cycle_launches(ctx, rep);
  const int hl = rep.st[0].hist_len;
  info->hist_len = 0;
  if (info->hist && info->hist_type && info->hist_cap > 0) {
    const int m = hl < info->hist_cap ? hl : info->hist_cap;
    if (m > 0) {
      CK(cudaMemcpyAsync(info->hist, ctx->hist, m * sizeof(double), cudaMemcpyDefault, ctx->s));
      CK(cudaMemcpyAsync(info->hist_type, ctx->hist_type, m * sizeof(int), cudaMemcpyDefault, ctx->s));
      CK(cudaStreamSynchronize(ctx->s));
    }
    info->hist_len = m;
  }
}

// FP64 iterative refinement around the FP32 inner K-cycle (KCMG_IR32, KCMG_IR32_BF16INV).
// Outer step: r = b - A x with the FP64 operator (compensated sums); stop when
// ||r|| <= max(rtol ||r0||, atol); else solve A e = r / ||r|| by the K-cycle in FP32 to
// the inner tolerance (level 0 from e = 0, empty basis) and take x + ||r|| e if that lowers
// the FP64 residual.  A step that does not is discarded and ends the solve, so x is never
// worse than x0.
kcmg_status solve_ir(kcmg_ctx* ctx, const double* b, double* x, double rtol, double atol,
                     int maxiter, kcmg_info* info) {
  Level& L = ctx->lv[0];
  const size_t N = L.N;
  copy_in(ctx, ctx->bo, b, N);
  copy_in(ctx, ctx->xo, x, N);
  double rn = fp64_residual(ctx, ctx->xo, ctx->bo, ctx->ro);
  const double r0 = rn;
  const double eps = fmax(rtol * r0, atol);
  std::vector<double> hist(1, rn);
  std::vector<int> htype(1, 0);
  StateReport rep;
  int cycles = 0, steps = 0, restarts = 0, status = KCMG_OK;
  int lit[KCMG_MAX_LEVELS] = {0};
  long long launches = 1;
  while (std::isfinite(rn) && rn > eps && cycles < maxiter && steps < ctx->p.ir_max_steps) {
    launch_scale_to_float(ctx->ro, static_cast<float*>(L.b), 1.0 / rn, N, ctx->s);   // inner b
    CK(cudaMemsetAsync(L.x, 0, N * sizeof(float), ctx->s));                          // inner x0
    init_states(ctx, ctx->p.ir_inner_rtol, 0.0, std::min(maxiter - cycles, ctx->p.ir_inner_maxit));
    run_cycle<float, float>(ctx);
    read_states(ctx, rep);
    if (ctx->coarse_kernel) {
      int bar_err = 0;
      CK(cudaMemcpyAsync(&bar_err, ctx->cc.err, sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
      CK(cudaStreamSynchronize(ctx->s));
      if (bar_err) {
        set_err(ctx, "coarse cycle: a grid barrier timed out; the result is invalid");
        return KCMG_CUDA_ERROR;
      }
    }
    cycles += rep.st[0].iters_total;
    restarts += rep.st[0].nrestart;
    for (int l = 0; l < ctx->nlev; ++l) lit[l] += rep.st[l].iters_total;
    launches += cycle_launches(ctx, rep) + 3;   // + inner b, update, FP64 residual
    ++steps;
    if (rep.st[0].status != KCMG_OK) {          // breakdown or non-finite inner iterate
      status = rep.st[0].status;
      break;
    }
    // trial x_t = x + ||r|| e and its FP64 residual (into ro)
    CK(cudaMemcpyAsync(ctx->xt, ctx->xo, N * sizeof(double), cudaMemcpyDeviceToDevice, ctx->s));
    launch_axpy_scaled_to_double(static_cast<const float*>(L.x), ctx->xt, rn, N, ctx->s);
    const double rt = fp64_residual(ctx, ctx->xt, ctx->bo, ctx->ro);
    if (!(rt < rn)) break;                      // no progress: keep x, stop
    std::swap(ctx->xo, ctx->xt);
    rn = rt;
    hist.push_back(rn);
    htype.push_back(6);
  }
  copy_out(ctx, x, ctx->xo, N);
  CK(cudaStreamSynchronize(ctx->s));
  if (info) {
    info->iters = cycles;
    for (int l = 0; l < KCMG_MAX_LEVELS; ++l) info->level_iters[l] = l < ctx->nlev ? lit[l] : 0;
    info->restarts = restarts;
    info->refinements = steps;
    info->res0 = r0;
    info->rel_res = r0 > 0 ? rn / r0 : 0.0;
    info->kernel_launches = launches;
    info->hist_len = 0;
    if (info->hist && info->hist_type && info->hist_cap > 0) {
      const int m = std::min<int>((int)hist.size(), info->hist_cap);
      CK(cudaMemcpy(info->hist, hist.data(), m * sizeof(double), cudaMemcpyDefault));
      CK(cudaMemcpy(info->hist_type, htype.data(), m * sizeof(int), cudaMemcpyDefault));
      info->hist_len = m;
    }
  }
  if (status != KCMG_OK) return (kcmg_status)status;
  if (!std::isfinite(rn)) return KCMG_NONFINITE;
  return (rn <= eps) ? KCMG_OK : KCMG_NOT_CONVERGED;
}

kcmg_status solve_impl(kcmg_ctx* ctx, const double* b, double* x, double rtol, double atol,
                       int maxiter, kcmg_info* info) {
  if (ctx->ir) return solve_ir(ctx, b, x, rtol, atol, maxiter, info);
  Level& L = ctx->lv[0];
  const size_t N = L.N;
  StateReport rep;
  copy_in(ctx, static_cast<double*>(L.b), b, N);
  copy_in(ctx, static_cast<double*>(L.x), x, N);
  init_states(ctx, rtol, atol, maxiter);
  if (ctx->mixed) run_cycle<double, float>(ctx);
  else run_cycle<double, double>(ctx);
  read_states(ctx, rep);
  if (ctx->coarse_kernel) {
    int bar_err = 0;
    CK(cudaMemcpyAsync(&bar_err, ctx->cc.err, sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    if (bar_err) {
      set_err(ctx, "coarse cycle: a grid barrier timed out; the result is invalid");
      return KCMG_CUDA_ERROR;
    }
  }
  const double rn = fp64_residual(ctx, static_cast<double*>(L.x), static_cast<double*>(L.b), ctx->ro);
  const double r0 = rep.st[0].rnorm0;
  copy_out(ctx, x, static_cast<double*>(L.x), N);
  CK(cudaStreamSynchronize(ctx->s));
  const double rel = r0 > 0 ? rn / r0 : 0.0;
  fill_info(ctx, info, rep, r0, rel);
  if (rep.st[0].status != KCMG_OK) return (kcmg_status)rep.st[0].status;
  if (!std::isfinite(rn)) return KCMG_NONFINITE;
  return (rn <= fmax(rtol * r0, atol)) ? KCMG_OK : KCMG_NOT_CONVERGED;
}

kcmg_ctx* build_ctx(const kcmg_params* p, cudaStream_t user, const double* blocks_override,
                    kcmg_status* out_status, std::string* msg);

// the hierarchy of ctx as the batched solver sees it
MrhsView mrhs_view(kcmg_ctx* ctx) {
  MrhsView v;
  memset(&v, 0, sizeof v);
  v.dim = ctx->dim;
  v.np = ctx->np;
  v.nlev = ctx->nlev;
  for (int l = 0; l < ctx->nlev; ++l) {
    const Level& L = ctx->lv[l];
    for (int j = 0; j < 3; ++j) v.n[l][j] = L.n[j];
    v.ncell[l] = L.ncell;
    v.N[l] = L.N;
    v.nat[l] = L.nat;
    v.nbr[l] = L.nbr;
  }
  v.P = ctx->P64;
  v.Ainv = ctx->Ainv;
  v.Nc = ctx->Nc;
  v.omega = ctx->p.omega;
  v.sweeps = ctx->p.sweeps;
  for (int l = 0; l < KCMG_MAX_LEVELS; ++l) {
    v.lvl_rtol[l] = ctx->p.lvl_rtol[l];
    v.lvl_maxit[l] = ctx->p.lvl_maxit[l];
  }
  v.lmax = ctx->p.lmax;
  v.precision = ctx->p.precision;
  v.tc_tf32_only = ctx->p.tc_tf32_only;
  v.async_smooth = ctx->p.async_smooth;
  v.s = ctx->s;
  return v;
}

// batched solve of nrhs > 1 columns on the hierarchy of ctx
kcmg_status solve_multi(kcmg_ctx* ctx, const double* b, double* x, int nrhs, double rtol, double atol,
                        int maxiter, kcmg_info* info) {
  return mrhs_solve(&ctx->mrhs, mrhs_view(ctx), b, x, nrhs, rtol, atol, maxiter, info, &ctx->err);
}

}  // namespace

// ====================================================================== C interface
extern "C" {

void kcmg_default_params(kcmg_params* p, int dim, int np, const int n[3], int nlevels) {
  memset(p, 0, sizeof *p);
  p->dim = dim;
  p->np = np;
  for (int j = 0; j < 3; ++j) p->n[j] = n ? n[j] : 1;
  p->nlevels = nlevels;
  p->omega = 0.7;
  p->sweeps = 5;
  for (int l = 0; l < KCMG_MAX_LEVELS; ++l) { p->lvl_rtol[l] = 0.0; p->lvl_maxit[l] = 1; }
  p->lvl_rtol[1] = 0.1; p->lvl_maxit[1] = 20;
  p->lvl_rtol[2] = 0.5; p->lvl_maxit[2] = 2;
  p->lmax = 0;
  p->precision = KCMG_FP64;
  p->use_graph = 1;
  p->coarse_persistent = 1;
  p->ir_inner_rtol = 1e-3;
  p->ir_max_steps = 64;
  p->ir_inner_maxit = 300;
}

const char* kcmg_status_string(kcmg_status s) {
  switch (s) {
    case KCMG_OK: return "ok";
    case KCMG_NOT_CONVERGED: return "not converged";
    case KCMG_BREAKDOWN: return "breakdown";
    case KCMG_NONFINITE: return "non-finite value";
    case KCMG_SINGULAR: return "singular block or coarse operator";
    case KCMG_INVALID_ARG: return "invalid argument";
    case KCMG_OOM: return "out of device memory";
    case KCMG_CUDA_ERROR: return "CUDA error";
  }
  return "unknown";
}

const char* kcmg_last_error(const kcmg_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int kcmg_level_cells(const kcmg_ctx* ctx, int level) {
  if (!ctx || level < 0 || level >= ctx->nlev) return 0;
  return ctx->lv[level].ncell;
}

void kcmg_destroy(kcmg_ctx* ctx) {
  if (!ctx) return;
  if (ctx->adj && ctx->adj != ctx) kcmg_destroy(ctx->adj);
  if (ctx->s) cudaStreamSynchronize(ctx->s);
  if (ctx->mrhs) mrhs_destroy(ctx->mrhs);
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  for (void* p : ctx->allocs) cudaFree(p);
  if (ctx->stage_big) cudaFree(ctx->stage_big);
  for (auto& c : ctx->cap) if (c) cudaStreamDestroy(c);
  if (ctx->s) cudaStreamDestroy(ctx->s);
  if (ctx->ev) cudaEventDestroy(ctx->ev);
  if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
  if (ctx->join_ev) cudaEventDestroy(ctx->join_ev);
  delete ctx;
}

kcmg_status kcmg_setup(kcmg_ctx** out, const kcmg_params* p, void* cuda_stream) {
  if (!out || !p) return KCMG_INVALID_ARG;
  *out = nullptr;
  kcmg_status st = KCMG_OK;
  std::string msg;
  kcmg_ctx* ctx = build_ctx(p, (cudaStream_t)cuda_stream, nullptr, &st, &msg);
  *out = ctx;
  return st;
}

}  // extern "C"

namespace {

kcmg_ctx* build_ctx(const kcmg_params* p, cudaStream_t user, const double* blocks_override,
                    kcmg_status* out_status, std::string* msg) {
  kcmg_ctx* ctx = new kcmg_ctx();
  ctx->p = *p;
  try {
    REQUIRE(p->dim == 2 || p->dim == 3, "dim must be 2 or 3");
    REQUIRE(np_supported(p->np, p->dim), "unsupported np %d for dim %d (2-D: 3, 6, 10; 3-D: 4, 10, 20)",
            p->np, p->dim);
    REQUIRE(p->nlevels >= 2 && p->nlevels <= KCMG_MAX_LEVELS, "nlevels must be in [2, %d]", KCMG_MAX_LEVELS);
    REQUIRE(p->blocks && p->prolong, "blocks and prolong must be set");
    REQUIRE(p->sweeps >= 1 && p->sweeps <= 64, "sweeps must be in [1, 64]");
    REQUIRE(p->precision >= 0 && p->precision <= KCMG_IR32_BF16INV, "unknown precision %d", p->precision);
    if (p->precision >= KCMG_IR32) {
      REQUIRE(p->ir_inner_rtol > 0.0 && p->ir_inner_rtol < 1.0, "ir_inner_rtol must be in (0, 1)");
      REQUIRE(p->ir_max_steps >= 1, "ir_max_steps must be >= 1");
      REQUIRE(p->ir_inner_maxit >= 1, "ir_inner_maxit must be >= 1");
    }
    for (int j = 0; j < p->dim; ++j)
      REQUIRE(p->n[j] > 0 && p->n[j] % (1 << (p->nlevels - 1)) == 0,
              "n[%d] = %d is not divisible by 2^(nlevels-1)", j, p->n[j]);
    REQUIRE(p->lmax >= 0 && p->lmax <= kLcapMax - 3, "lmax must be in [0, %d]", kLcapMax - 3);
    REQUIRE(p->async_smooth >= 0 && p->async_smooth <= 64, "async_smooth must be in [0, 64]");
    REQUIRE(p->smoother == 0 || p->smoother == 1, "smoother must be 0 (block Jacobi) or 1 (additive Schwarz)");
    ctx->dim = p->dim;
    ctx->np = p->np;
    ctx->S = 2 * p->dim + 1;
    ctx->nlev = p->nlevels;
    ctx->nch = 1 << p->dim;
    ctx->mixed = p->precision != KCMG_FP64;
    ctx->ir = p->precision >= KCMG_IR32;
    ctx->user = user;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    ctx->dev = dev;
    CK(cudaStreamCreateWithFlags(&ctx->s, cudaStreamNonBlocking));
    {
      // Capture streams: cap[l + 1] records the loop body of level l.  The coarse path of
      // the task-parallel cycle (its stream, and the bodies of levels >= 1 that it nests)
      // takes the highest priority, so that its latency-bound kernels get SMs first while
      // the smoother path fills the rest; kernels captured in a graph keep the priority of
      // the stream they were captured on.  KCMG_COARSE_PRIORITY=0 turns this off (tuning).
      int lo = 0, hi = 0;
      CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
      int prio_on = 1;
      if (const char* ev = getenv("KCMG_COARSE_PRIORITY")) prio_on = atoi(ev) != 0;
      for (int l = 0; l < KCMG_MAX_LEVELS + 1; ++l) {
        const bool coarse = prio_on && p->async_smooth > 0 && l >= 2;
        CK(cudaStreamCreateWithPriority(&ctx->cap[l], cudaStreamNonBlocking, coarse ? hi : lo));
      }
      CK(cudaStreamCreateWithPriority(&ctx->cap[KCMG_MAX_LEVELS + 1], cudaStreamNonBlocking,
                                      prio_on ? hi : lo));
    }
    CK(cudaEventCreateWithFlags(&ctx->ev, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ctx->join_ev, cudaEventDisableTiming));
    if (user) {
      CK(cudaEventRecord(ctx->ev, user));
      CK(cudaStreamWaitEvent(ctx->s, ctx->ev, 0));
    }
    ctx->lv.resize(ctx->nlev);
    ctx->dflag = dalloc<int>(ctx, 4);
    ctx->scal = dalloc<double>(ctx, 8);
    const size_t bs = (size_t)ctx->np * ctx->np;
    ctx->P64 = dalloc<double>(ctx, ctx->nch * bs);
    copy_in(ctx, ctx->P64, p->prolong, ctx->nch * bs);
    ctx->P32 = dalloc<float>(ctx, ctx->nch * bs);
    launch_convert<double, float>(ctx->P64, ctx->P32, ctx->nch * bs, ctx->s);
    build_hierarchy(ctx, blocks_override ? blocks_override : p->blocks);
    if (p->mf_nu || p->mf_F) {   // matrix-free level-0 coupling for the FP32 sweeps
      REQUIRE(p->mf_nu && p->mf_F, "mf_nu and mf_F go together");
      REQUIRE(ctx->mixed, "the matrix-free level-0 sweeps serve the FP32-smoother forms");
      REQUIRE(!blocks_override, "matrix-free data describes the forward operator only");
      Level& L0 = ctx->lv[0];
      const size_t nF = (size_t)ctx->dim * 4 * ctx->np * ctx->np;
      double* nu64 = dalloc<double>(ctx, L0.ncell);
      double* F64 = dalloc<double>(ctx, nF);
      copy_in(ctx, nu64, p->mf_nu, L0.ncell);
      copy_in(ctx, F64, p->mf_F, nF);
      double md = 0, ma = 0;
      CK(mf_check(ctx->np, ctx->dim, L0.n, nu64, F64, L0.nat, &md, &ma, ctx->s));
      REQUIRE(md <= 1e-12 * ma, "matrix-free data does not reproduce the off-diagonal blocks "
              "(max difference %.3e, max entry %.3e)", md, ma);
      L0.mf_nu = dalloc<float>(ctx, L0.ncell);
      L0.mf_F = dalloc<float>(ctx, nF);
      launch_convert<double, float>(nu64, L0.mf_nu, L0.ncell, ctx->s);
      launch_convert<double, float>(F64, L0.mf_F, nF, ctx->s);
      CK(cudaGetLastError());
    }
    // cycle vectors: level 0 basis capacity from lmax (or a default), coarse levels from
    // the per-level iteration caps (3 stored corrections per cycle)
    for (int l = 0; l < ctx->nlev - 1; ++l) {
      int cap;
      // level 0 holds lmax vectors plus one cycle's corrections (3 in Alg. 2, m + 1 in
      // the task-parallel cycle): the restart test runs at the end of a cycle
      const int per_cycle0 = std::max(3, p->async_smooth + 1);
      if (l == 0) cap = (p->lmax > 0 ? p->lmax : 512 - per_cycle0) + per_cycle0;
      else cap = 3 * (p->lvl_maxit[l] > 0 ? p->lvl_maxit[l] : 1) + 3;
      if (p->lmax > 0 && l > 0 && p->lmax + 3 < cap) cap = p->lmax + 3;
      if (cap > kLcapMax) cap = kLcapMax;
      // keep the level-0 basis within a third of the free device memory
      if (l == 0) {
        size_t fr = 0, tot = 0;
        CK(cudaMemGetInfo(&fr, &tot));
        const size_t per = (size_t)2 * ctx->lv[0].N * (ctx->ir ? sizeof(float) : sizeof(double));
        while (cap > 16 && (size_t)cap * per > fr / 3) cap /= 2;
        if (cap < per_cycle0 + 3) cap = per_cycle0 + 3;   // one cycle must always fit
      }
      if (ctx->ir) alloc_cycle_vectors<float>(ctx, ctx->lv[l], cap);
      else alloc_cycle_vectors<double>(ctx, ctx->lv[l], cap);
      if (ctx->mixed) {   // FP32 smoother buffers (and FP32 scratch of the component calls)
        Level& Lm = ctx->lv[l];
        Lm.r_lo = dalloc<float>(ctx, Lm.N);
        Lm.z_lo = dalloc<float>(ctx, Lm.N);
        Lm.t_lo = dalloc<float>(ctx, Lm.N);
      }
    }
    {  // coarsest level: b (restricted residual) and x (direct solution) only
      Level& C = ctx->lv[ctx->nlev - 1];
      C.b = dalloc<double>(ctx, C.N);   // FP32 vectors of the inner solve fit as well
      C.x = dalloc<double>(ctx, C.N);
    }
    // persistent coarse cycle for levels >= 1 (needs at least one iterated coarse level)
    // The persistent kernel takes the coarse levels from the first one small enough that
    // a kernel per step would be latency-bound (levels above stay on full-occupancy
    // kernels under a nested conditional node); it needs at least one iterated level.
    {
      int rows_max = 100000;
      if (const char* ev = getenv("KCMG_PERSISTENT_ROWS")) rows_max = atoi(ev);
      ctx->cc_lev0 = 0;
      for (int l = 1; l < ctx->nlev - 1; ++l)
        if (ctx->lv[l].N <= rows_max) { ctx->cc_lev0 = l; break; }
    }
    ctx->coarse_kernel = p->coarse_persistent && ctx->cc_lev0 > 0;
    if (ctx->coarse_kernel) {
      for (int l = ctx->cc_lev0; l < ctx->nlev - 1; ++l)
        REQUIRE(ctx->lv[l].lcap + 1 <= kCoarseMaxCols,
                "level %d keeps %d basis vectors; the persistent coarse cycle supports %d",
                l, ctx->lv[l].lcap, kCoarseMaxCols - 1);
      int grid = 0;
      const int thr = ctx->lv[ctx->cc_lev0].block_rows;
      cudaError_t ge;
      const bool bf16 = p->precision == KCMG_MIXED_BF16INV || p->precision == KCMG_IR32_BF16INV;
      if (!ctx->mixed) ge = coarse_cycle_grid<double, double, double>(ctx->np, ctx->dim, thr, &grid);
      else if (ctx->ir && bf16) ge = coarse_cycle_grid<float, float, __nv_bfloat16>(ctx->np, ctx->dim, thr, &grid);
      else if (ctx->ir) ge = coarse_cycle_grid<float, float, float>(ctx->np, ctx->dim, thr, &grid);
      else if (bf16) ge = coarse_cycle_grid<double, float, __nv_bfloat16>(ctx->np, ctx->dim, thr, &grid);
      else ge = coarse_cycle_grid<double, float, float>(ctx->np, ctx->dim, thr, &grid);
      CK(ge);
      if (const char* ev = getenv("KCMG_COARSE_GRID")) {   // tuning override, capped at residency
        const int g = atoi(ev);
        if (g > 0 && g < grid) grid = g;
      }
      ctx->cc_grid = grid;
      CoarseArgs& a = ctx->cc;
      memset(&a, 0, sizeof a);
      a.lev0 = ctx->cc_lev0;
      a.nlev = ctx->nlev;
      a.dim = ctx->dim;
      a.np = ctx->np;
      a.P = ctx->P64;
      a.omega = p->omega;
      a.sweeps = p->sweeps;
      a.lmax = p->lmax;
      a.brk = 1e-14;
      a.partial_stride = (size_t)grid * kCoarseMaxCols;
      a.partial = dalloc<double>(ctx, 2 * a.partial_stride);
      a.red = dalloc<double>(ctx, kCoarseMaxCols);
      a.bar_count = dalloc<unsigned int>(ctx, 1);
      a.bar_gen = dalloc<unsigned int>(ctx, 1);
      a.err = dalloc<int>(ctx, 1);
      CK(cudaMemsetAsync(a.bar_gen, 0, sizeof(unsigned int), ctx->s));
      for (int l = 1; l < ctx->nlev; ++l) {
        Level& L = ctx->lv[l];
        CoarseLevel& c = a.lv[l];
        c.A = ctx->ir ? (const void*)L.A32 : (const void*)L.A64;      // Alg. 1 operator
        c.As = ctx->mixed ? (const void*)L.A32 : (const void*)L.A64;  // smoother operator
        c.Dinv = !ctx->mixed ? (const void*)L.D64 : L.D16 ? (const void*)L.D16 : (const void*)L.D32;
        const bool lo = ctx->mixed && !ctx->ir;                       // FP64 vectors, FP32 sweeps
        c.s0 = lo ? (void*)L.z_lo : L.t;                              // smoother scratch
        c.s1 = lo ? (void*)L.t_lo : L.wre;
        c.nbr = L.nbr;
        for (int j = 0; j < 3; ++j) c.n[j] = L.n[j];
        c.N = L.N;
        c.G = L.G;
        c.rows_pad = L.rows_pad;
        c.x = L.x; c.r = L.r; c.b = L.b; c.z = L.z; c.t = L.t; c.w = L.w; c.wre = L.wre;
        c.W = L.W; c.Z = L.Z;
        c.lcap = L.lcap;
        c.maxit = p->lvl_maxit[l];
        c.rtol = p->lvl_rtol[l];
        c.st = L.st;
        c.as_inv0 = L.as_inv0;
        c.as_inv1 = L.as_inv1;
        c.as_z = L.as_z;
        c.as_r = L.as_r;
      }
      a.smoother = p->smoother;
      a.Ainv = ctx->Ainv;
      a.Nc = ctx->Nc;
      ctx->stat_ns = dalloc<unsigned long long>(ctx, 1);
      ctx->stat_launches = dalloc<unsigned long long>(ctx, 1);
      ctx->stat_bytes = dalloc<double>(ctx, 1);
      ctx->stat_level_ns = dalloc<unsigned long long>(ctx, KCMG_MAX_LEVELS);
      CK(cudaMemsetAsync(ctx->stat_level_ns, 0, 8 * KCMG_MAX_LEVELS, ctx->s));
      a.stat_level_ns = ctx->stat_level_ns;
      ctx->stat_phase_ns = dalloc<unsigned long long>(ctx, kCoarsePhases);
      CK(cudaMemsetAsync(ctx->stat_phase_ns, 0, 8 * kCoarsePhases, ctx->s));
      a.stat_phase_ns = ctx->stat_phase_ns;
      CK(cudaMemsetAsync(ctx->stat_ns, 0, 8, ctx->s));
      CK(cudaMemsetAsync(ctx->stat_launches, 0, 8, ctx->s));
      CK(cudaMemsetAsync(ctx->stat_bytes, 0, 8, ctx->s));
      a.stat_ns = ctx->stat_ns;
      a.stat_launches = ctx->stat_launches;
      a.stat_bytes = ctx->stat_bytes;
      a.smoother_bytes = ctx->mixed ? 4 : 8;
      a.inverse_bytes = !ctx->mixed ? 8 : (bf16 ? 2 : 4);
    }
    const size_t N0 = ctx->lv[0].N;
    ctx->ro = dalloc<double>(ctx, N0);
    if (ctx->ir) {   // FP64 vectors of the outer refinement loop
      ctx->xo = dalloc<double>(ctx, N0);
      ctx->bo = dalloc<double>(ctx, N0);
      ctx->xt = dalloc<double>(ctx, N0);
    }
    if (p->async_smooth > 0) ctx->zc = dalloc<double>(ctx, N0);
    ctx->hist = dalloc<double>(ctx, ctx->hist_cap);
    ctx->hist_type = dalloc<int>(ctx, ctx->hist_cap);
    size_t maxN = 0;
    for (auto& L : ctx->lv) maxN = maxN > (size_t)L.N ? maxN : (size_t)L.N;
    ctx->stage_in = dalloc<double>(ctx, maxN);
    ctx->stage_out = dalloc<double>(ctx, maxN);
    // the no-allocation residual's static scratch on this device (address and kernels)
    CK(noalloc_prepare(dev, &ctx->na_scratch));
    CK(cudaStreamSynchronize(ctx->s));
    *out_status = KCMG_OK;
    return ctx;
  } catch (Fail& f) {
    *out_status = f.st;
    if (msg) *msg = ctx->err;
    // keep the context so that kcmg_last_error can report; the caller destroys it
    return ctx;
  }
}

// vectors of every level are FP64 (the mixed forms use FP32 only in the smoother sweeps),
// or FP32 in the inner solve of the iterative-refinement forms
bool level_is_f32(const kcmg_ctx* ctx, int) { return ctx->ir; }

// FP64 user vector -> level buffer of the level's type
void load_vec(kcmg_ctx* ctx, int lev, void* dst, const double* src, size_t n) {
  copy_in(ctx, ctx->stage_in, src, n);
  if (level_is_f32(ctx, lev)) launch_convert<double, float>(ctx->stage_in, static_cast<float*>(dst), n, ctx->s);
  else CK(cudaMemcpyAsync(dst, ctx->stage_in, n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->s));
}
void store_vec(kcmg_ctx* ctx, int lev, double* dst, const void* src, size_t n) {
  if (level_is_f32(ctx, lev)) launch_convert<float, double>(static_cast<const float*>(src), ctx->stage_out, n, ctx->s);
  else CK(cudaMemcpyAsync(ctx->stage_out, src, n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->s));
  copy_out(ctx, dst, ctx->stage_out, n);
  CK(cudaStreamSynchronize(ctx->s));
}

template <typename F>
kcmg_status guarded(kcmg_ctx* ctx, F&& f) {
  if (!ctx) return KCMG_INVALID_ARG;
  try {
    if (ctx->user) {
      CK(cudaEventRecord(ctx->ev, ctx->user));
      CK(cudaStreamWaitEvent(ctx->s, ctx->ev, 0));
    }
    kcmg_status st = f();
    if (ctx->user) {
      CK(cudaEventRecord(ctx->ev, ctx->s));
      CK(cudaStreamWaitEvent(ctx->user, ctx->ev, 0));
    }
    return st;
  } catch (Fail& e) {
    return e.st;
  }
}

kcmg_status ensure_adjoint(kcmg_ctx* ctx) {
  if (ctx->adj_built) return KCMG_OK;
  Level& F = ctx->lv[0];
  const size_t tot = (size_t)ctx->S * F.ncell * ctx->np * ctx->np;
  double* tr = nullptr;
  CK(cudaMalloc(&tr, tot * sizeof(double)));
  launch_transpose_blocks(ctx->np, ctx->dim, F.nat, F.nbr, F.ncell, tr, ctx->s);
  unsigned int* cnt = reinterpret_cast<unsigned int*>(ctx->dflag);
  CK(cudaMemsetAsync(cnt, 0, sizeof(unsigned int), ctx->s));
  launch_count_diff(F.nat, tr, tot, cnt, ctx->s);
  unsigned int nd = 0;
  CK(cudaMemcpyAsync(&nd, cnt, sizeof nd, cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaStreamSynchronize(ctx->s));
  if (nd == 0) {
    ctx->adj = ctx;
  } else {
    kcmg_status st = KCMG_OK;
    std::string msg;
    kcmg_params pa = ctx->p;
    pa.prolong = ctx->P64;   // the caller's setup arrays may be gone by now
    pa.blocks = tr;
    kcmg_ctx* a = build_ctx(&pa, nullptr, tr, &st, &msg);
    if (st != KCMG_OK) {
      set_err(ctx, "adjoint setup failed: %s", msg.c_str());
      kcmg_destroy(a);
      cudaFree(tr);
      return st;
    }
    ctx->adj = a;
  }
  cudaFree(tr);
  ctx->adj_built = true;
  return KCMG_OK;
}

}  // namespace

extern "C" {

kcmg_status kcmg_solve(kcmg_ctx* ctx, const double* b, double* x, int nrhs, double rtol,
                       double atol, int maxiter, kcmg_info* info) {
  return guarded(ctx, [&]() -> kcmg_status {
    REQUIRE(b && x, "b and x must be non-null");
    REQUIRE(nrhs >= 1 && nrhs <= kMaxRhs, "nrhs must be in [1, %d]", kMaxRhs);
    REQUIRE(rtol >= 0 && atol >= 0 && maxiter >= 0, "negative tolerance or maxiter");
    REQUIRE(nrhs == 1 || !ctx->ir, "batched solves (nrhs > 1) support the FP64 and mixed forms");
    REQUIRE(nrhs == 1 || ctx->p.smoother == 0, "batched solves (nrhs > 1) use the block-Jacobi smoother");
    if (nrhs > 1) return solve_multi(ctx, b, x, nrhs, rtol, atol, maxiter, info);
    return solve_impl(ctx, b, x, rtol, atol, maxiter, info);
  });
}

kcmg_status kcmg_solve_adjoint(kcmg_ctx* ctx, const double* g, double* lambda, int nrhs,
                               double rtol, double atol, int maxiter, kcmg_info* info) {
  return guarded(ctx, [&]() -> kcmg_status {
    REQUIRE(g && lambda, "g and lambda must be non-null");
    REQUIRE(nrhs >= 1 && nrhs <= kMaxRhs, "nrhs must be in [1, %d]", kMaxRhs);
    REQUIRE(rtol >= 0 && atol >= 0 && maxiter >= 0, "negative tolerance or maxiter");
    REQUIRE(nrhs == 1 || !ctx->ir, "batched solves (nrhs > 1) support the FP64 and mixed forms");
    kcmg_status st = ensure_adjoint(ctx);
    if (st != KCMG_OK) return st;
    kcmg_ctx* a = ctx->adj;
    kcmg_status s2 = nrhs > 1 ? solve_multi(a, g, lambda, nrhs, rtol, atol, maxiter, info)
                              : solve_impl(a, g, lambda, rtol, atol, maxiter, info);
    if (a == ctx) return s2;
    if (s2 != KCMG_OK && s2 != KCMG_NOT_CONVERGED) set_err(ctx, "%s", ctx->adj->err.c_str());
    return s2;
  });
}

kcmg_status kcmg_apply(kcmg_ctx* ctx, int level, int op, const double* x, double* y) {
  return guarded(ctx, [&]() -> kcmg_status {
    REQUIRE(level >= 0 && level < ctx->nlev && x && y, "bad level or null vector");
    REQUIRE(op == 0 || (op == 1 && ctx->mixed), "op 1 needs a mixed-precision context");
    Level& L = ctx->lv[level];
    copy_in(ctx, ctx->stage_in, x, L.N);
    EpiArgs none;
    if (op == 0) {
      launch_spmv<double>(ctx->np, ctx->dim, L.A64, L.nbr, L.N, L.G, L.rows_pad, L.block_rows,
                          ctx->stage_in, ctx->stage_out, nullptr, nullptr, none, 0, ctx->s);
    } else {
      float* xi = ctx->lv[0].r_lo;    // FP32 scratch of the finest size
      float* yi = ctx->lv[0].z_lo;     // (the inner-precision operator of the mixed forms)
      launch_convert<double, float>(ctx->stage_in, xi, L.N, ctx->s);
      launch_spmv<float>(ctx->np, ctx->dim, L.A32, L.nbr, L.N, L.G, L.rows_pad, L.block_rows, xi,
                         yi, nullptr, nullptr, none, 0, ctx->s);
      launch_convert<float, double>(yi, ctx->stage_out, L.N, ctx->s);
    }
    CK(cudaGetLastError());
    copy_out(ctx, y, ctx->stage_out, L.N);
    CK(cudaStreamSynchronize(ctx->s));
    return KCMG_OK;
  });
}

kcmg_status kcmg_smooth(kcmg_ctx* ctx, int level, const double* r, double* z) {
  return guarded(ctx, [&]() -> kcmg_status {
    REQUIRE(level >= 0 && level < ctx->nlev - 1 && r && z, "bad level or null vector");
    Level& L = ctx->lv[level];
    load_vec(ctx, level, L.b, r, L.N);
    const void* out;
    if (ctx->ir) {
      Cycle<float, float> cy{ctx};
      out = cy.smooth<float>(level, static_cast<float*>(L.b), ctx->s);
    } else if (ctx->mixed) {
      Cycle<double, float> cy{ctx};
      out = cy.smooth<double>(level, static_cast<double*>(L.b), ctx->s);
    } else {
      Cycle<double, double> cy{ctx};
      out = cy.smooth<double>(level, static_cast<double*>(L.b), ctx->s);
    }
    CK(cudaGetLastError());
    store_vec(ctx, level, z, out, L.N);
    return KCMG_OK;
  });
}

kcmg_status kcmg_restrict(kcmg_ctx* ctx, int level, const double* r, double* rc) {
  return guarded(ctx, [&]() -> kcmg_status {
    REQUIRE(level >= 0 && level < ctx->nlev - 1 && r && rc, "bad level or null vector");
    Level &L = ctx->lv[level], &C = ctx->lv[level + 1];
    load_vec(ctx, level, L.t, r, L.N);
    if (ctx->ir)
      launch_restrict<float, float>(ctx->np, ctx->dim, L.n, C.n, ctx->P32, static_cast<float*>(L.t),
                                    static_cast<float*>(C.b), nullptr, nullptr, nullptr, EpiArgs{}, ctx->s);
    else
      launch_restrict<double, double>(ctx->np, ctx->dim, L.n, C.n, ctx->P64, static_cast<double*>(L.t),
                                      static_cast<double*>(C.b), nullptr, nullptr, nullptr, EpiArgs{}, ctx->s);
    CK(cudaGetLastError());
    store_vec(ctx, level + 1, rc, C.b, C.N);
    return KCMG_OK;
  });
}

kcmg_status kcmg_prolong(kcmg_ctx* ctx, int level, const double* zc, double* z) {
  return guarded(ctx, [&]() -> kcmg_status {
    REQUIRE(level >= 0 && level < ctx->nlev - 1 && zc && z, "bad level or null vector");
    Level &L = ctx->lv[level], &C = ctx->lv[level + 1];
    load_vec(ctx, level + 1, C.x, zc, C.N);
    if (ctx->ir)
      launch_prolong<float, float>(ctx->np, ctx->dim, L.n, C.n, ctx->P32, static_cast<float*>(C.x),
                                   static_cast<float*>(L.t), ctx->s);
    else
      launch_prolong<double, double>(ctx->np, ctx->dim, L.n, C.n, ctx->P64, static_cast<double*>(C.x),
                                     static_cast<double*>(L.t), ctx->s);
    CK(cudaGetLastError());
    store_vec(ctx, level, z, L.t, L.N);
    return KCMG_OK;
  });
}

kcmg_status kcmg_coarse_solve(kcmg_ctx* ctx, const double* r, double* z) {
  return guarded(ctx, [&]() -> kcmg_status {
    REQUIRE(r && z, "null vector");
    copy_in(ctx, ctx->stage_in, r, ctx->Nc);
    launch_coarse_gemv<double>(ctx->Ainv, ctx->Nc, ctx->stage_in, ctx->stage_out, ctx->s);
    CK(cudaGetLastError());
    copy_out(ctx, z, ctx->stage_out, ctx->Nc);
    CK(cudaStreamSynchronize(ctx->s));
    return KCMG_OK;
  });
}

kcmg_status kcmg_get_blocks(kcmg_ctx* ctx, int level, double* out) {
  return guarded(ctx, [&]() -> kcmg_status {
    REQUIRE(level >= 0 && level < ctx->nlev && out, "bad level or null output");
    Level& L = ctx->lv[level];
    copy_out(ctx, out, L.nat, (size_t)ctx->S * L.ncell * ctx->np * ctx->np);
    CK(cudaStreamSynchronize(ctx->s));
    return KCMG_OK;
  });
}

}  // extern "C"

namespace {
template <typename T0, typename T, typename V>
void rm_sequence_impl(kcmg_ctx* ctx, int level, const double* z, int ncorr) {
  Level& L = ctx->lv[level];
  Cycle<T0, T> cy{ctx};
  const V* Aop = level_op<V>(L);
  launch_spmv<V>(ctx->np, ctx->dim, Aop, L.nbr, L.N, L.G, L.rows_pad, L.block_rows,
                 static_cast<V*>(L.x), static_cast<V*>(L.r), static_cast<V*>(L.b), L.partial,
                 cy.epi(level, EPI_MG_BEGIN), 0, ctx->s);
  for (int k = 0; k < ncorr; ++k) {
    load_vec(ctx, level, L.z, z + (size_t)k * L.N, L.N);
    cy.template rm<V>(level, Aop, static_cast<V*>(L.z), 0, 1, ctx->s);
  }
}
}  // namespace

extern "C" {

kcmg_status kcmg_rm_sequence(kcmg_ctx* ctx, int level, const double* b, const double* x0,
                             const double* z, int ncorr, double* x, double* r, int* l) {
  return guarded(ctx, [&]() -> kcmg_status {
    REQUIRE(level >= 0 && level < ctx->nlev - 1 && b && x0 && x && r && l && (ncorr == 0 || z),
            "bad arguments");
    Level& L = ctx->lv[level];
    REQUIRE(ncorr <= L.lcap, "ncorr %d exceeds the basis capacity %d", ncorr, L.lcap);
    init_states(ctx, 0.0, 0.0, 1 << 30);
    load_vec(ctx, level, L.b, b, L.N);
    load_vec(ctx, level, L.x, x0, L.N);
    if (ctx->ir) rm_sequence_impl<float, float, float>(ctx, level, z, ncorr);
    else if (!ctx->mixed) rm_sequence_impl<double, double, double>(ctx, level, z, ncorr);
    else rm_sequence_impl<double, float, double>(ctx, level, z, ncorr);
    CK(cudaGetLastError());
    store_vec(ctx, level, x, L.x, L.N);
    store_vec(ctx, level, r, L.r, L.N);
    LevelState h;
    CK(cudaMemcpyAsync(&h, L.st, sizeof h, cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    *l = h.l;
    return KCMG_OK;
  });
}

kcmg_status kcmg_apply_multi(kcmg_ctx* ctx, int level, int nrhs, const double* x, double* y) {
  return guarded(ctx, [&]() -> kcmg_status {
    REQUIRE(level >= 0 && level < ctx->nlev - 1 && x && y, "bad level or null vector");
    REQUIRE(nrhs >= 2 && nrhs <= kMaxRhs, "nrhs must be in [2, %d]", kMaxRhs);
    REQUIRE(!ctx->ir, "batched calls support the FP64 and mixed forms");
    kcmg_status st = mrhs_ensure(&ctx->mrhs, mrhs_view(ctx), nrhs, &ctx->err);
    if (st != KCMG_OK) return st;
    return mrhs_apply(ctx->mrhs, level, x, y);
  });
}

kcmg_status kcmg_smooth_multi(kcmg_ctx* ctx, int level, int nrhs, const double* r, double* z) {
  return guarded(ctx, [&]() -> kcmg_status {
    REQUIRE(level >= 0 && level < ctx->nlev - 1 && r && z, "bad level or null vector");
    REQUIRE(nrhs >= 2 && nrhs <= kMaxRhs, "nrhs must be in [2, %d]", kMaxRhs);
    REQUIRE(!ctx->ir, "batched calls support the FP64 and mixed forms");
    kcmg_status st = mrhs_ensure(&ctx->mrhs, mrhs_view(ctx), nrhs, &ctx->err);
    if (st != KCMG_OK) return st;
    return mrhs_smooth(ctx->mrhs, level, r, z);
  });
}

kcmg_status kcmg_mrhs_tuning(kcmg_ctx* ctx, double* out, int nout) {
  return guarded(ctx, [&]() -> kcmg_status {
    REQUIRE(out && nout >= 1, "out must hold at least one value");
    for (int i = 0; i < nout; ++i) out[i] = 0.0;
    REQUIRE(ctx->mrhs, "no multi-right-hand-side solve has run on this context");
    mrhs_tuning(ctx->mrhs, out, nout);
    return KCMG_OK;
  });
}

kcmg_status kcmg_kernel_report(kcmg_ctx* ctx, int reps, double* out, int nout) {
  return guarded(ctx, [&]() -> kcmg_status {
    REQUIRE(out && nout >= 7 && reps >= 0, "kcmg_kernel_report needs out[7] and reps >= 0");
    for (int i = 0; i < nout; ++i) out[i] = 0.0;
    if (ctx->coarse_kernel) {
      unsigned long long ns = 0, nl = 0;
      double by = 0;
      CK(cudaMemcpyAsync(&ns, ctx->stat_ns, 8, cudaMemcpyDeviceToHost, ctx->s));
      CK(cudaMemcpyAsync(&nl, ctx->stat_launches, 8, cudaMemcpyDeviceToHost, ctx->s));
      CK(cudaMemcpyAsync(&by, ctx->stat_bytes, 8, cudaMemcpyDeviceToHost, ctx->s));
      unsigned long long lns[KCMG_MAX_LEVELS] = {0};
      CK(cudaMemcpyAsync(lns, ctx->stat_level_ns, sizeof lns, cudaMemcpyDeviceToHost, ctx->s));
      CK(cudaMemsetAsync(ctx->stat_level_ns, 0, sizeof lns, ctx->s));
      unsigned long long pns[kCoarsePhases] = {0};
      CK(cudaMemcpyAsync(pns, ctx->stat_phase_ns, sizeof pns, cudaMemcpyDeviceToHost, ctx->s));
      CK(cudaMemsetAsync(ctx->stat_phase_ns, 0, sizeof pns, ctx->s));
      CK(cudaStreamSynchronize(ctx->s));
      for (int l = 0; l < KCMG_MAX_LEVELS && 7 + l < nout; ++l) out[7 + l] = lns[l] * 1e-6;
      for (int k = 0; k < kCoarsePhases && 7 + KCMG_MAX_LEVELS + k < nout; ++k)
        out[7 + KCMG_MAX_LEVELS + k] = pns[k] * 1e-6;
      CK(cudaMemsetAsync(ctx->stat_ns, 0, 8, ctx->s));
      CK(cudaMemsetAsync(ctx->stat_launches, 0, 8, ctx->s));
      CK(cudaMemsetAsync(ctx->stat_bytes, 0, 8, ctx->s));
      CK(cudaStreamSynchronize(ctx->s));
      out[0] = (double)nl;
      out[1] = ns * 1e-6;
      out[2] = by;
    }
    if (reps > 0) {
      const int S = ctx->S, np = ctx->np;
      cudaEvent_t e0, e1;
      CK(cudaEventCreate(&e0));
      CK(cudaEventCreate(&e1));
      // the operator of a level's residual minimisation (Alg. 1 SpMV: FP64, or FP32 in the
      // inner solve of the iterative-refinement forms) and one full block-Jacobi sweep in
      // the smoother's precision, reps launches each: out[o] ms and out[o + 1] algorithmic
      // bytes per operator launch, out[o + 2], out[o + 3] per sweep
      auto time_level = [&](int lev, int o) {
        Level& L = ctx->lv[lev];
        const size_t vb = ctx->ir ? sizeof(float) : sizeof(double);   // level vector element
        CK(cudaMemsetAsync(L.b, 0, L.N * vb, ctx->s));
        CK(cudaMemsetAsync(L.t, 0, L.N * vb, ctx->s));
        EpiArgs none;
        CK(cudaEventRecord(e0, ctx->s));
        for (int k = 0; k < reps; ++k) {
          if (ctx->ir)
            launch_spmv<float>(np, ctx->dim, L.A32, L.nbr, L.N, L.G, L.rows_pad, L.block_rows,
                               static_cast<float*>(L.t), static_cast<float*>(L.w), nullptr, nullptr, none, 0, ctx->s);
          else
            launch_spmv<double>(np, ctx->dim, L.A64, L.nbr, L.N, L.G, L.rows_pad, L.block_rows,
                                static_cast<double*>(L.t), static_cast<double*>(L.w), nullptr, nullptr, none, 0, ctx->s);
        }
        CK(cudaEventRecord(e1, ctx->s));
        CK(cudaEventSynchronize(e1));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        out[o] = ms / reps;
        out[o + 1] = (double)S * L.N * np * vb + 2.0 * L.N * vb;
        const double sb = ctx->mixed ? 4 : 8;
        const double ib = !ctx->mixed ? 8 : ((L.D16 || ctx->p.precision == KCMG_IR32_BF16INV) ? 2 : 4);
        if (ctx->mixed) {
          CK(cudaMemsetAsync(L.r_lo, 0, L.N * sizeof(float), ctx->s));
          CK(cudaMemsetAsync(L.t_lo, 0, L.N * sizeof(float), ctx->s));
        }
        if (ctx->p.smoother == 1) {
          // one full Schwarz sweep: residual, both partitions' patch solves, combination
          const bool b16 = ctx->p.precision == KCMG_MIXED_BF16INV || ctx->p.precision == KCMG_IR32_BF16INV;
          const int m = (1 << ctx->dim) * np;
          const double npat = (double)as_npatch(L.n, ctx->dim, 0) + as_npatch(L.n, ctx->dim, 1);
          CK(cudaEventRecord(e0, ctx->s));
          for (int k = 0; k < reps; ++k) {
            if (!ctx->mixed) {
              const double *r = static_cast<double*>(L.b), *zo = static_cast<double*>(L.t);
              launch_spmv<double>(np, ctx->dim, L.A64, L.nbr, L.N, L.G, L.rows_pad, L.block_rows, zo,
                                  static_cast<double*>(L.as_r), r, nullptr, EpiArgs{}, 0, ctx->s);
              launch_as_patch<double, double>(np, ctx->dim, L.n, (const double*)L.as_inv0, (const double*)L.as_inv1,
                                              static_cast<double*>(L.as_r), static_cast<double*>(L.as_z), ctx->s);
              launch_as_combine<double>(np, ctx->dim, L.n, L.N, static_cast<double*>(L.as_z), zo,
                                        static_cast<double*>(L.z), ctx->p.omega, 0, ctx->s);
            } else {
              launch_spmv<float>(np, ctx->dim, L.A32, L.nbr, L.N, L.G, L.rows_pad, L.block_rows, L.t_lo,
                                 static_cast<float*>(L.as_r), L.r_lo, nullptr, EpiArgs{}, 0, ctx->s);
              if (b16)
                launch_as_patch<float, __nv_bfloat16>(np, ctx->dim, L.n, (const __nv_bfloat16*)L.as_inv0,
                                                      (const __nv_bfloat16*)L.as_inv1, static_cast<float*>(L.as_r),
                                                      static_cast<float*>(L.as_z), ctx->s);
              else
                launch_as_patch<float, float>(np, ctx->dim, L.n, (const float*)L.as_inv0, (const float*)L.as_inv1,
                                              static_cast<float*>(L.as_r), static_cast<float*>(L.as_z), ctx->s);
              launch_as_combine<float>(np, ctx->dim, L.n, L.N, static_cast<float*>(L.as_z), L.t_lo, L.z_lo,
                                       ctx->p.omega, 0, ctx->s);
            }
          }
          CK(cudaEventRecord(e1, ctx->s));
          CK(cudaEventSynchronize(e1));
          CK(cudaEventElapsedTime(&ms, e0, e1));
          out[o + 2] = ms / reps;
          // operator and r, x, residual; patch inverses and their gathered/solved vectors;
          // the combination reads both patch solutions and x, writes x
          out[o + 3] = (double)S * L.N * np * sb + 3.0 * L.N * sb + npat * m * m * ib + npat * m * 2 * sb +
                       4.0 * L.N * sb;
          return;
        }
        CK(cudaEventRecord(e0, ctx->s));
        for (int k = 0; k < reps; ++k) {
          if (!ctx->mixed)
            launch_bj_sweep<double, double>(np, ctx->dim, L.A64, L.D64, L.nbr, L.N, L.G, L.rows_pad, L.block_rows,
                                            static_cast<double*>(L.b), static_cast<double*>(L.t),
                                            static_cast<double*>(L.z), ctx->p.omega, 0, ctx->s);
          else if (L.mf_nu && L.D16)
            launch_bj_sweep_mf<__nv_bfloat16>(np, ctx->dim, L.n, L.mf_nu, L.mf_F, L.D16, L.N, L.rows_pad,
                                              L.block_rows, L.r_lo, L.t_lo, L.z_lo, ctx->p.omega, 0, ctx->s);
          else if (L.mf_nu)
            launch_bj_sweep_mf<float>(np, ctx->dim, L.n, L.mf_nu, L.mf_F, L.D32, L.N, L.rows_pad, L.block_rows,
                                      L.r_lo, L.t_lo, L.z_lo, ctx->p.omega, 0, ctx->s);
          else if (L.D16)
            launch_bj_sweep<float, __nv_bfloat16>(np, ctx->dim, L.A32, L.D16, L.nbr, L.N, L.G, L.rows_pad,
                                                  L.block_rows, L.r_lo, L.t_lo, L.z_lo, ctx->p.omega, 0, ctx->s);
          else
            launch_bj_sweep<float, float>(np, ctx->dim, L.A32, L.D32, L.nbr, L.N, L.G, L.rows_pad, L.block_rows,
                                          L.r_lo, L.t_lo, L.z_lo, ctx->p.omega, 0, ctx->s);
        }
        CK(cudaEventRecord(e1, ctx->s));
        CK(cudaEventSynchronize(e1));
        CK(cudaEventElapsedTime(&ms, e0, e1));
        out[o + 2] = ms / reps;
        out[o + 3] = L.mf_nu ? (double)L.ncell * 4 + (double)L.N * np * ib + 3.0 * L.N * sb   // coefficient,
                             : (double)(S - 1) * L.N * np * sb + (double)L.N * np * ib + 3.0 * L.N * sb;  // inverses, vectors
      };
      time_level(0, 3);
      const int o1 = 7 + KCMG_MAX_LEVELS + kCoarsePhases;
      if (ctx->nlev > 2 && nout >= o1 + 4) time_level(1, o1);
      // the level-0 Gram kernels of Alg. 1 at the basis length halfway through a restart
      // period: out[o1 + 4] ms and out[o1 + 5] FLOPs of the first Gram pass (W^T w, ||w||^2),
      // out[o1 + 6], out[o1 + 7] of the new column's update (w - W h, z - Z h); out[o1 + 8]
      // the basis length used.  The calls overwrite the level's basis scratch.
      if (nout >= o1 + 9) {
        Level& L = ctx->lv[0];
        const int per = ctx->p.async_smooth > 0 ? ctx->p.async_smooth + 1 : 3;
        const int cap = (ctx->p.lmax > 0 && ctx->p.lmax < L.lcap) ? ctx->p.lmax : L.lcap - per;
        int lt = (cap + per) / 2;
        if (lt > L.lcap - 1) lt = L.lcap - 1;
        if (lt < 1) lt = 1;
        LevelState h;
        CK(cudaMemcpyAsync(&h, L.st, sizeof h, cudaMemcpyDeviceToHost, ctx->s));
        CK(cudaStreamSynchronize(ctx->s));
        h.l = lt;
        h.flags = 0;
        h.ticket = 0;
        CK(cudaMemcpyAsync(L.st, &h, sizeof h, cudaMemcpyHostToDevice, ctx->s));
        const size_t vb = ctx->ir ? sizeof(float) : sizeof(double);
        CK(cudaMemsetAsync(L.w, 0, L.N * vb, ctx->s));
        EpiArgs g1;
        g1.st = L.st;
        g1.kind = EPI_GRAM1;
        g1.h = L.h;
        g1.h2 = L.h2;
        EpiArgs up = g1;
        up.kind = EPI_UPDATE;
        float ms = 0;
        CK(cudaEventRecord(e0, ctx->s));
        for (int k = 0; k < reps; ++k) {
          if (ctx->ir)
            launch_gram_dots<float>(static_cast<float*>(L.W), L.N, static_cast<float*>(L.w), L.lcap, L.nblk,
                                    L.partial, g1, 0, ctx->s);
          else
            launch_gram_dots<double>(static_cast<double*>(L.W), L.N, static_cast<double*>(L.w), L.lcap, L.nblk,
                                     L.partial, g1, 0, ctx->s);
        }
        CK(cudaEventRecord(e1, ctx->s));
        CK(cudaEventSynchronize(e1));
        CK(cudaEventElapsedTime(&ms, e0, e1));
        out[o1 + 4] = ms / reps;
        out[o1 + 5] = 2.0 * (lt + 1) * L.N;
        // the first pass set the flags from zero vectors: clear them for a plain update
        h.flags = 0;
        CK(cudaMemcpyAsync(&L.st->flags, &h.flags, sizeof(int), cudaMemcpyHostToDevice, ctx->s));
        CK(cudaEventRecord(e0, ctx->s));
        for (int k = 0; k < reps; ++k) {
          if (ctx->ir)
            launch_gram_update<float>(static_cast<float*>(L.W), static_cast<float*>(L.Z), L.N,
                                      static_cast<float*>(L.w), static_cast<float*>(L.wre),
                                      static_cast<float*>(L.z), static_cast<float*>(L.r), L.lcap, L.nblk2,
                                      L.partial, up, ctx->s);
          else
            launch_gram_update<double>(static_cast<double*>(L.W), static_cast<double*>(L.Z), L.N,
                                       static_cast<double*>(L.w), static_cast<double*>(L.wre),
                                       static_cast<double*>(L.z), static_cast<double*>(L.r), L.lcap, L.nblk2,
                                       L.partial, up, ctx->s);
        }
        CK(cudaEventRecord(e1, ctx->s));
        CK(cudaEventSynchronize(e1));
        CK(cudaEventElapsedTime(&ms, e0, e1));
        out[o1 + 6] = ms / reps;
        out[o1 + 7] = 4.0 * lt * L.N;
        out[o1 + 8] = lt;
      }
      CK(cudaGetLastError());
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
    }
    return KCMG_OK;
  });
}

kcmg_status kcmg_residual_noalloc(kcmg_ctx* ctx, const double* b, const double* x, double* r,
                                  double* rnorm) {
  return guarded(ctx, [&]() -> kcmg_status {
    REQUIRE(b && x && r && rnorm, "null argument");
    for (const void* p : {(const void*)b, (const void*)x, (const void*)r}) {
      cudaPointerAttributes at;
      const bool dev = cudaPointerGetAttributes(&at, p) == cudaSuccess &&
                       (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
      cudaGetLastError();
      REQUIRE(dev, "kcmg_residual_noalloc: b, x and r must be device memory");
    }
    const Level& L = ctx->lv[0];
    Level0View v{L.A64, L.nbr, L.N, L.G, L.rows_pad, L.block_rows, ctx->np, ctx->dim, ctx->s,
                 ctx->na_scratch};
    // run on the context's device (its scratch address, operator and stream live there)
    int cur = 0;
    CK(cudaGetDevice(&cur));
    if (cur != ctx->dev) CK(cudaSetDevice(ctx->dev));
    int too_large = 0;
    const cudaError_t e = residual_noalloc(v, b, x, r, rnorm, &too_large);
    if (cur != ctx->dev) CK(cudaSetDevice(cur));
    CK(e);
    REQUIRE(!too_large, "kcmg_residual_noalloc: %d rows need more than the 32768 thread blocks "
            "its static scratch holds", L.N);
    return KCMG_OK;
  });
}

kcmg_status kcmg_grad_lognu(kcmg_ctx* ctx, const double* nu, const double* V, const double* F,
                            const double* B, const double* lambda, const double* u, double* g) {
  return guarded(ctx, [&]() -> kcmg_status {
    REQUIRE(nu && V && F && B && lambda && u && g, "null argument");
    Level& L = ctx->lv[0];
    const size_t bs = (size_t)ctx->np * ctx->np;
    const size_t need = L.ncell + bs + 4 * ctx->dim * bs + 2 * ctx->dim * bs + 2 * (size_t)L.N + L.ncell;
    if (ctx->stage_big_len < need) {
      if (ctx->stage_big) cudaFree(ctx->stage_big);
      ctx->stage_big = nullptr;
      CK(cudaMalloc(&ctx->stage_big, need * sizeof(double)));
      ctx->stage_big_len = need;
    }
    double* p = ctx->stage_big;
    double *dnu = p, *dV = dnu + L.ncell, *dF = dV + bs, *dB = dF + 4 * ctx->dim * bs,
           *dl = dB + 2 * ctx->dim * bs, *du = dl + L.N, *dg = du + L.N;
    copy_in(ctx, dnu, nu, L.ncell);
    copy_in(ctx, dV, V, bs);
    copy_in(ctx, dF, F, 4 * ctx->dim * bs);
    copy_in(ctx, dB, B, 2 * ctx->dim * bs);
    copy_in(ctx, dl, lambda, L.N);
    copy_in(ctx, du, u, L.N);
    launch_grad_lognu(ctx->np, ctx->dim, L.n, dnu, dV, dF, dB, dl, du, dg, ctx->s);
    CK(cudaGetLastError());
    copy_out(ctx, g, dg, L.ncell);
    CK(cudaStreamSynchronize(ctx->s));
    return KCMG_OK;
  });
}

}  // extern "C"
