// Internal declarations shared by the kernel and engine translation units of libkcmg.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstddef>
#include <cstdint>
#include <string>

#include "kcmg.h"

namespace kcmg {

// Fixed launch shapes.  Grid sizes of reductions depend only on the vector length, so
// every reduction tree (and therefore every result) is bitwise reproducible.
constexpr int kVecThreads = 256;   // element-wise / dot kernels
constexpr int kDotBlocksMax = 304; // 2 blocks per SM on a 152-SM GB300
constexpr int kMaxNp = 20;
constexpr int kLcapMax = 2048;     // basis capacity cap per level (shared-memory sizing)
constexpr int kMaxChild = 8;

// flags of the RM call in flight
enum : int { F_REORTH = 1, F_DISCARD = 2 };

// Device-resident scalar state of one level of the cycle.  One MG call is active per
// level at any time (Alg. 2 recursion), so one state per level suffices.
struct LevelState {
  int level;
  int l;            // stored basis vectors (columns of W, Z)
  int lcap;         // device capacity of W, Z
  int lmax;         // user restart length (0 = capacity)
  int it, maxit;    // cycles of the current MG call and the cap
  int iters_total;  // cycles summed over visits
  int flags;        // F_REORTH / F_DISCARD of the RM call in flight
  int breakdowns;   // consecutive discarded corrections (level 0)
  int status;       // kcmg_status (level 0)
  int cond;         // loop condition of the while node
  int restart_req;  // restart at the end of this cycle
  int nrestart;
  int hist_len, hist_cap;
  int guard, guard_cap; // loop bodies executed on this level in this solve, and their cap
  int per_cycle;        // corrections appended per cycle (restart when l + per_cycle > cap)
  unsigned int ticket;  // last-block counter of the reduction kernels
  double rnorm, rnorm0, eps, rtol, atol;
  double naz2;      // ||A z||^2 of the RM call in flight
  double gamma, alpha;
  double brk;       // breakdown threshold relative to ||A z||
};

enum EpiKind : int {
  EPI_NONE = 0,
  EPI_MG_BEGIN,     // sum = ||r0||^2: start of an MG call on the level
  EPI_GRAM1,        // sums = W^T w, ||w||^2
  EPI_GRAM2,        // sums = W^T w' (reorthogonalisation pass)
  EPI_UPDATE,       // sums = ||w_hat||^2, w_hat . r
  EPI_FINISH,       // sum = ||r||^2 after the x, r update
  EPI_RESTART,      // sum = ||b - A x||^2: restart of the level
  EPI_NORM          // sum = ||y||^2 stored into *out (component calls, refinement)
};

struct EpiArgs {
  LevelState* st = nullptr;
  int kind = EPI_NONE;
  int end_iter = 0;      // EPI_FINISH: last RM of the cycle
  int hist_type = 0;     // EPI_FINISH: 1 pre, 2 coarse, 3 post
  int use_handle = 0;
  cudaGraphConditionalHandle handle = 0;
  double* h = nullptr;   // Gram coefficients, pass 1 [lcap]
  double* h2 = nullptr;  // Gram coefficients, pass 2 [lcap]
  double* hist = nullptr;
  int* hist_type_buf = nullptr;
  double* out = nullptr; // EPI_NORM destination
};

// ---------------------------------------------------------------- kernel launchers
// All take the stream last; T = double or float (storage and arithmetic type).
// Operator layout ("row-interleaved"): element (s, row, j) of slot s, DOF row
// row = cell*np + i, column j sits at ((s*G + row/32)*JP + j/2)*64 + (row%32)*2 + j%2,
// G = padded rows / 32, JP = ceil(np/2); padded rows and odd-np padding are zero.

template <typename T>
void launch_spmv(int np, int dim, const T* A, const int* nbr, int N, int G, int rows_pad,
                 int block_rows, const T* x, T* y, const T* b, double* partial,
                 const EpiArgs& e, int conditional, cudaStream_t s);
// compensated (double-double accumulated) residual r = b - A x with ||r||^2 and epilogue
void launch_residual_dd(int np, int dim, const double* A, const int* nbr, int N, int G, int rows_pad,
                        int block_rows, const double* x, double* r, const double* b, double* partial,
                        const EpiArgs& e, int conditional, cudaStream_t s);
template <typename T, typename TI>
void launch_bj_sweep(int np, int dim, const T* A, const TI* Dinv, const int* nbr, int N, int G,
                     int rows_pad, int block_rows, const T* r, const T* zold, T* znew,
                     double omega, int first, cudaStream_t s);
// restriction reads the fine residual in TIN (FP64 at level 0 of the mixed form),
// prolongation writes the fine correction in TOUT
template <typename T, typename TIN>
void launch_restrict(int np, int dim, const int* nf, const int* nc, const T* P, const TIN* rf,
                     T* b, T* r, T* x, double* partial, const EpiArgs& e, cudaStream_t s);
template <typename T, typename TOUT>
void launch_prolong(int np, int dim, const int* nf, const int* nc, const T* P, const T* zc,
                    TOUT* zf, cudaStream_t s);
template <typename T>
void launch_coarse_gemv(const double* Ainv, int n, const T* b, T* x, cudaStream_t s);
template <typename T>
void launch_gram_dots(const T* W, int N, const T* w, int lcap, int nblk, double* partial,
                      const EpiArgs& e, int conditional, cudaStream_t s);
template <typename T>
void launch_gram_apply(const T* W, int N, const T* w, T* wout, int lcap, int nblk,
                       LevelState* st, const double* h, cudaStream_t s);
template <typename T>
void launch_gram_update(const T* W, const T* Z, int N, const T* w, const T* wre, const T* z,
                        const T* r, int lcap, int nblk, double* partial, const EpiArgs& e,
                        cudaStream_t s);
template <typename T>
void launch_rm_finish(T* W, T* Z, int N, T* x, T* r, int nblk, double* partial,
                      const EpiArgs& e, cudaStream_t s);
template <typename T>
void launch_norm(const T* v, int N, int nblk, double* partial, const EpiArgs& e,
                 cudaStream_t s);
void launch_control(const EpiArgs& e, cudaStream_t s);  // cond from the current state

// conversions and vector utilities
template <typename Ts, typename Td>
void launch_convert(const Ts* src, Td* dst, size_t n, cudaStream_t s);
template <typename T>
void launch_axpy_to_double(const T* e, double* x, size_t n, cudaStream_t s); // x += e
// iterative refinement: dst = (float)(a * src); x += a * (double)e
void launch_scale_to_float(const double* src, float* dst, double a, size_t n, cudaStream_t s);
void launch_axpy_scaled_to_double(const float* e, double* x, double a, size_t n, cudaStream_t s);

// additive Schwarz smoother on cell patches (schwarz.cu, schwarz.cuh)
cudaError_t launch_patch_inverse(int np, int dim, const double* nat, const int* nbr, const int* n, int part,
                                 double* invT, int* fail, cudaStream_t s);
template <typename T, typename TI>
void launch_as_patch(int np, int dim, const int* n, const TI* inv0, const TI* inv1, const T* r, T* zP,
                     cudaStream_t s);
template <typename T>
void launch_as_combine(int np, int dim, const int* n, int N, const T* zP, const T* xold, T* xnew,
                       double omega, int first, cudaStream_t s);

// matrix-free coupling of the finest level (matfree.cu)
template <typename TI>
void launch_bj_sweep_mf(int np, int dim, const int* n, const float* nu, const float* F, const TI* Dinv, int N,
                        int rows_pad, int block_rows, const float* r, const float* zold, float* znew,
                        double omega, int first, cudaStream_t s);
cudaError_t mf_check(int np, int dim, const int* n, const double* nu, const double* F, const double* nat,
                     double* maxdiff, double* maxabs, cudaStream_t s);

// setup kernels (FP64, natural layout [S][C][np][np])
int launch_galerkin(int np, int dim, const double* Af, const int* nbrf, const int* nf,
                    const int* nc, const double* P, double* Ac, cudaStream_t s);
int launch_block_inverse(int np, const double* diag, int ncell, double* inv, int* fail,
                         cudaStream_t s);
void launch_dense_gj_step(double* M, int n, int c, double* fcol, int* fail, cudaStream_t s);
void launch_assemble_dense(int np, int dim, const double* blk, const int* nbr, int ncell,
                           double* M /*[n][2n]*/, cudaStream_t s);
void launch_extract_inverse(const double* M, int n, double* Ainv, cudaStream_t s);
template <typename T>
void launch_interleave(int np, int nslot, const double* nat, int ncell, int G, T* out,
                       cudaStream_t s);
void launch_transpose_blocks(int np, int dim, const double* in, const int* nbr, int ncell,
                             double* out, cudaStream_t s);
void launch_count_diff(const double* a, const double* b, size_t n, unsigned int* cnt,
                       cudaStream_t s);
void launch_build_nbr(int dim, const int* n, int* nbr, cudaStream_t s);
void launch_grad_lognu(int np, int dim, const int* n, const double* nu, const double* V,
                       const double* F, const double* B, const double* lam, const double* u,
                       double* g, cudaStream_t s);

// ---------------------------------------------------------------- coarse cycle kernel
constexpr int kCoarseMaxCols = 128;   // basis capacity + 1 on the coarse levels
// phase kinds timed inside the persistent coarse cycle (each includes its closing barrier)
enum CoarsePhase : int {
  PH_SWEEP = 0,      // one block-Jacobi sweep
  PH_RM_GRAM1,       // w = A z, W^T w, ||w||^2 and their grid reduction
  PH_RM_REORTH,      // second Gram-Schmidt pass
  PH_RM_UPDATE,      // new basis column, ||w_hat||^2, w_hat . r
  PH_RM_FINISH,      // normalisation, x and r update
  PH_TRANSFER,       // restriction (with ||b_c||) or prolongation
  PH_COARSEST,       // dense solve on the coarsest level
  PH_RESTART,        // r = b - A x on a level restart
  PH_CONTROL,        // level entry and return
  kCoarsePhases
};

struct CoarseLevel {
  const void* A;        // row-interleaved operator of the residual minimisation (vector type)
  const void* As;       // row-interleaved operator of the smoother (its precision)
  const void* Dinv;     // row-interleaved block inverses (smoother precision or BF16)
  void *s0, *s1;        // smoother scratch vectors (smoother precision)
  const int* nbr;
  int n[3];
  int N, G, rows_pad;
  void *x, *r, *b, *z, *t, *w, *wre, *W, *Z;
  int lcap, maxit;
  double rtol;
  LevelState* st;       // iteration/restart counters for the report
  // additive Schwarz smoother: transposed patch inverses of partitions 0 and 1 (stored like
  // Dinv), patch solutions and the sweep's residual (smoother precision)
  const void *as_inv0, *as_inv1;
  void *as_z, *as_r;
};

struct CoarseArgs {
  CoarseLevel lv[KCMG_MAX_LEVELS];
  int lev0, nlev, dim, np;
  const void* P;               // prolongation matrices (FP64; the kernel converts them)
  const double* Ainv;          // dense inverse of the coarsest operator
  int Nc;
  double omega;
  int sweeps, lmax;
  double brk;                  // breakdown threshold of Alg. 1
  double* partial;             // 2 buffers of partial_stride doubles
  size_t partial_stride;       // grid * kCoarseMaxCols
  double* red;                 // kCoarseMaxCols reduced sums
  unsigned int* bar_count;
  unsigned int* bar_gen;
  int* err;                    // set when a grid barrier timed out
  // measurement: launches, device nanoseconds and algorithmic bytes of every launch
  unsigned long long* stat_ns;
  unsigned long long* stat_launches;
  double* stat_bytes;
  unsigned long long* stat_level_ns;   // [KCMG_MAX_LEVELS] time spent on each level
  unsigned long long* stat_phase_ns;   // [kCoarsePhases] time spent in each kind of phase
  int smoother_bytes;          // bytes per element of the smoother operator
  int inverse_bytes;           // bytes per element of the stored block inverses
  int smoother;                // 0 block Jacobi (Alg. BJ), 1 additive Schwarz (Alg. AS)
};

// TV: vectors, bases and the residual minimisation; T: smoother sweeps; TI: stored inverses
template <typename TV, typename T, typename TI>
cudaError_t coarse_cycle_grid(int np, int dim, int threads, int* grid);
template <typename TV, typename T, typename TI>
cudaError_t launch_coarse_cycle(const CoarseArgs& a, int grid, int threads, cudaStream_t s);

// finest-level FP64 operator of a context, for the no-allocation residual (noalloc.cu)
struct Level0View {
  const double* A;
  const int* nbr;
  int N, G, rows_pad, block_rows, np, dim;
  cudaStream_t stream;
  double* scratch;   // device address of the static scratch (from noalloc_prepare)
};
// With device dev current: look up the static scratch's device address (once per device)
// and load the no-allocation kernels.  Called by kcmg_setup.
cudaError_t noalloc_prepare(int dev, double** scratch);
cudaError_t residual_noalloc(const Level0View& v, const double* b, const double* x, double* r,
                             double* rnorm_host, int* too_large);

// ---------------------------------------------------------------- multi-right-hand-side solve
// Batched K-cycle over up to kMaxRhs right-hand sides (mrhs.cu).  Every right-hand side
// keeps its own basis W, Z, coefficients and level criteria; all of them share each
// operator application.  Vectors are [N][R] (right-hand sides fastest).
constexpr int kMaxRhs = 32;

struct MrhsView {               // the context's hierarchy, as the batched solve sees it
  int dim, np, nlev;
  int n[KCMG_MAX_LEVELS][3];
  int ncell[KCMG_MAX_LEVELS], N[KCMG_MAX_LEVELS];
  const double* nat[KCMG_MAX_LEVELS];   // FP64 blocks [S][C][np][np]
  const int* nbr[KCMG_MAX_LEVELS];
  const double* P;                       // [2^dim][np][np]
  const double* Ainv;                    // dense inverse of the coarsest operator
  int Nc;
  double omega;
  int sweeps;
  double lvl_rtol[KCMG_MAX_LEVELS];
  int lvl_maxit[KCMG_MAX_LEVELS];
  int lmax;
  int precision;                         // kcmg_precision
  int tc_tf32_only;                      // single-product TF32 sweeps
  int async_smooth;                      // level 0 as Alg. AsyncMG with this many smoother steps
  cudaStream_t s;
};

struct MrhsEngine;
// Solve A X = B for R = nrhs columns (X holds X0 on entry).  Returns the status; on a
// failure *err receives a message.
kcmg_status mrhs_solve(MrhsEngine** eng, const MrhsView& v, const double* b, double* x, int nrhs,
                       double rtol, double atol, int maxiter, kcmg_info* info, std::string* err);
// Build (or rebuild for another nrhs / precision) the engine without solving.
kcmg_status mrhs_ensure(MrhsEngine** eng, const MrhsView& v, int nrhs, std::string* err);
// Batched component calls on an ensured engine (host or device pointers, [N_level][R]).
kcmg_status mrhs_apply(MrhsEngine* eng, int level, const double* x, double* y);
kcmg_status mrhs_smooth(MrhsEngine* eng, int level, const double* r, double* z);
// Launch shapes the autotuner chose (out[0..nout)), see kcmg_mrhs_tuning.
int mrhs_tuning(const MrhsEngine* eng, double* out, int nout);

// The batched FP32 block-Jacobi sweep on the CUDA cores (mrhs_simt.cu): Ac [C][S][np][np]
// FP32 cell-major blocks, D [C][np][np] inverses, r32 / zo [C np][R] FP32, zn [C np][R];
// wpb warps per block, grid blocks (resident; each warp walks cell groups).
size_t msweep_simt_smem(int np, int dim, bool bf16, int R, int wpb);   // dynamic shared memory per block
int msweep_simt_units(int np, int R, int C);                            // cell groups of a level
int msweep_simt_blocks_per_sm(int np, int dim, bool bf16, int R, int wpb, bool out64);   // resident blocks per SM
cudaError_t msweep_simt_prepare(int np, int dim, int smem_optin);
template <typename TI, typename TOUT>
void launch_msweep_simt(int np, int dim, const float* Ac, const TI* D, const int* nbr, int C, int R,
                        const float* r32, const float* zo, TOUT* zn, float om, int first, int wpb, int grid,
                        cudaStream_t s);
void mrhs_destroy(MrhsEngine* eng);

int block_rows_for(int np);  // threads per block of the operator kernels (whole cells)
bool np_supported(int np, int dim);

}  // namespace kcmg
