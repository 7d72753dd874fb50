/*
 * kcmg.h -- C interface of the GB300 K-cycle orthonormalization multigrid library.
 *
 * The library solves A x = b for a block-sparse operator A with one Np x Np block row per
 * cell of a Cartesian grid (the per-cell local DOF blocks of a DG discretisation, Sec. 2
 * "XDG discretization" of Toprak & Kummer) by the orthonormalization multigrid K-cycle:
 * Alg. 2 (MG) with the residual minimisation Alg. 1 (RM) after every smoother and
 * coarse-grid correction, the damped block-Jacobi smoother of Alg. BJ, the level-local
 * convergence criteria of Sec. 4.2, restriction/prolongation across a 2^d cell-
 * agglomeration hierarchy (Alg. 2, R^lambda and P^lambda) and a direct coarsest solve.
 *
 * Conventions shared by every call:
 *   - Vectors are FP64, length N = ncells * np, DOF index = cell * np + mode; cells are
 *     numbered lexicographically with x fastest.  Multi-right-hand-side vectors are
 *     [N][nrhs] row-major (right-hand sides fastest).
 *   - A pointer argument may be host or device memory (unified addressing tells them
 *     apart); host data is staged through the library's own device buffers, so the
 *     host-pointer path includes the host<->device copies.
 *   - Every call is stream-ordered on the stream given at setup and returns after its
 *     results are complete on that stream (solves synchronise to read their status).
 *   - The caller owns every pointer it passes; the library never frees caller memory.
 *     The library owns everything it allocates until kcmg_destroy.
 *   - Errors are reported through the return value; kcmg_last_error gives a message.
 *     After any status other than KCMG_OK or KCMG_NOT_CONVERGED the output vectors are
 *     unspecified.  On KCMG_NOT_CONVERGED x holds the last iterate, whose true residual
 *     is no larger than that of x0 (Alg. 2 "ENSURE" clause).
 *   - Calls on one context must not overlap (one host thread at a time).
 */
#ifndef KCMG_H
#define KCMG_H

#ifdef __cplusplus
extern "C" {
#endif

#define KCMG_MAX_LEVELS 12

typedef struct kcmg_ctx kcmg_ctx;

typedef enum {
    KCMG_OK = 0,             /* converged to the requested tolerance */
    KCMG_NOT_CONVERGED = 1,  /* maxiter reached; x is the best iterate */
    KCMG_BREAKDOWN = 2,      /* two consecutive level-0 corrections were linearly dependent */
    KCMG_NONFINITE = 3,      /* NaN/Inf in an input or in the iteration */
    KCMG_SINGULAR = 4,       /* a diagonal block or the coarsest operator is singular */
    KCMG_INVALID_ARG = 5,    /* bad sizes, null pointers, unsupported np, ... */
    KCMG_OOM = 6,            /* device allocation failed */
    KCMG_CUDA_ERROR = 7      /* a CUDA runtime call failed */
} kcmg_status;

typedef enum {
    KCMG_FP64 = 0,         /* every kernel in FP64 */
    KCMG_MIXED = 1,        /* block-Jacobi sweeps in FP32 (FP32 operator blocks and
                              inverses, FP32 intermediate iterates) on every level; the
                              residual minimisation (w = A z with the FP64 operator, W, Z,
                              x, r, Gram coefficients), the transfers and the coarsest solve
                              in FP64.  The FP64 minimisation over FP32-computed corrections
                              is the iterative refinement: the attainable residual is
                              FP64's */
    KCMG_MIXED_BF16INV = 2,/* as KCMG_MIXED with the block-Jacobi inverses stored in BF16 */
    KCMG_IR32 = 3,         /* FP64 iterative refinement around an FP32 inner solve.  Outer
                              loop in FP64: r = b - A x with the FP64 operator (compensated
                              sums), stop when ||r|| <= max(rtol ||r0||, atol); otherwise solve
                              A e = r / ||r|| by the K-cycle entirely in FP32 (FP32 operators
                              for w = A z and the sweeps, FP32 transfers, vectors and bases
                              W, Z) with FP64 reductions for the Gram coefficients and norms
                              and the FP64 dense coarsest solve, to ||r_in|| <= ir_inner_rtol;
                              then x += ||r|| e in FP64.  A refinement step that does not
                              lower the FP64 residual is rolled back and ends the solve. */
    KCMG_IR32_BF16INV = 4  /* as KCMG_IR32 with the block-Jacobi inverses stored in BF16 */
} kcmg_precision;

/* Setup input: the fine operator, the hierarchy and the smoother/cycle parameters. */
typedef struct {
    int dim;                 /* 2 or 3 */
    int np;                  /* local DOFs per cell; supported: 3, 4, 6, 10, 20 */
    int n[3];                /* cells per direction (n[2] ignored for dim 2); each divisible
                                by 2^(nlevels-1) */
    int nlevels;             /* >= 2; the last level is solved directly */
    const double *blocks;    /* fine operator, [2*dim+1][ncells][np][np] row-major blocks;
                                slot 0 = diagonal block of the cell, slot 1+2k / 2+2k = the
                                coupling to the -e_k / +e_k face neighbour (zero where the
                                neighbour is outside the grid).  Copied at setup. */
    const double *prolong;   /* [2^dim][np][np]: P_k maps coarse modes to the modes of child
                                k = cx + 2 cy + 4 cz of an agglomerated cell; the same P_k on
                                every level.  R = P^T; coarse operators are P^T A P. */
    double omega;            /* block-Jacobi damping (Alg. BJ) */
    int sweeps;              /* block-Jacobi sweeps per smoother call, from x = 0 */
    double lvl_rtol[KCMG_MAX_LEVELS];  /* levels >= 1: stop when ||r|| <= rtol ||r0||   */
    int lvl_maxit[KCMG_MAX_LEVELS];    /* levels >= 1: ... or after maxit iterations     */
                                       /* (Sec. 4.2: 0.1/20, 0.5/2, then 0/1)           */
    int lmax;                /* restart a level when its basis would exceed lmax vectors
                                (0 = only when the device capacity is reached) */
    int precision;           /* kcmg_precision */
    int use_graph;           /* 1: run the cycle as a CUDA graph with conditional while
                                nodes; 0: host-driven control (reads a flag per loop test) */
    int coarse_persistent;   /* 1: every level below the finest runs in one persistent
                                cooperative kernel per finest-level cycle; 0: one kernel
                                per step (nested loops as conditional graph nodes) */
    int tc_tf32_only;        /* batched solves (nrhs > 1) in the mixed forms: 0 (default) =
                                every block product of the tensor-core sweeps is split into
                                three TF32 products (head*head + head*tail + tail*head,
                                FP32-level accuracy); 1 = a single TF32 product (about 2^-11
                                relative per product; can stall the coarse levels) */
    int async_smooth;        /* 0: level 0 runs Alg. 2 (multiplicative K-cycle).  m > 0:
                                level 0 runs the task-parallel cycle of Alg. AsyncMG with
                                a fixed m: the coarse path (restriction of the cycle-start
                                residual, MG on level 1, prolongation) runs on a second
                                stream while the smoother path applies m smoother + RM
                                steps; one RM with the coarse correction closes the cycle.
                                The level restarts when its basis could not take one more
                                cycle (m + 1 vectors); level 0 holds lmax vectors plus one
                                cycle's corrections.  Batched solves (nrhs > 1) run the same
                                cycle per column, the coarse path first on one stream (it
                                reads only the cycle-start residual, so the iterates are
                                those of the concurrent form).  m in [0, 64]. */
    double ir_inner_rtol;    /* KCMG_IR32*: relative tolerance of every inner FP32 solve
                                (default 1e-3; in (0, 1)) */
    int ir_max_steps;        /* KCMG_IR32*: cap on FP64 refinement steps (default 64) */
    int ir_inner_maxit;      /* KCMG_IR32*: cap on level-0 cycles of one inner solve (default
                                300; the solve's maxiter caps their sum) */
    int smoother;            /* smoother of every iterated level: 0 (default) the block
                                Jacobi of Alg. BJ; 1 the additive Schwarz of Alg. AS on
                                overlapping 2^d-cell patches (Sec. 3.2): the 2^d blocks of two
                                partitions of the cells, one aligned with the agglomeration
                                and one shifted by a cell in every direction, each patch's
                                local matrix inverted densely at setup (in the smoother's
                                precision: FP64, FP32, or BF16 in the *_BF16INV forms);
                                a sweep is x += omega (z_0 + z_1) with z_k the patch solutions
                                of partition k for the residual b - A x.  omega and sweeps
                                as above (0.5 and 2 are typical).  Single right-hand side
                                solves only. */
    const double *mf_nu;     /* optional, with mf_F: the fine operator is the SIPG operator of
                                the cell-wise coefficient mf_nu [ncells] whose off-diagonal
                                blocks are gamma_F F_k^{RL} (slot 1 + 2k) and gamma_F F_k^{LR}
                                (slot 2 + 2k), gamma_F = 2 nu_K nu_J / (nu_K + nu_J), with mf_F
                                [dim][4][np][np] the face reference matrices (LL, LR, RL, RR;
                                the layout of kcmg_grad_lognu).  Setup checks that they
                                reproduce the given blocks (KCMG_INVALID_ARG otherwise); the
                                FP32 block-Jacobi sweeps of level 0 then apply the coupling
                                matrix-free, reading one coefficient per cell instead of six
                                FP32 blocks.  FP32-smoother forms only (mixed and
                                iterative-refinement); NULL = stored blocks.  Copied at setup. */
    const double *mf_F;
} kcmg_params;

/* Fill p with the defaults of Sec. 4.2 / Alg. BJ for the given sizes (blocks, prolong
   must still be set). */
void kcmg_default_params(kcmg_params *p, int dim, int np, const int n[3], int nlevels);

/* Convergence report.  hist/hist_type are caller-owned arrays of length hist_cap (may be
   NULL): ||r|| after every level-0 RM call with type 0 initial, 1 pre-smoother, 2 coarse
   correction, 3 post-smoother, 4 restart (true residual replaces the recursive one); the
   task-parallel cycle records its m smoother RMs as type 1 and its coarse RM as type 2;
   batched solves record instead the active columns at each level-0 loop test (type 5). */
typedef struct {
    int iters;                          /* level-0 cycles */
    int level_iters[KCMG_MAX_LEVELS];   /* cycles per level, summed over visits */
    int restarts;                       /* level-0 restarts */
    int refinements;                    /* mixed forms: FP64 true-residual evaluations on
                                           level 0 (restarts + 1), i.e. refinement steps */
    double res0;                        /* ||b - A x0|| */
    double rel_res;                     /* ||b - A x|| / res0, FP64 true residual */
    long long kernel_launches;          /* kernels launched by the solve (-1: unknown) */
    int hist_cap, hist_len;
    double *hist;
    int *hist_type;
} kcmg_info;

/* Build the hierarchy on the device: copies blocks and prolong, forms the Galerkin
   operators A_{l+1} = P^T A_l P, inverts every diagonal block, inverts the coarsest
   operator densely, and lays out the FP64 (and for mixed precision FP32/BF16) copies
   for the kernels.  cuda_stream: a cudaStream_t (NULL = default stream); every call
   orders the library's own stream after it.  *out receives a context even on failure,
   so that kcmg_last_error can explain the failure: destroy it in every case. */
kcmg_status kcmg_setup(kcmg_ctx **out, const kcmg_params *p, void *cuda_stream);

/* Solve A x = b (Alg. 2 at level 0, or Alg. AsyncMG when async_smooth > 0) until
   ||b - A x|| <= max(rtol ||b - A x0||, atol) or maxiter level-0 cycles.  x: in x0, out x.  info may be NULL.
   nrhs in [1, 32].  With nrhs > 1, b and x are [N][nrhs] (right-hand sides fastest) and
   the columns are solved together: every column runs its own K-cycle (its own bases,
   Gram coefficients and level criteria, Alg. 2 / Alg. 1 per column) while all columns
   share each operator application.  A level's loop runs while any column is active on
   it; a column that is not has its corrections discarded (masked).  Each column stops at
   ||b_j - A x_j|| <= max(rtol ||b_j - A x0_j||, atol), confirmed by a compensated FP64
   true residual.  The batched form is host-driven (use_graph is ignored).  Its level-0
   basis holds lmax vectors per column (default 60 when lmax = 0) plus one cycle's
   corrections, shrunk to what the device can hold.  In the mixed forms the block-Jacobi sweeps run on the tensor cores
   (TF32 products, FP32 accumulation), with launch shapes chosen by an autotuner at the
   first batched solve (see kcmg_mrhs_tuning).  info: iters and level_iters count the
   shared loop; rel_res is the largest relative residual over the columns and res0 the
   largest initial residual; the history records the number of active columns at every
   level-0 loop test (hist_type 5). */
kcmg_status kcmg_solve(kcmg_ctx *ctx, const double *b, double *x, int nrhs, double rtol,
                       double atol, int maxiter, kcmg_info *info);

/* Solve A^T lambda = g with the same cycle on the transposed hierarchy (built at the
   first call; shared with the forward hierarchy when A is bitwise symmetric).  Used for
   the adjoint gradient dL/db = lambda. */
kcmg_status kcmg_solve_adjoint(kcmg_ctx *ctx, const double *g, double *lambda, int nrhs,
                               double rtol, double atol, int maxiter, kcmg_info *info);

/* Adjoint coefficient gradient of the SWIP operator A = sum_K nu_K V + sum_F gamma_F F_F +
   sum_{boundary F} nu_K B_F with gamma_F = 2 nu_K nu_K'/(nu_K + nu_K'):
   g_K = -lambda^T (dA/d log nu_K) u for every cell K.
   nu [ncells]; V [np][np]; F [dim][4][np][np] (interior face, unit gamma: LL, LR, RL, RR,
   L = cell on the low side of the face); B [dim][2][np][np] (boundary face, unit nu: low,
   high face of the cell); lambda, u [N]; g [ncells] out.  Uses the grid of ctx. */
kcmg_status kcmg_grad_lognu(kcmg_ctx *ctx, const double *nu, const double *V, const double *F,
                            const double *B, const double *lambda, const double *u, double *g);

/* ---- component calls (for verification; each runs the same kernels as the solve) ---- */

/* y = A_level x with the FP64 operator (op = 0) or the inner-precision operator (op = 1,
   mixed precision only; inputs/outputs still FP64). */
kcmg_status kcmg_apply(kcmg_ctx *ctx, int level, int op, const double *x, double *y);
/* z = BJ_level(r) from z = 0 (Alg. BJ, omega and sweeps of setup), inner precision. */
kcmg_status kcmg_smooth(kcmg_ctx *ctx, int level, const double *r, double *z);
/* rc = P^T r (level -> level+1) and z = P zc (level+1 -> level), FP64 in every form. */
kcmg_status kcmg_restrict(kcmg_ctx *ctx, int level, const double *r, double *rc);
kcmg_status kcmg_prolong(kcmg_ctx *ctx, int level, const double *zc, double *z);
/* z = A_coarsest^{-1} r (FP64). */
kcmg_status kcmg_coarse_solve(kcmg_ctx *ctx, const double *r, double *z);
/* Galerkin blocks of a level in the setup layout [2d+1][ncells][np][np] (FP64). */
kcmg_status kcmg_get_blocks(kcmg_ctx *ctx, int level, double *out);
/* Alg. 1 on a level in the inner precision: start from x0 (r0 = b - A x0, empty basis),
   then apply RM to the corrections z[0..ncorr) ([ncorr][N_level]) in turn.  Returns the
   final x and r (recursive residual) and the basis size in *l. */
kcmg_status kcmg_rm_sequence(kcmg_ctx *ctx, int level, const double *b, const double *x0,
                             const double *z, int ncorr, double *x, double *r, int *l);

/* Measurement support (no counterpart in the paper).  out[0..2]: launches, total device
   milliseconds (GPU global timer, entry to last barrier) and algorithmic bytes (unique
   operator and vector bytes of every phase) of the persistent coarse-cycle kernel since
   the previous call; the counters are then reset.  If reps > 0 also times, with CUDA events
   on the library's stream, reps launches each of the level-0 FP64 operator application
   (out[3] ms per launch, out[4] algorithmic bytes) and of one full block-Jacobi sweep in
   the smoother's precision (out[5] ms, out[6] bytes).  out[7 + l] (if nout allows): device
   milliseconds the coarse-cycle kernel spent on level l (the coarsest: its direct solves).
   out[19 + k] (if nout allows): milliseconds it spent in phases of kind k, each with its
   closing grid barrier: 0 block-Jacobi sweep, 1 w = A z with the first Gram pass and its
   reduction, 2 second Gram pass, 3 new basis column with its norms, 4 normalisation and
   x, r update, 5 restriction or prolongation, 6 coarsest solve, 7 restart residual,
   8 level entry and return.  out[28..31] (if nout allows, reps > 0 and level 1 is iterated):
   the same four timings as out[3..6] on level 1.  out[32..36] (if nout allows, reps > 0):
   the level-0 Gram kernels of Alg. 1 at the basis length halfway through a restart period:
   ms and FLOPs of the first Gram pass, ms and FLOPs of the update of the new column, and
   the basis length used (these calls overwrite the basis; the next solve starts afresh).
   nout >= 7. */
kcmg_status kcmg_kernel_report(kcmg_ctx *ctx, int reps, double *out, int nout);

/* r = b - A x with the finest-level FP64 operator, and *rnorm = ||r|| (a host double),
   for callers that must not allocate device memory: processes whose device memory is
   already claimed (for example by a framework's caching allocator that holds most of the
   free memory, where a cudaMalloc fails or forces the framework to release its cache),
   code running under a fixed device-memory budget, and error-recovery paths after an
   out-of-memory failure.  The paper has no counterpart; this is a service of the library.
   b, x, r: device pointers of length N (anything else returns KCMG_INVALID_ARG).
   The call allocates nothing: its reduction scratch is a static device array of 257 KB,
   present on every GPU that loads the library until the process exits.  It handles up to
   32768 thread blocks (up to 10,485,760 rows at np = 10 or 20, 9,437,184 at np = 3 or 6,
   8,388,608 at np = 4); larger problems return KCMG_INVALID_ARG.  kcmg_setup looks up the
   scratch's device address (cudaGetSymbolAddress, with the context's device current) and
   loads the call's kernels, so the call does no set-up of its own; the call runs on the
   context's device (it makes that device current for its duration).  All calls share the
   scratch and it keeps the last call's contents (the reduction counter is cleared at every
   call): calls that overlap on the GPU (other streams, other host threads, other contexts
   on the same device) race and must not be issued.  Stream-ordered on the context's
   stream; it copies ||r|| to host memory and synchronises that stream before returning. */
kcmg_status kcmg_residual_noalloc(kcmg_ctx *ctx, const double *b, const double *x, double *r,
                                  double *rnorm);

/* Batched component calls (right-hand sides fastest, [N_level][nrhs], nrhs in [2, 32],
   level in [0, nlevels-2]); they run the kernels of the batched solve:
   Y = A_level X with the FP64 operator, and Z = BJ_level(R) from Z = 0 (Alg. BJ, omega and
   sweeps of setup) in the context's precision (mixed forms: the FP32 sweep kernel the
   autotuner chose, see kcmg_mrhs_tuning). */
kcmg_status kcmg_apply_multi(kcmg_ctx *ctx, int level, int nrhs, const double *x, double *y);
kcmg_status kcmg_smooth_multi(kcmg_ctx *ctx, int level, int nrhs, const double *r, double *z);

/* Launch shapes the multi-right-hand-side autotuner chose at the first batched solve of
   ctx: out[0] warps per block of the FP64 block SpMM, out[1] its time (ms), out[2] warps
   per block of the FP32 sweep, out[3] its grid (0 = one warp per cell), out[4] its
   time (ms), out[5] level-0 basis capacity per column, out[6] nrhs, out[7] 1 if the
   tensor-core sweeps split each product into three TF32 products (tc_tf32_only = 0),
   out[8] the level-0 sweep kernel, the fastest of three: 0 = tensor cores (one warp per
   cell), 1 = tensor cores with each cell's blocks, inverse, r and neighbour slabs staged
   by double-buffered 1-D bulk copies, 2 = FP32 CUDA cores (register-blocked; exact FP32
   products).  The environment variable KCMG_SWEEP = tc | tcb | simt, read at the first
   batched solve, forces one kernel on every level.  Zero-filled up to nout. */
kcmg_status kcmg_mrhs_tuning(kcmg_ctx *ctx, double *out, int nout);

/* Level sizes: number of cells of a level (0 if out of range). */
int kcmg_level_cells(const kcmg_ctx *ctx, int level);

const char *kcmg_last_error(const kcmg_ctx *ctx);
const char *kcmg_status_string(kcmg_status s);
void kcmg_destroy(kcmg_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* KCMG_H */
