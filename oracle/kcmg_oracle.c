/*
 * kcmg_oracle.c -- plain, slow, obviously-correct FP64 CPU reference of the K-cycle
 * orthonormalization multigrid (OrthoMG) solve of Toprak & Kummer, "A Task Parallel
 * Orthonormalization Multigrid Method for Multiphase Elliptic Problems".
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call this
 * file; it is used by the tests, by the smoke check and by the benchmark's CPU-baseline
 * leg.  It shares no code, header, table or helper with the CUDA library.
 *
 * What it follows:
 *   rm_step     Alg. 1 (residual minimization): w = A z; modified Gram-Schmidt of w against
 *               the stored orthonormal W with the same coefficients applied to z against Z;
 *               normalise; append; alpha_{l+1} = w_{l+1} . r0; x = x0 + Z alpha;
 *               r = r0 - W alpha.
 *   mg          Alg. 2 (orthonormalization multigrid, multiplicative K-cycle): while
 *               ||r|| > eps: pre-smoother, RM, restrict, recursive MG or direct solve on the
 *               next level, prolongate, RM, post-smoother, RM.
 *   smooth      Alg. BJ (block Jacobi) started from x = 0 with a fixed sweep count:
 *               r = b - A x; x_i += omega A_ii^{-1} r_i for every cell block i.
 *   smooth_as   Alg. AS (additive Schwarz, Sec. 3.2) on overlapping cell patches, from x = 0
 *               with a fixed sweep count: r = b - A x; x += omega sum_i P_i A_i^{-1} R_i r over
 *               the patches i of two partitions of the grid into 2^d-cell blocks (one
 *               aligned with the agglomeration, one shifted by a cell in every direction),
 *               A_i = R_i A P_i inverted densely.
 *   async_mg0   Alg. AsyncMG (task-parallel OrthoMG) on level 0, with the smoother group's
 *               loop run a fixed number m of times per cycle so that the result does not
 *               depend on timing: per cycle the coarse path restricts the residual of the
 *               cycle start, solves the coarse problem (recursive MG, or directly) and
 *               prolongates; the smoother path applies m smoother + RM steps to the
 *               current residual meanwhile; then one RM with the coarse correction.
 *   criteria    Sec. 4.2 (convergence criteria): level 0 the user tolerance; level 1
 *               ||r|| <= 0.1 ||r0|| or 20 iterations; level 2 ||r|| <= 0.5 ||r0|| or 2
 *               iterations; deeper levels one iteration per visit; the last level of the
 *               hierarchy is solved directly.
 * Readings where the paper is silent:
 *   - R = P^T, A_{l+1} = P^T A_l P (Galerkin) with P the exact injection of nested
 *     polynomial spaces (given as 2^d constant child matrices);
 *   - a second MGS pass when the orthogonalised norm drops below half of ||A z||;
 *   - a correction whose orthogonalised norm is <= 1e-14 ||A z|| (or not finite) is
 *     discarded (no append, no update);
 *   - the coarsest system is solved with a dense LU factorisation (partial pivoting);
 *   - restart: Alg. 2 never clears W, Z inside one call, and in floating point the
 *     recursive residual r = r0 - W alpha drifts from b - A x as A Z = W degrades with
 *     the basis length.  At the end of a cycle whose basis could not take another three
 *     vectors within lmax (lmax > 0: l + 3 > lmax), and on level 0 whenever the recursive
 *     residual meets the tolerance, the level restarts: x0 := x, r0 := b - A x (true
 *     residual), W, Z := {}.  The true residual stays monotone; the top-level stopping
 *     test is taken on it.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Loops over cells or over vector elements whose every output element is computed by the
   same sequential arithmetic whichever thread runs it.  Built with -fopenmp they run on
   all host cores and give bitwise the results of the serial build; every sum over
   elements (dot products, the restriction's accumulation into a coarse cell) stays
   sequential. */
#ifdef _OPENMP
#define ORC_PARALLEL_FOR _Pragma("omp parallel for schedule(static)")
#else
#define ORC_PARALLEL_FOR
#endif

#define ORC_MAXLEV 16

enum { ORC_OK = 0, ORC_NOT_CONVERGED = 1, ORC_BREAKDOWN = 2, ORC_NONFINITE = 3,
       ORC_SINGULAR = 4, ORC_INVALID_ARG = 5 };

typedef struct {
    int n[3];        /* cells per direction (n[2] = 1 in 2-D) */
    int ncell;
    int *nbr;        /* [ncell][2*dim]: -e0, +e0, -e1, +e1, -e2, +e2; -1 = none */
    double *blk;     /* [ncell][S][np][np], slot 0 = diagonal, slot s>0 = nbr[s-1] */
    double *inv;     /* [ncell][np][np] inverse of the diagonal block */
    /* per-level Alg. 2 state */
    int lcap, l;
    double *W, *Z;   /* [lcap][N] stored orthonormal basis and its search directions */
    /* Alg. AS patches: partition 0 = aligned 2^d blocks, 1 = shifted by one cell */
    int npatch[2];
    int *pcell[2];   /* [npatch][2^d] member cells, -1 = outside the grid */
    double *pinv[2]; /* [npatch][m][m] inverse of the local matrix, m = 2^d np */
    double *alpha;   /* [lcap] */
    double *x0, *r0, *x, *r, *z, *w, *t, *bc, *xc;
} olevel;

typedef struct {
    int dim, np, S, nlev, nchild;
    olevel lv[ORC_MAXLEV];
    double *P;       /* [nchild][np][np] */
    double omega;
    int sweeps;
    double lvl_rtol[ORC_MAXLEV];
    int lvl_maxit[ORC_MAXLEV];
    int Nc;
    double *Lc;      /* [Nc][Nc] packed LU factors of the coarsest operator */
    int *piv;        /* [Nc] row interchanges of the LU factorisation */
    /* solve bookkeeping */
    double *hist; int *hist_type; int hist_cap, hist_len;
    int level_iters[ORC_MAXLEV];
    int breakdowns_in_row, status_flag;
    int lmax, restarts;
    int async_m;     /* 0: Alg. 2 on level 0; m > 0: Alg. AsyncMG with m smoother steps */
    int smoother;    /* 0: Alg. BJ (block Jacobi); 1: Alg. AS (additive Schwarz, patches) */
    double res0;     /* ||b - A x0|| of the top-level solve */
} osolver;

static double dot(int n, const double *a, const double *b) {
    double s = 0.0;
    for (int i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

static int ndof(const osolver *S, int lev) { return S->lv[lev].ncell * S->np; }
static int invert_block(int n, const double *A, double *Ainv);

/* y = A x on level lev (block row K: sum over slots of blk[K][s] x[nbr]) */
static void apply(const osolver *S, int lev, const double *x, double *y) {
    const olevel *L = &S->lv[lev];
    int np = S->np, nf = 2 * S->dim;
    ORC_PARALLEL_FOR
    for (int K = 0; K < L->ncell; K++) {
        for (int i = 0; i < np; i++) {
            double s = 0.0;
            for (int sl = 0; sl < S->S; sl++) {
                int J = (sl == 0) ? K : L->nbr[K * nf + sl - 1];
                if (J < 0) continue;
                const double *B = L->blk + ((size_t)K * S->S + sl) * np * np;
                for (int j = 0; j < np; j++) s += B[i * np + j] * x[(size_t)J * np + j];
            }
            y[(size_t)K * np + i] = s;
        }
    }
}

/* Alg. BJ from x^(0) = 0 with S->sweeps iterations (no norm test inside MG). */
static void smooth_bj(osolver *S, int lev, const double *b, double *x) {
    olevel *L = &S->lv[lev];
    int np = S->np, N = ndof(S, lev);
    double *r = L->t;
    for (int i = 0; i < N; i++) x[i] = 0.0;
    for (int k = 0; k < S->sweeps; k++) {
        apply(S, lev, x, r);
        ORC_PARALLEL_FOR
        for (int i = 0; i < N; i++) r[i] = b[i] - r[i];
        ORC_PARALLEL_FOR
        for (int K = 0; K < L->ncell; K++) {
            const double *D = L->inv + (size_t)K * np * np;
            for (int i = 0; i < np; i++) {
                double dx = 0.0;
                for (int j = 0; j < np; j++) dx += D[i * np + j] * r[(size_t)K * np + j];
                x[(size_t)K * np + i] += S->omega * dx;
            }
        }
    }
}

/* Alg. AS from x^(0) = 0 with S->sweeps iterations: each iteration forms the global
   residual r = b - A x, restricts it to every patch of both partitions, solves the local
   problems A_i z_i = R_i r with the stored inverses, and adds omega times the sum of the
   prolongated z_i to x.  The patches of one partition are disjoint, so every cell gets one
   contribution per partition; partition 0 is added first. */
static void smooth_as(osolver *S, int lev, const double *b, double *x) {
    olevel *L = &S->lv[lev];
    int np = S->np, N = ndof(S, lev), nc = S->nchild, m = nc * np;
    double *r = L->t;
    double *e = malloc(sizeof(double) * N);
    for (int i = 0; i < N; i++) x[i] = 0.0;
    for (int k = 0; k < S->sweeps; k++) {
        apply(S, lev, x, r);
        ORC_PARALLEL_FOR
        for (int i = 0; i < N; i++) r[i] = b[i] - r[i];
        for (int i = 0; i < N; i++) e[i] = 0.0;
        for (int part = 0; part < 2; part++) {
            ORC_PARALLEL_FOR
            for (int pi = 0; pi < L->npatch[part]; pi++) {
                const int *cells = L->pcell[part] + (size_t)pi * nc;
                const double *Ainv = L->pinv[part] + (size_t)pi * m * m;
                double rl[8 * 32];                            /* m <= 8 * 32 */
                for (int a = 0; a < nc; a++)
                    for (int q = 0; q < np; q++)
                        rl[a * np + q] = cells[a] >= 0 ? r[(size_t)cells[a] * np + q] : 0.0;
                for (int a = 0; a < nc; a++) {
                    if (cells[a] < 0) continue;
                    for (int q = 0; q < np; q++) {
                        double z = 0.0;
                        for (int j = 0; j < m; j++) z += Ainv[(size_t)(a * np + q) * m + j] * rl[j];
                        e[(size_t)cells[a] * np + q] += z;
                    }
                }
            }
        }
        ORC_PARALLEL_FOR
        for (int i = 0; i < N; i++) x[i] += S->omega * e[i];
    }
    free(e);
}

static void smooth(osolver *S, int lev, const double *b, double *x) {
    if (S->smoother == 1) smooth_as(S, lev, b, x);
    else smooth_bj(S, lev, b, x);
}

/* The patches of partition part (0: aligned, 1: shifted by one cell) on level lev and the
   inverses of their local matrices A_i = R_i A P_i: member a = cx + 2 cy + 4 cz of patch
   (px, py, pz) is the cell (2 px - part + cx, ...) if it lies in the grid.  The local matrix
   holds the blocks of A that couple two members (slot 0 on the diagonal, the face slot
   towards a neighbour member elsewhere); an absent member gets an identity block and no
   coupling, so its row of the solve is zero for a zero right-hand side.  Returns 0, or 1
   if a local matrix is singular. */
static int build_patches(osolver *S, int lev, int part) {
    olevel *L = &S->lv[lev];
    int np = S->np, nc = S->nchild, m = nc * np, nf = 2 * S->dim;
    int pn[3] = {1, 1, 1};
    for (int j = 0; j < S->dim; j++) pn[j] = L->n[j] / 2 + part;
    int npatch = pn[0] * pn[1] * pn[2];
    L->npatch[part] = npatch;
    L->pcell[part] = malloc(sizeof(int) * npatch * nc);
    L->pinv[part] = malloc(sizeof(double) * (size_t)npatch * m * m);
    double *M = malloc(sizeof(double) * m * m);
    for (int pi = 0; pi < npatch; pi++) {
        int pc[3] = {pi % pn[0], (pi / pn[0]) % pn[1], pi / (pn[0] * pn[1])};
        int *cells = L->pcell[part] + (size_t)pi * nc;
        for (int a = 0; a < nc; a++) {
            int c[3] = {0, 0, 0}, inside = 1;
            for (int j = 0; j < S->dim; j++) {
                c[j] = 2 * pc[j] - part + ((a >> j) & 1);
                if (c[j] < 0 || c[j] >= L->n[j]) inside = 0;
            }
            cells[a] = inside ? c[0] + L->n[0] * (c[1] + L->n[1] * c[2]) : -1;
        }
        for (int i = 0; i < m * m; i++) M[i] = 0.0;
        for (int a = 0; a < nc; a++) {
            if (cells[a] < 0) {
                for (int q = 0; q < np; q++) M[(size_t)(a * np + q) * m + a * np + q] = 1.0;
                continue;
            }
            for (int b = 0; b < nc; b++) {
                if (cells[b] < 0) continue;
                int slot = -1;
                if (b == a) slot = 0;
                else
                    for (int s = 1; s <= nf; s++)
                        if (L->nbr[cells[a] * nf + s - 1] == cells[b]) slot = s;
                if (slot < 0) continue;
                const double *B = L->blk + ((size_t)cells[a] * S->S + slot) * np * np;
                for (int q = 0; q < np; q++)
                    for (int t = 0; t < np; t++) M[(size_t)(a * np + q) * m + b * np + t] = B[q * np + t];
            }
        }
        if (invert_block(m, M, L->pinv[part] + (size_t)pi * m * m)) { free(M); return 1; }
    }
    free(M);
    return 0;
}

/* child index and parent of fine cell K on level lev */
static void cell_coords(const olevel *L, int K, int c[3]) {
    c[0] = K % L->n[0];
    c[1] = (K / L->n[0]) % L->n[1];
    c[2] = K / (L->n[0] * L->n[1]);
}
static int parent_of(const osolver *S, int lev, int K, int *child) {
    int c[3];
    cell_coords(&S->lv[lev], K, c);
    const olevel *C = &S->lv[lev + 1];
    int k = 0;
    for (int j = 0; j < S->dim; j++) k |= (c[j] & 1) << j;
    *child = k;
    int pc[3] = {c[0] / 2, c[1] / 2, S->dim == 3 ? c[2] / 2 : 0};
    return pc[0] + C->n[0] * (pc[1] + C->n[1] * pc[2]);
}

/* r_c = P^T r : coarse cell J gets sum over children k of P_k^T r[child] */
static void restrict_(const osolver *S, int lev, const double *rf, double *rc) {
    int np = S->np;
    memset(rc, 0, sizeof(double) * ndof(S, lev + 1));
    for (int K = 0; K < S->lv[lev].ncell; K++) {
        int k, J = parent_of(S, lev, K, &k);
        const double *Pk = S->P + (size_t)k * np * np;
        for (int i = 0; i < np; i++) {
            double s = 0.0;
            for (int a = 0; a < np; a++) s += Pk[a * np + i] * rf[(size_t)K * np + a];
            rc[(size_t)J * np + i] += s;
        }
    }
}

/* z = P z_c : child k of coarse cell J gets P_k z_c[J] */
static void prolong(const osolver *S, int lev, const double *zc, double *zf) {
    int np = S->np;
    ORC_PARALLEL_FOR
    for (int K = 0; K < S->lv[lev].ncell; K++) {
        int k, J = parent_of(S, lev, K, &k);
        const double *Pk = S->P + (size_t)k * np * np;
        for (int a = 0; a < np; a++) {
            double s = 0.0;
            for (int i = 0; i < np; i++) s += Pk[a * np + i] * zc[(size_t)J * np + i];
            zf[(size_t)K * np + a] = s;
        }
    }
}

/* Gauss-Jordan inverse with partial pivoting of an np x np block; 0 on success */
static int invert_block(int n, const double *A, double *Ainv) {
    double *M = malloc(sizeof(double) * n * 2 * n);
    for (int i = 0; i < n; i++)
        for (int j = 0; j < 2 * n; j++)
            M[i * 2 * n + j] = (j < n) ? A[i * n + j] : (j - n == i ? 1.0 : 0.0);
    for (int c = 0; c < n; c++) {
        int piv = c;
        for (int i = c + 1; i < n; i++)
            if (fabs(M[i * 2 * n + c]) > fabs(M[piv * 2 * n + c])) piv = i;
        if (M[piv * 2 * n + c] == 0.0) { free(M); return 1; }
        if (piv != c)
            for (int j = 0; j < 2 * n; j++) {
                double t = M[c * 2 * n + j]; M[c * 2 * n + j] = M[piv * 2 * n + j]; M[piv * 2 * n + j] = t;
            }
        double d = M[c * 2 * n + c];
        for (int j = 0; j < 2 * n; j++) M[c * 2 * n + j] /= d;
        for (int i = 0; i < n; i++) {
            if (i == c) continue;
            double f = M[i * 2 * n + c];
            for (int j = 0; j < 2 * n; j++) M[i * 2 * n + j] -= f * M[c * 2 * n + j];
        }
    }
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) Ainv[i * n + j] = M[i * 2 * n + n + j];
    free(M);
    return 0;
}

/* Galerkin coarse operator A_{lev+1} = P^T A_lev P, formed block by block */
static void galerkin(osolver *S, int lev) {
    olevel *F = &S->lv[lev], *C = &S->lv[lev + 1];
    int np = S->np, nf = 2 * S->dim, Sl = S->S;
    size_t bs = (size_t)np * np;
    C->blk = calloc((size_t)C->ncell * Sl * bs, sizeof(double));
    double *tmp = malloc(sizeof(double) * bs);
    for (int K = 0; K < F->ncell; K++) {
        int k, J = parent_of(S, lev, K, &k);
        for (int sl = 0; sl < Sl; sl++) {
            int K2 = (sl == 0) ? K : F->nbr[K * nf + sl - 1];
            if (K2 < 0) continue;
            int k2, J2 = parent_of(S, lev, K2, &k2);
            int cs = (J2 == J) ? 0 : sl;   /* crossing a coarse face keeps the direction */
            const double *Ab = F->blk + ((size_t)K * Sl + sl) * bs;
            const double *Pk = S->P + (size_t)k * bs, *Pk2 = S->P + (size_t)k2 * bs;
            /* tmp = A_b P_k2 ; C[J][cs] += P_k^T tmp */
            for (int a = 0; a < np; a++)
                for (int j = 0; j < np; j++) {
                    double s = 0.0;
                    for (int m = 0; m < np; m++) s += Ab[a * np + m] * Pk2[m * np + j];
                    tmp[a * np + j] = s;
                }
            double *Cb = C->blk + ((size_t)J * Sl + cs) * bs;
            for (int i = 0; i < np; i++)
                for (int j = 0; j < np; j++) {
                    double s = 0.0;
                    for (int a = 0; a < np; a++) s += Pk[a * np + i] * tmp[a * np + j];
                    Cb[i * np + j] += s;
                }
        }
    }
    free(tmp);
}

static void build_nbr(osolver *S, olevel *L) {
    int nf = 2 * S->dim;
    L->nbr = malloc(sizeof(int) * L->ncell * nf);
    for (int K = 0; K < L->ncell; K++) {
        int c[3];
        cell_coords(L, K, c);
        int stride[3] = {1, L->n[0], L->n[0] * L->n[1]};
        for (int j = 0; j < S->dim; j++) {
            L->nbr[K * nf + 2 * j] = (c[j] > 0) ? K - stride[j] : -1;
            L->nbr[K * nf + 2 * j + 1] = (c[j] < L->n[j] - 1) ? K + stride[j] : -1;
        }
    }
}

static void alloc_work(osolver *S, olevel *L) {
    size_t N = (size_t)L->ncell * S->np;
    double **v[] = {&L->x0, &L->r0, &L->x, &L->r, &L->z, &L->w, &L->t, &L->bc, &L->xc};
    for (int i = 0; i < 9; i++) *v[i] = calloc(N, sizeof(double));
    L->lcap = 0; L->l = 0; L->W = L->Z = L->alpha = NULL;
}

/* dense LU factorisation with partial pivoting, P A = L U, of the coarsest operator
   (A^T for the adjoint solver is not symmetric in general); 0 on success */
static int coarse_factor(osolver *S) {
    olevel *L = &S->lv[S->nlev - 1];
    int np = S->np, nf = 2 * S->dim, n = L->ncell * np;
    S->Nc = n;
    double *A = calloc((size_t)n * n, sizeof(double));
    S->piv = malloc(sizeof(int) * n);
    for (int K = 0; K < L->ncell; K++)
        for (int sl = 0; sl < S->S; sl++) {
            int J = (sl == 0) ? K : L->nbr[K * nf + sl - 1];
            if (J < 0) continue;
            const double *B = L->blk + ((size_t)K * S->S + sl) * np * np;
            for (int i = 0; i < np; i++)
                for (int j = 0; j < np; j++) A[(size_t)(K * np + i) * n + J * np + j] += B[i * np + j];
        }
    S->Lc = A;
    for (int c = 0; c < n; c++) {
        int p = c;
        for (int i = c + 1; i < n; i++)
            if (fabs(A[(size_t)i * n + c]) > fabs(A[(size_t)p * n + c])) p = i;
        S->piv[c] = p;
        if (A[(size_t)p * n + c] == 0.0) return 1;
        if (p != c)
            for (int j = 0; j < n; j++) {
                double t = A[(size_t)c * n + j]; A[(size_t)c * n + j] = A[(size_t)p * n + j]; A[(size_t)p * n + j] = t;
            }
        for (int i = c + 1; i < n; i++) {
            double f = A[(size_t)i * n + c] / A[(size_t)c * n + c];
            A[(size_t)i * n + c] = f;
            for (int j = c + 1; j < n; j++) A[(size_t)i * n + j] -= f * A[(size_t)c * n + j];
        }
    }
    return 0;
}

static void coarse_solve(const osolver *S, const double *r, double *z) {
    int n = S->Nc;
    const double *A = S->Lc;
    for (int i = 0; i < n; i++) z[i] = r[i];
    for (int c = 0; c < n; c++)                             /* apply the row swaps */
        if (S->piv[c] != c) { double t = z[c]; z[c] = z[S->piv[c]]; z[S->piv[c]] = t; }
    for (int i = 0; i < n; i++)                             /* L y = P r (unit diagonal) */
        for (int k = 0; k < i; k++) z[i] -= A[(size_t)i * n + k] * z[k];
    for (int i = n - 1; i >= 0; i--) {                      /* U z = y */
        for (int k = i + 1; k < n; k++) z[i] -= A[(size_t)i * n + k] * z[k];
        z[i] /= A[(size_t)i * n + i];
    }
}

/* ------------------------------------------------------------------------ Alg. 1 */
static void ensure_cap(osolver *S, olevel *L) {
    if (L->l < L->lcap) return;
    size_t N = (size_t)L->ncell * S->np;
    int nc = L->lcap ? 2 * L->lcap : 16;
    L->W = realloc(L->W, sizeof(double) * N * nc);
    L->Z = realloc(L->Z, sizeof(double) * N * nc);
    L->alpha = realloc(L->alpha, sizeof(double) * nc);
    L->lcap = nc;
}

/* RM(A, r0, z, W, Z) on level lev; z is overwritten.  Returns 0 if the correction was
   appended, 1 if it was discarded (breakdown), 2 if a non-finite value appeared. */
static int rm_step(osolver *S, int lev, double *z) {
    olevel *L = &S->lv[lev];
    int N = ndof(S, lev);
    double *w = L->w;
    apply(S, lev, z, w);                                   /* w_{l+1} := A z */
    double naz = sqrt(dot(N, w, w));
    if (!isfinite(naz)) return 2;
    for (int pass = 0; pass < 2; pass++) {
        double before = (pass == 0) ? naz : sqrt(dot(N, w, w));
        for (int i = 0; i < L->l; i++) {                   /* for all columns w_i of W */
            const double *Wi = L->W + (size_t)i * N, *Zi = L->Z + (size_t)i * N;
            double beta = dot(N, Wi, w);                   /* beta := w_i . w_{l+1} */
            ORC_PARALLEL_FOR
            for (int k = 0; k < N; k++) w[k] -= beta * Wi[k];
            ORC_PARALLEL_FOR
            for (int k = 0; k < N; k++) z[k] -= beta * Zi[k];
        }
        if (sqrt(dot(N, w, w)) >= 0.5 * before) break;    /* second pass only if needed */
    }
    double nw = sqrt(dot(N, w, w));
    if (!isfinite(nw)) return 2;
    if (!(nw > 1e-14 * naz)) return 1;
    double gamma = 1.0 / nw;                               /* gamma := 1/||w_{l+1}|| */
    ensure_cap(S, L);
    double *Wl = L->W + (size_t)L->l * N, *Zl = L->Z + (size_t)L->l * N;
    ORC_PARALLEL_FOR
    for (int k = 0; k < N; k++) { Wl[k] = gamma * w[k]; Zl[k] = gamma * z[k]; }
    L->alpha[L->l] = dot(N, Wl, L->r0);                    /* alpha_{l+1} := w_{l+1} . r0 */
    L->l++;
    ORC_PARALLEL_FOR
    for (int k = 0; k < N; k++) {                          /* x := x0 + Z alpha; r := r0 - W alpha */
        double xs = L->x0[k], rs = L->r0[k];
        for (int i = 0; i < L->l; i++) {
            xs += L->alpha[i] * L->Z[(size_t)i * N + k];
            rs -= L->alpha[i] * L->W[(size_t)i * N + k];
        }
        L->x[k] = xs; L->r[k] = rs;
    }
    return 0;
}

static void record(osolver *S, int lev, int type) {
    if (lev != 0 || !S->hist || S->hist_len >= S->hist_cap) return;
    int N = ndof(S, 0);
    S->hist[S->hist_len] = sqrt(dot(N, S->lv[0].r, S->lv[0].r));
    S->hist_type[S->hist_len] = type;
    S->hist_len++;
}

/* x0 := x, r0 := b - A x, W, Z := {} on level lev (see "restart" above) */
static void restart(osolver *S, int lev, const double *b) {
    olevel *L = &S->lv[lev];
    int N = ndof(S, lev);
    apply(S, lev, L->x, L->r0);
    for (int k = 0; k < N; k++) { L->r0[k] = b[k] - L->r0[k]; L->r[k] = L->r0[k]; L->x0[k] = L->x[k]; }
    L->l = 0;
    if (lev == 0) S->restarts++;
    record(S, lev, 4);
}

/* one RM call inside MG with the level-0 breakdown bookkeeping */
static void mg_rm(osolver *S, int lev, const double *b, double *z, int type) {
    (void)b;
    int rc = rm_step(S, lev, z);
    if (rc == 2) S->status_flag = ORC_NONFINITE;
    if (lev == 0) {
        S->breakdowns_in_row = (rc == 1) ? S->breakdowns_in_row + 1 : 0;
        if (S->breakdowns_in_row >= 2 && S->status_flag == ORC_OK) S->status_flag = ORC_BREAKDOWN;
    }
    record(S, lev, type);
}

/* ------------------------------------------------------------------------ Alg. 2 */
/* x := MG(A_lev, b, x0); on entry x holds x0.  eps0/maxit0 apply to level 0. */
static void mg(osolver *S, int lev, const double *b, double *x, double rtol0, double atol0,
               int maxit0) {
    olevel *L = &S->lv[lev];
    int N = ndof(S, lev);
    L->l = 0;                                                 /* Z := {}, W := {} */
    apply(S, lev, x, L->r0);                                  /* r0 := b - A x0 */
    for (int k = 0; k < N; k++) { L->r0[k] = b[k] - L->r0[k]; L->r[k] = L->r0[k]; L->x0[k] = x[k]; L->x[k] = x[k]; }
    double n0 = sqrt(dot(N, L->r0, L->r0));
    if (lev == 0) S->res0 = n0;
    double eps = (lev == 0) ? fmax(rtol0 * n0, atol0) : S->lvl_rtol[lev] * n0;
    int maxit = (lev == 0) ? maxit0 : S->lvl_maxit[lev];
    record(S, lev, 0);
    int it = 0;
    for (;;) {
        if (!(sqrt(dot(N, L->r, L->r)) > eps)) {
            if (lev != 0 || L->l == 0) break;                 /* level 0: confirm on b - A x */
            restart(S, lev, b);
            if (!(sqrt(dot(N, L->r, L->r)) > eps)) break;
        }
        if (it >= maxit || S->status_flag != ORC_OK) break;
        smooth(S, lev, L->r, L->z);                           /* pre-smoother */
        mg_rm(S, lev, b, L->z, 1);
        restrict_(S, lev, L->r, S->lv[lev + 1].bc);           /* r_c := R r */
        olevel *C = &S->lv[lev + 1];
        if (lev + 1 == S->nlev - 1) {
            coarse_solve(S, C->bc, C->xc);                    /* z_c := A_c \ r_c */
        } else {
            memset(C->xc, 0, sizeof(double) * ndof(S, lev + 1));
            mg(S, lev + 1, C->bc, C->xc, 0, 0, 0);            /* z_c := MG(A_c, r_c, 0) */
        }
        prolong(S, lev, C->xc, L->z);                         /* z := P z_c */
        mg_rm(S, lev, b, L->z, 2);
        smooth(S, lev, L->r, L->z);                           /* post-smoother */
        mg_rm(S, lev, b, L->z, 3);
        it++;
        S->level_iters[lev]++;
        if (S->lmax > 0 && L->l + 3 > S->lmax) restart(S, lev, b);
    }
    memcpy(x, L->x, sizeof(double) * N);
}

/* Alg. AsyncMG on level 0 (async_m smoother steps per cycle); x: in x0, out x.  The
   stopping test, the level-0 confirmation restart and the lmax restart (now when the
   basis could not take one more cycle's async_m + 1 corrections) are those of mg. */
static void async_mg0(osolver *S, const double *b, double *x, double rtol0, double atol0,
                      int maxit0) {
    olevel *L = &S->lv[0];
    olevel *C = &S->lv[1];
    int N = ndof(S, 0);
    const int per_cycle = S->async_m + 1;
    L->l = 0;                                                 /* Z := {}, W := {} */
    apply(S, 0, x, L->r0);                                    /* r0 := b - A x0 */
    for (int k = 0; k < N; k++) { L->r0[k] = b[k] - L->r0[k]; L->r[k] = L->r0[k]; L->x0[k] = x[k]; L->x[k] = x[k]; }
    double n0 = sqrt(dot(N, L->r0, L->r0));
    S->res0 = n0;
    double eps = fmax(rtol0 * n0, atol0);
    record(S, 0, 0);
    double *zc = malloc(sizeof(double) * N);
    int it = 0;
    for (;;) {
        if (!(sqrt(dot(N, L->r, L->r)) > eps)) {
            if (L->l == 0) break;                             /* confirm on b - A x */
            restart(S, 0, b);
            if (!(sqrt(dot(N, L->r, L->r)) > eps)) break;
        }
        if (it >= maxit0 || S->status_flag != ORC_OK) break;
        /* coarse group: works on the residual of the cycle start */
        restrict_(S, 0, L->r, C->bc);                         /* r_c := R r */
        if (S->nlev == 2) {
            coarse_solve(S, C->bc, C->xc);                    /* z_c := A_c \ r_c */
        } else {
            memset(C->xc, 0, sizeof(double) * ndof(S, 1));
            mg(S, 1, C->bc, C->xc, 0, 0, 0);                  /* z_c := MG(A_c, r_c, 0) */
        }
        prolong(S, 0, C->xc, zc);                             /* z_cor := P z_c */
        /* smoother group: m smoothing + RM steps on the current residual */
        for (int k = 0; k < S->async_m; k++) {
            smooth(S, 0, L->r, L->z);
            mg_rm(S, 0, b, L->z, 1);
        }
        /* the synchronisation: RM with the coarse correction */
        memcpy(L->z, zc, sizeof(double) * N);
        mg_rm(S, 0, b, L->z, 2);
        it++;
        S->level_iters[0]++;
        if (S->lmax > 0 && L->l + per_cycle > S->lmax) restart(S, 0, b);
    }
    free(zc);
    memcpy(x, L->x, sizeof(double) * N);
}

/* ------------------------------------------------------------------------ C interface */
void orc_destroy(void *h);

/* blocks: [S][C][np][np] (slot-major input layout); nbr: [C][2d] or NULL (derived).
   transpose != 0 builds the solver of A^T (slot s of K := (slot opp(s) of nbr)^T). */
void *orc_create(int dim, int np, const int *n, int nlevels, const double *blocks,
                 const double *P, double omega, int sweeps, const double *lvl_rtol,
                 const int *lvl_maxit, int lmax, int transpose, int *status) {
    *status = ORC_INVALID_ARG;
    if (dim < 2 || dim > 3 || np < 1 || nlevels < 2 || nlevels > ORC_MAXLEV) return NULL;
    for (int j = 0; j < dim; j++)
        if (n[j] <= 0 || n[j] % (1 << (nlevels - 1))) return NULL;
    osolver *S = calloc(1, sizeof(osolver));
    S->dim = dim; S->np = np; S->S = 2 * dim + 1; S->nlev = nlevels; S->nchild = 1 << dim;
    S->omega = omega; S->sweeps = sweeps; S->lmax = lmax;
    for (int l = 0; l < nlevels; l++) { S->lvl_rtol[l] = lvl_rtol[l]; S->lvl_maxit[l] = lvl_maxit[l]; }
    size_t bs = (size_t)np * np;
    S->P = malloc(sizeof(double) * S->nchild * bs);
    memcpy(S->P, P, sizeof(double) * S->nchild * bs);
    for (int l = 0; l < nlevels; l++) {
        olevel *L = &S->lv[l];
        L->n[0] = n[0] >> l; L->n[1] = n[1] >> l; L->n[2] = dim == 3 ? n[2] >> l : 1;
        L->ncell = L->n[0] * L->n[1] * L->n[2];
        build_nbr(S, L);
        alloc_work(S, L);
    }
    olevel *F = &S->lv[0];
    int nf = 2 * dim;
    F->blk = malloc(sizeof(double) * F->ncell * S->S * bs);
    for (int K = 0; K < F->ncell; K++)
        for (int sl = 0; sl < S->S; sl++) {
            double *dst = F->blk + ((size_t)K * S->S + sl) * bs;
            if (!transpose) {
                memcpy(dst, blocks + ((size_t)sl * F->ncell + K) * bs, sizeof(double) * bs);
            } else {
                int J = (sl == 0) ? K : F->nbr[K * nf + sl - 1];
                int opp = (sl == 0) ? 0 : (((sl - 1) ^ 1) + 1);
                if (J < 0) { memset(dst, 0, sizeof(double) * bs); continue; }
                const double *src = blocks + ((size_t)opp * F->ncell + J) * bs;
                for (int i = 0; i < np; i++)
                    for (int j = 0; j < np; j++) dst[i * np + j] = src[j * np + i];
            }
        }
    for (int l = 0; l + 1 < nlevels; l++) galerkin(S, l);
    for (int l = 0; l < nlevels; l++) {
        olevel *L = &S->lv[l];
        L->inv = malloc(sizeof(double) * L->ncell * bs);
        for (int K = 0; K < L->ncell; K++)
            if (invert_block(np, L->blk + (size_t)K * S->S * bs, L->inv + (size_t)K * bs)) {
                *status = ORC_SINGULAR; orc_destroy(S); return NULL;
            }
    }
    if (coarse_factor(S)) { *status = ORC_SINGULAR; orc_destroy(S); return NULL; }
    *status = ORC_OK;
    return S;
}

void orc_destroy(void *h) {
    osolver *S = h;
    if (!S) return;
    for (int l = 0; l < S->nlev; l++) {
        olevel *L = &S->lv[l];
        void *p[] = {L->nbr, L->blk, L->inv, L->W, L->Z, L->alpha, L->x0, L->r0, L->x, L->r,
                     L->z, L->w, L->t, L->bc, L->xc, L->pcell[0], L->pcell[1], L->pinv[0],
                     L->pinv[1]};
        for (int i = 0; i < 19; i++) free(p[i]);
    }
    free(S->P); free(S->Lc); free(S->piv); free(S);
}

/* Solve A x = b to ||r|| <= max(rtol ||b - A x0||, atol).  x: in x0, out x.
   hist/hist_type (capacity hist_cap) receive ||r|| after each level-0 RM with type
   0 initial, 1 pre-smoother, 2 coarse correction, 3 post-smoother, 4 restart (true
   residual). */
int orc_solve(void *h, const double *b, double *x, double rtol, double atol, int maxiter,
              double *hist, int *hist_type, int hist_cap, int *hist_len, int *iters,
              double *rel_res, int *level_iters) {
    osolver *S = h;
    int N = ndof(S, 0);
    for (int k = 0; k < N; k++)
        if (!isfinite(b[k]) || !isfinite(x[k])) return ORC_NONFINITE;
    S->hist = hist; S->hist_type = hist_type; S->hist_cap = hist ? hist_cap : 0; S->hist_len = 0;
    memset(S->level_iters, 0, sizeof(S->level_iters));
    S->breakdowns_in_row = 0; S->status_flag = ORC_OK; S->restarts = 0;
    if (S->async_m > 0) async_mg0(S, b, x, rtol, atol, maxiter);
    else mg(S, 0, b, x, rtol, atol, maxiter);
    olevel *L = &S->lv[0];
    apply(S, 0, x, L->t);                                     /* report the true residual */
    for (int k = 0; k < N; k++) L->t[k] = b[k] - L->t[k];
    double n0 = S->res0, nr = sqrt(dot(N, L->t, L->t));
    if (hist_len) *hist_len = S->hist_len;
    if (iters) *iters = S->level_iters[0];
    if (rel_res) *rel_res = (n0 > 0) ? nr / n0 : 0.0;
    if (level_iters) memcpy(level_iters, S->level_iters, sizeof(int) * S->nlev);
    if (S->status_flag != ORC_OK) return S->status_flag;
    return (nr <= fmax(rtol * n0, atol)) ? ORC_OK : ORC_NOT_CONVERGED;
}

/* component access for the tests */
int orc_ncell(void *h, int lev) { return ((osolver *)h)->lv[lev].ncell; }
void orc_apply(void *h, int lev, const double *x, double *y) { apply(h, lev, x, y); }
void orc_smooth(void *h, int lev, const double *b, double *x) { smooth(h, lev, b, x); }
void orc_restrict(void *h, int lev, const double *rf, double *rc) { restrict_(h, lev, rf, rc); }
void orc_prolong(void *h, int lev, const double *zc, double *zf) { prolong(h, lev, zc, zf); }
void orc_coarse_solve(void *h, const double *r, double *z) { coarse_solve(h, r, z); }
/* blocks of level lev in the input layout [S][C][np][np] */
void orc_get_blocks(void *h, int lev, double *out) {
    osolver *S = h;
    olevel *L = &S->lv[lev];
    size_t bs = (size_t)S->np * S->np;
    for (int K = 0; K < L->ncell; K++)
        for (int sl = 0; sl < S->S; sl++)
            memcpy(out + ((size_t)sl * L->ncell + K) * bs, L->blk + ((size_t)K * S->S + sl) * bs,
                   sizeof(double) * bs);
}
void orc_get_inv(void *h, int lev, double *out) {
    osolver *S = h;
    memcpy(out, S->lv[lev].inv, sizeof(double) * S->lv[lev].ncell * S->np * S->np);
}

/* RM driver on level lev: start a fresh basis with x0 and r0 = b - A x0 */
void orc_rm_begin(void *h, int lev, const double *b, const double *x0) {
    osolver *S = h;
    olevel *L = &S->lv[lev];
    int N = ndof(S, lev);
    L->l = 0;
    apply(S, lev, x0, L->r0);
    for (int k = 0; k < N; k++) { L->r0[k] = b[k] - L->r0[k]; L->r[k] = L->r0[k]; L->x0[k] = x0[k]; L->x[k] = x0[k]; }
}
/* one Alg. 1 call with correction z (copied); returns rm_step's code; x, r, l out */
int orc_rm_call(void *h, int lev, const double *z, double *x, double *r, int *l) {
    osolver *S = h;
    olevel *L = &S->lv[lev];
    int N = ndof(S, lev);
    memcpy(L->z, z, sizeof(double) * N);
    int rc = rm_step(S, lev, L->z);
    memcpy(x, L->x, sizeof(double) * N);
    memcpy(r, L->r, sizeof(double) * N);
    *l = L->l;
    return rc;
}
void orc_rm_basis(void *h, int lev, double *W, double *Z) {
    osolver *S = h;
    olevel *L = &S->lv[lev];
    size_t N = (size_t)ndof(S, lev);
    memcpy(W, L->W, sizeof(double) * N * L->l);
    memcpy(Z, L->Z, sizeof(double) * N * L->l);
}

/* ------------------------------------------------------------------------ adjoint gradient */
/* g_K = -lambda^T (dA/d log nu_K) u for A = sum_K nu_K V + sum_F gamma_F F_F +
   sum_{bnd F} nu_K B_F, gamma_F = 2 nu_K nu_K' / (nu_K + nu_K').
   V [np][np]; F [dim][4][np][np] (LL, LR, RL, RR; L = low-side cell); B [dim][2][np][np]. */
static double bil(int np, const double *M, const double *l, const double *u) {
    double s = 0.0;
    for (int i = 0; i < np; i++)
        for (int j = 0; j < np; j++) s += l[i] * M[i * np + j] * u[j];
    return s;
}
void orc_grad_lognu(int dim, int np, const int *n, const double *nu, const double *V,
                    const double *F, const double *B, const double *lam, const double *u,
                    double *g) {
    int C = n[0] * n[1] * (dim == 3 ? n[2] : 1);
    int stride[3] = {1, n[0], n[0] * n[1]};
    size_t bs = (size_t)np * np;
    for (int K = 0; K < C; K++) {
        int c[3] = {K % n[0], (K / n[0]) % n[1], dim == 3 ? K / (n[0] * n[1]) : 0};
        const double *lK = lam + (size_t)K * np, *uK = u + (size_t)K * np;
        double s = bil(np, V, lK, uK);                       /* d(nu_K V)/d nu_K */
        for (int k = 0; k < dim; k++) {
            const double *Fk = F + (size_t)k * 4 * bs, *Bk = B + (size_t)k * 2 * bs;
            /* high face of K: K is the low-side cell L, neighbour R */
            if (c[k] < n[k] - 1) {
                int R = K + stride[k];
                double a = nu[K], b = nu[R], dg = 2.0 * b * b / ((a + b) * (a + b));
                const double *lR = lam + (size_t)R * np, *uR = u + (size_t)R * np;
                s += dg * (bil(np, Fk, lK, uK) + bil(np, Fk + bs, lK, uR) +
                           bil(np, Fk + 2 * bs, lR, uK) + bil(np, Fk + 3 * bs, lR, uR));
            } else {
                s += bil(np, Bk + bs, lK, uK);
            }
            /* low face of K: K is the high-side cell R, neighbour L */
            if (c[k] > 0) {
                int Lc = K - stride[k];
                double a = nu[K], b = nu[Lc], dg = 2.0 * b * b / ((a + b) * (a + b));
                const double *lL = lam + (size_t)Lc * np, *uL = u + (size_t)Lc * np;
                s += dg * (bil(np, Fk, lL, uL) + bil(np, Fk + bs, lL, uK) +
                           bil(np, Fk + 2 * bs, lK, uL) + bil(np, Fk + 3 * bs, lK, uK));
            } else {
                s += bil(np, Bk, lK, uK);
            }
        }
        g[K] = -nu[K] * s;
    }
}

/* number of stored basis vectors on level lev (after a solve: of its last MG call) */
int orc_basis_size(void *h, int lev) { return ((osolver *)h)->lv[lev].l; }
int orc_restarts(void *h) { return ((osolver *)h)->restarts; }
/* m > 0: level 0 runs Alg. AsyncMG with m smoother steps per cycle; 0: Alg. 2 */
void orc_set_async(void *h, int m) { ((osolver *)h)->async_m = m > 0 ? m : 0; }
/* smoother of every iterated level: 0 Alg. BJ, 1 Alg. AS (builds the patches and their
   inverses on first use); returns 0, or 1 if a patch matrix is singular */
int orc_set_smoother(void *h, int kind) {
    osolver *S = h;
    if (kind == 1) {
        if (S->nchild * S->np > 8 * 32) return 1;
        for (int l = 0; l + 1 < S->nlev; l++)
            if (!S->lv[l].pcell[0])
                for (int part = 0; part < 2; part++)
                    if (build_patches(S, l, part)) return 1;
    }
    S->smoother = kind == 1 ? 1 : 0;
    return 0;
}
/* threads of the OpenMP build's parallel loops (n <= 0: all host cores); returns the
   number in use, 1 for the serial build */
int orc_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    else omp_set_num_threads(omp_get_num_procs());
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
