"""Pins of the CPU oracle against facts the paper and the mathematics fix.

Each pin is independent of the oracle's own code: dense LU (LAPACK), a from-scratch
Arnoldi least-squares GMRES, the closed form of damped block-Jacobi sweeps, orthonormality
and A Z = W of the stored basis (Alg. 1), the monotone residual that the minimisation
guarantees (Alg. 1/2 "ENSURE" clauses), the transfer identities of nested spaces, the
Galerkin energy identity, and central finite differences of the adjoint gradient.
"""
import numpy as np
import pytest

from oracle import ORC_BREAKDOWN, ORC_NOT_CONVERGED, ORC_OK, OracleSolver, grad_lognu
from workloads import dense_matrix, eval_field, make_problem, neighbours, project, workload


def _solver(pr, **kw):
    return OracleSolver.from_problem(pr, **kw)


# ------------------------------------------------------------------ plain definition
@pytest.mark.parametrize("name", ["sipg2d_p1_16x16", "sipg3d_p1_8x4x4", "sipg2d_p2_32x16",
                                  "sipg3d_p2_8cube"])
def test_solution_matches_dense_lu(name):
    pr = workload(name).make(0)
    A = dense_matrix(pr.blocks, pr.nbr)
    xs = np.linalg.solve(A, pr.b)
    x, info = _solver(pr).solve(pr.b, rtol=1e-10)
    assert info["status"] == ORC_OK
    assert info["rel_res"] <= 1e-10                   # reported on the true residual
    assert np.linalg.norm(pr.b - A @ x) <= 1e-10 * np.linalg.norm(pr.b)
    assert np.linalg.norm(x - xs) <= 1e-8 * np.linalg.norm(xs)


def test_manufactured_solution_with_nonzero_initial_guess():
    pr = workload("sipg3d_p1_8x4x4").make(3)
    A = dense_matrix(pr.blocks, pr.nbr)
    u = np.random.default_rng(7).uniform(-1, 1, pr.ndof)
    x0 = np.random.default_rng(8).uniform(-1, 1, pr.ndof)
    x, info = _solver(pr).solve(A @ u, x0=x0, rtol=1e-11)
    assert info["status"] == ORC_OK
    ev = np.linalg.eigvalsh(A)
    kappa = ev[-1] / ev[0]
    rel = np.linalg.norm(A @ u - A @ x) / np.linalg.norm(A @ u)
    assert np.linalg.norm(x - u) <= kappa * rel * np.linalg.norm(u)
    assert np.linalg.norm(x - u) <= 1e-6 * np.linalg.norm(u)


def test_stretched_high_contrast_p3():
    pr = workload("sipg3d_p3_8cube_zstretch").make(0)
    A = dense_matrix(pr.blocks, pr.nbr)
    x, info = _solver(pr).solve(pr.b, rtol=1e-10, maxiter=400)
    assert info["status"] == ORC_OK
    assert np.linalg.norm(pr.b - A @ x) <= 1e-10 * np.linalg.norm(pr.b)
    xs = np.linalg.solve(A, pr.b)
    assert np.linalg.norm(x - xs) <= 1e-7 * np.linalg.norm(xs)


# ------------------------------------------------------------------ Alg. 1 = GCR/GMRES
def _gmres_residuals(A, r0, k):
    """From-scratch GMRES: Arnoldi with MGS, then min ||beta e1 - H y|| by lstsq."""
    n = r0.size
    V = np.zeros((n, k + 1))
    H = np.zeros((k + 1, k))
    beta = np.linalg.norm(r0)
    V[:, 0] = r0 / beta
    res = []
    for j in range(k):
        w = A @ V[:, j]
        for i in range(j + 1):
            H[i, j] = V[:, i] @ w
            w = w - H[i, j] * V[:, i]
        H[j + 1, j] = np.linalg.norm(w)
        V[:, j + 1] = w / H[j + 1, j]
        e1 = np.zeros(j + 2)
        e1[0] = beta
        y = np.linalg.lstsq(H[:j + 2, :j + 1], e1, rcond=None)[0]
        res.append(np.linalg.norm(e1 - H[:j + 2, :j + 1] @ y))
    return np.array(res)


def test_residual_minimization_with_z_equal_r_is_gmres():
    """With z := r each Alg. 1 call extends span(Z) to the next Krylov space and minimises
    the residual over it, so the residual norms are GMRES's."""
    pr = workload("sipg2d_p1_16x16").make(0)
    S = _solver(pr)
    A = dense_matrix(pr.blocks, pr.nbr)
    x0 = np.zeros(pr.ndof)
    S.rm_begin(0, pr.b, x0)
    r = pr.b.copy()
    ours = []
    for _ in range(25):
        rc, x, r, l = S.rm_call(0, r)
        assert rc == 0
        ours.append(np.linalg.norm(r))
    ref = _gmres_residuals(A, pr.b, 25)
    assert np.allclose(ours, ref, rtol=1e-9, atol=0)


def test_basis_invariants_and_recursive_residual():
    """W^T W = I, A Z = W, ||r|| non-increasing, and the recursively updated r equals
    b - A x, after every Alg. 1 call with smoother, coarse and random corrections."""
    pr = workload("sipg3d_p1_8x4x4").make(1)
    S = _solver(pr)
    A = dense_matrix(pr.blocks, pr.nbr)
    rng = np.random.default_rng(5)
    x0 = rng.uniform(-1, 1, pr.ndof)
    S.rm_begin(0, pr.b, x0)
    r = pr.b - A @ x0
    last = np.linalg.norm(r)
    for k in range(30):
        kind = k % 3
        if kind == 0:
            z = S.smooth(0, r)
        elif kind == 1:
            z = S.prolong(0, S.restrict(0, r))       # a correction from the coarse space
        else:
            z = rng.uniform(-1, 1, pr.ndof)
        rc, x, r, l = S.rm_call(0, z)
        assert rc == 0
        W, Z = S.rm_basis(0, l)
        assert np.abs(W @ W.T - np.eye(l)).max() < 1e-12
        assert np.abs(A @ Z.T - W.T).max() < 1e-9 * np.abs(W).max()
        nr = np.linalg.norm(r)
        assert nr <= last * (1 + 1e-14)
        last = nr
        # equal up to the rounding drift of a recursive residual (a wrong sign or index
        # would show at O(1))
        assert np.linalg.norm(r - (pr.b - A @ x)) < 1e-8 * np.linalg.norm(pr.b)


def test_breakdown_discards_dependent_correction():
    pr = workload("sipg2d_p1_16x16").make(0)
    S = _solver(pr)
    S.rm_begin(0, pr.b, np.zeros(pr.ndof))
    z1 = S.smooth(0, pr.b)
    rc, x1, r1, l1 = S.rm_call(0, z1)
    assert rc == 0 and l1 == 1
    rc, x2, r2, l2 = S.rm_call(0, 3.0 * z1)         # already in span(Z)
    assert rc == 1 and l2 == 1 and np.array_equal(x2, x1) and np.array_equal(r2, r1)
    rc, x3, r3, l3 = S.rm_call(0, np.zeros(pr.ndof))
    assert rc == 1 and l3 == 1


def test_monotone_history_and_level_criteria():
    pr = workload("sipg2d_p2_32x16").make(2)         # 4 levels: 0,1,2 iterate, 3 direct
    S = _solver(pr)
    x, info = S.solve(pr.b, rtol=1e-10)
    h, t = info["hist"], info["hist_type"]
    assert info["status"] == ORC_OK
    # Alg. 1 never increases ||r||: within each run of RM calls, and across restarts on
    # the true residual (a restart entry, type 4, replaces the recursive residual by
    # b - A x, which may sit above it by the rounding drift)
    d = np.diff(h)
    assert np.all(d[t[1:] != 4] <= 1e-13 * h[0])
    ht = h[t == 4]
    assert np.all(np.diff(ht) <= 0) and h[-1] <= 1e-10 * h[0]
    assert t[0] == 0 and list(t[1:4]) == [1, 2, 3]
    it = info["level_iters"]
    assert it[1] <= 20 * it[0] and it[1] >= it[0]      # level 1: at most 20 per visit
    assert it[2] <= 2 * it[1] and it[2] >= it[1]       # level 2: at most 2 per visit


def test_deep_levels_run_one_iteration_per_visit():
    pr = make_problem(2, 1, (32, 32), 5, seed=4)       # levels 0..3 iterate, 4 direct
    x, info = _solver(pr).solve(pr.b, rtol=1e-8)
    it = info["level_iters"]
    assert info["status"] == ORC_OK
    assert it[3] == it[2]


def test_maxiter_returns_not_converged_but_no_worse():
    pr = workload("sipg2d_p1_16x16").make(0)
    x, info = _solver(pr).solve(pr.b, rtol=1e-14, maxiter=2)
    assert info["status"] == ORC_NOT_CONVERGED and info["iters"] == 2
    assert info["rel_res"] < 1.0


# ------------------------------------------------------------------ Alg. BJ
@pytest.mark.parametrize("omega,sweeps", [(0.7, 1), (0.7, 5), (1.0, 3)])
def test_block_jacobi_closed_form(omega, sweeps):
    """Alg. BJ from x = 0: x_k = sum_{j<k} (I - w D^-1 A)^j w D^-1 b (D block diagonal)."""
    pr = workload("sipg3d_p1_8x4x4").make(0)
    S = _solver(pr, omega=omega, sweeps=sweeps)
    A = dense_matrix(pr.blocks, pr.nbr)
    Np = pr.np_
    Dinv = np.zeros_like(A)
    for K in range(pr.ncells):
        sl = slice(K * Np, (K + 1) * Np)
        Dinv[sl, sl] = np.linalg.inv(A[sl, sl])
    M = omega * Dinv
    E = np.eye(A.shape[0]) - M @ A
    x, term = np.zeros(pr.ndof), M @ pr.b
    for _ in range(sweeps):
        x, term = x + term, E @ term
    z = S.smooth(0, pr.b)
    assert np.abs(z - x).max() <= 1e-12 * np.abs(x).max()


def test_block_inverses():
    pr = workload("sipg3d_p2_8cube").make(0)
    S = _solver(pr)
    for lev in range(pr.nlevels):
        B = S.blocks(lev)[0]
        I = np.einsum("kij,kjl->kil", S.inverses(lev), B)
        assert np.abs(I - np.eye(pr.np_)).max() < 1e-10


# ------------------------------------------------------------------ transfers, Galerkin
def test_restriction_is_transpose_of_prolongation_and_orthonormal():
    pr = workload("sipg3d_p2_8cube").make(0)
    S = _solver(pr)
    rng = np.random.default_rng(0)
    for lev in range(pr.nlevels - 1):
        rf, zc = rng.standard_normal(S.ndof(lev)), rng.standard_normal(S.ndof(lev + 1))
        assert abs(S.restrict(lev, rf) @ zc - rf @ S.prolong(lev, zc)) < 1e-12 * np.abs(rf).sum()
        assert np.abs(S.restrict(lev, S.prolong(lev, zc)) - zc).max() < 1e-13


@pytest.mark.parametrize("d,p,n", [(2, 2, (8, 4)), (3, 1, (4, 4, 4))])
def test_prolongation_reproduces_coarse_polynomial(d, p, n):
    pr = make_problem(d, p, n, 2)
    S = _solver(pr)
    nc = tuple(v // 2 for v in n)
    fun = lambda X: 0.3 + X[:, 0] - 2 * X[:, 1] ** p + (X[:, -1] * X[:, 0] if p > 1 else 0)
    hc = 2 * pr.h
    uf = S.prolong(0, project(fun, nc, p, hc))
    pts = np.random.default_rng(1).uniform(0, 1, (400, d))
    assert np.abs(eval_field(uf, n, p, pr.h, pts) - fun(pts)).max() < 1e-12


def test_galerkin_energy_identity_and_spd():
    pr = workload("sipg2d_p2_32x16").make(0)
    S = _solver(pr)
    rng = np.random.default_rng(2)
    for lev in range(pr.nlevels - 1):
        v = rng.standard_normal(S.ndof(lev + 1))
        Pv = S.prolong(lev, v)
        lhs = v @ S.apply(lev + 1, v)
        rhs = Pv @ S.apply(lev, Pv)
        assert abs(lhs - rhs) <= 1e-12 * abs(rhs)
        nc = tuple(m >> (lev + 1) for m in pr.n)
        Ac = dense_matrix(S.blocks(lev + 1), neighbours(nc))
        assert np.abs(Ac - Ac.T).max() <= 1e-12 * np.abs(Ac).max()
        np.linalg.cholesky(Ac)


def test_coarse_solve_is_exact():
    pr = workload("sipg3d_p2_8cube").make(0)
    S = _solver(pr)
    L = pr.nlevels - 1
    nc = tuple(m >> L for m in pr.n)
    Ac = dense_matrix(S.blocks(L), neighbours(nc))
    r = np.random.default_rng(3).standard_normal(Ac.shape[0])
    assert np.abs(S.coarse_solve(r) - np.linalg.solve(Ac, r)).max() <= 1e-10 * np.abs(np.linalg.solve(Ac, r)).max()


# ------------------------------------------------------------------ adjoint
def test_adjoint_of_symmetric_operator_equals_forward_bitwise():
    pr = workload("sipg3d_p1_8x4x4").make(0)
    x, _ = _solver(pr).solve(pr.b, rtol=1e-10)
    y, _ = _solver(pr, transpose=True).solve(pr.b, rtol=1e-10)
    assert np.array_equal(x, y)


def test_adjoint_of_nonsymmetric_operator():
    pr = workload("sipg3d_p1_8x4x4").make(0)
    blocks = pr.blocks.copy()
    rng = np.random.default_rng(4)
    for s in range(1, blocks.shape[0]):
        blocks[s] *= 1.0 + 0.2 * rng.uniform(-1, 1, blocks.shape[1])[:, None, None]
    A = dense_matrix(blocks, pr.nbr)
    S = OracleSolver(pr.d, pr.np_, pr.n, pr.nlevels, blocks, pr.prolong, transpose=True)
    lam, info = S.solve(pr.b, rtol=1e-12)
    assert info["status"] == ORC_OK
    ref = np.linalg.solve(A.T, pr.b)
    assert np.linalg.norm(lam - ref) <= 1e-9 * np.linalg.norm(ref)


def _loss_and_solution(pr, lognu, ut):
    from workloads.sipg import assemble
    blocks, nbr = assemble(pr.n, pr.p, pr.h, np.exp(lognu), pr.eta, pr.ref)
    A = dense_matrix(blocks, nbr)
    u = np.linalg.solve(A, pr.b)
    return 0.5 * np.sum((u - ut) ** 2), u, A


@pytest.mark.parametrize("d,p,n", [(2, 2, (4, 4)), (3, 1, (4, 4, 2))])
def test_adjoint_gradient_matches_central_differences(d, p, n):
    pr = make_problem(d, p, n, 2, nu_kind="lognormal", seed=3)
    lognu = np.log(pr.nu)
    ut = np.random.default_rng(9).uniform(-1, 1, pr.ndof) * 1e-3
    L0, u, A = _loss_and_solution(pr, lognu, ut)
    lam = np.linalg.solve(A.T, u - ut)
    g = grad_lognu(pr, pr.nu, lam, u)
    hstep = 1e-6
    fd = np.zeros_like(g)
    for K in range(g.size):
        e = np.zeros_like(lognu)
        e[K] = hstep
        fd[K] = (_loss_and_solution(pr, lognu + e, ut)[0] - _loss_and_solution(pr, lognu - e, ut)[0]) / (2 * hstep)
    assert np.abs(g - fd).max() <= 1e-6 * np.abs(fd).max()


# ------------------------------------------------------------------ Alg. AsyncMG (task-parallel)
def _dense_prolongation(pr):
    """P (N0 x N1) of a 2^d agglomeration from the child matrices P_k (input data)."""
    n0 = np.array(pr.n)
    n1 = n0 // 2
    d, Np = pr.d, pr.np_
    C0, C1 = int(np.prod(n0)), int(np.prod(n1))
    P = np.zeros((C0 * Np, C1 * Np))
    for K in range(C0):
        c = np.unravel_index(K, tuple(n0[::-1]))[::-1]          # x fastest
        J = np.ravel_multi_index(tuple((np.array(c) // 2)[::-1]), tuple(n1[::-1]))
        k = sum(((c[j] & 1) << j) for j in range(d))
        P[K * Np:(K + 1) * Np, J * Np:(J + 1) * Np] = pr.prolong[k]
    return P


def _dense_bj(A, Np, r, omega, sweeps):
    """Alg. BJ from z = 0 with dense algebra: z += omega D^-1 (r - A z)."""
    N = A.shape[0]
    Dinv = np.zeros_like(A)
    for K in range(N // Np):
        s = slice(K * Np, (K + 1) * Np)
        Dinv[s, s] = np.linalg.inv(A[s, s])
    z = np.zeros(N)
    for _ in range(sweeps):
        z = z + omega * Dinv @ (r - A @ z)
    return z


@pytest.mark.parametrize("m", [1, 2, 3])
def test_async_first_cycle_is_least_squares_over_its_corrections(m):
    """One cycle of Alg. AsyncMG on two levels.  The coarse correction is
    z_cor = P A_c^-1 P^T r0, from the cycle-start residual.  The smoother corrections are
    z_k = BJ(r_{k-1}), each from the residual the previous minimisation left.  By Alg. 1,
    the residual after the cycle is the least-squares residual of r0 over
    A span{z_1..z_m, z_cor}.  Everything here is rebuilt with dense algebra."""
    pr = make_problem(2, 1, (8, 8), 2, seed=11)
    A = dense_matrix(pr.blocks, pr.nbr)
    P = _dense_prolongation(pr)
    Ac = P.T @ A @ P
    r0 = pr.b.copy()
    zc = P @ np.linalg.solve(Ac, P.T @ r0)
    Zs, r = [], r0.copy()
    for _ in range(m):
        z = _dense_bj(A, pr.np_, r, 0.7, 5)
        Zs.append(z)
        Q, _ = np.linalg.qr(A @ np.stack(Zs, axis=1))
        r = r0 - Q @ (Q.T @ r0)
    Q, _ = np.linalg.qr(A @ np.stack(Zs + [zc], axis=1))
    r_expected = np.linalg.norm(r0 - Q @ (Q.T @ r0))
    S = _solver(pr, async_smooth=m)
    x, info = S.solve(pr.b, rtol=1e-14, maxiter=1)
    h, t = info["hist"], info["hist_type"]
    assert list(t[:m + 2]) == [0] + [1] * m + [2]
    assert abs(h[m + 1] - r_expected) <= 1e-10 * h[0]
    # and the iterate's true residual is that residual
    assert abs(np.linalg.norm(pr.b - A @ x) - r_expected) <= 1e-10 * h[0]


@pytest.mark.parametrize("name", ["sipg2d_p1_16x16", "sipg3d_p1_8x4x4", "sipg2d_p2_32x16",
                                  "sipg3d_p2_8cube"])
@pytest.mark.parametrize("m", [1, 3])
def test_async_solution_matches_dense_lu(name, m):
    pr = workload(name).make(0)
    A = dense_matrix(pr.blocks, pr.nbr)
    xs = np.linalg.solve(A, pr.b)
    x, info = _solver(pr, async_smooth=m).solve(pr.b, rtol=1e-10, maxiter=2000)
    assert info["status"] == ORC_OK
    assert np.linalg.norm(pr.b - A @ x) <= 1e-10 * np.linalg.norm(pr.b)
    assert np.linalg.norm(x - xs) <= 1e-8 * np.linalg.norm(xs)
    h, t = info["hist"], info["hist_type"]
    d = np.diff(h)
    assert np.all(d[t[1:] != 4] <= 1e-13 * h[0])      # Alg. 1: monotone within runs


def test_async_restart_keeps_basis_within_lmax():
    """With lmax = 8 and m = 3 (4 corrections per cycle) the level restarts before the
    basis would exceed 8 vectors; the solve still converges."""
    pr = workload("sipg2d_p1_16x16").make(1)
    S = _solver(pr, async_smooth=3, lmax=8)
    x, info = S.solve(pr.b, rtol=1e-10, maxiter=2000)
    assert info["status"] == ORC_OK and info["restarts"] >= 1
    assert S.basis_size(0) <= 8
    t = info["hist_type"]
    # between two restart entries (type 4) there are at most two cycles' corrections
    runs = np.split(t, np.where(t == 4)[0])
    assert max(int(np.sum(r != 4) - np.sum(r == 0)) for r in runs) <= 8


@pytest.mark.parametrize("async_m", [0, 2])
def test_exact_smoother_on_decoupled_cells_converges_after_one_correction(async_m):
    """With no coupling between cells (all face blocks zero) the block-Jacobi inverse is
    A^-1, so one sweep with omega = 1 from z = 0 gives z = A^-1 r and the first Alg. 1
    call reaches the exact solution (the paper's special case of an exact smoother)."""
    pr = make_problem(2, 2, (4, 4), 2, seed=2)
    blocks = pr.blocks.copy()
    blocks[1:] = 0.0                                   # decouple the cells
    rng = np.random.default_rng(5)
    for K in range(blocks.shape[1]):                  # well-conditioned SPD diagonal blocks
        M = rng.standard_normal((pr.np_, pr.np_))
        blocks[0, K] = M @ M.T + pr.np_ * np.eye(pr.np_)
    S = OracleSolver(pr.d, pr.np_, pr.n, pr.nlevels, blocks, pr.prolong, omega=1.0, sweeps=1,
                     async_smooth=async_m)
    x, info = S.solve(pr.b, rtol=1e-12, maxiter=5)
    h, t = info["hist"], info["hist_type"]
    assert t[1] == 1                                  # the first correction is the smoother's
    assert h[1] <= 1e-13 * h[0]
    xs = np.concatenate([np.linalg.solve(blocks[0, K], pr.b[K * pr.np_:(K + 1) * pr.np_])
                         for K in range(blocks.shape[1])])
    assert np.linalg.norm(x - xs) <= 1e-12 * np.linalg.norm(xs)


# ------------------------------------------------------------------ all-core build
@pytest.mark.parametrize("m", [0, 4])
def test_openmp_build_gives_bitwise_the_serial_results(m):
    """The OpenMP build of the oracle (the benchmark's all-core CPU baseline) runs only its
    cell- and element-parallel loops on several threads; every sum stays sequential, so
    solves, histories and level counts are bitwise those of the serial build."""
    import oracle
    assert oracle.threads(4) >= 1
    pr = make_problem(3, 2, (8, 8, 8), 3, seed=4)
    out = []
    for omp in (False, True):
        x, info = _solver(pr, openmp=omp, async_smooth=m).solve(pr.b, rtol=1e-10, maxiter=200)
        assert info["status"] == ORC_OK
        out.append((x, info))
    (x0, i0), (x1, i1) = out
    assert np.array_equal(x0, x1)
    assert np.array_equal(i0["hist"], i1["hist"]) and i0["iters"] == i1["iters"]
    assert np.array_equal(i0["level_iters"], i1["level_iters"])


# ------------------------------------------------------------------ Alg. AS (additive Schwarz)
def _patch_dofs(pr, part):
    """DOF index sets of the 2^d-cell patches of one partition, enumerated here from the
    grid alone: partition 0 = the aligned 2^d blocks, partition 1 = the blocks shifted by
    one cell in every direction (clipped at the boundary)."""
    n = list(pr.n) + [1] * (3 - len(pr.n))
    d, np_ = pr.d, pr.np_
    ranges = [range(n[j] // 2 + part) if j < d else range(1) for j in range(3)]
    out = []
    for pz in ranges[2]:
        for py in ranges[1]:
            for px in ranges[0]:
                cells = []
                for cz in ([0, 1] if d == 3 else [0]):
                    for cy in (0, 1):
                        for cx in (0, 1):
                            x, y = 2 * px - part + cx, 2 * py - part + cy
                            z = 2 * pz - part + cz if d == 3 else 0
                            if 0 <= x < n[0] and 0 <= y < n[1] and 0 <= z < n[2]:
                                cells.append(x + n[0] * (y + n[1] * z))
                out.append(np.concatenate([np.arange(K * np_, (K + 1) * np_) for K in cells]))
    return out


def _dense_as(A, pr, b, omega, sweeps):
    """Additive Schwarz iterations from x = 0 written with dense submatrices and LU solves."""
    x = np.zeros_like(b)
    parts = [_patch_dofs(pr, 0), _patch_dofs(pr, 1)]
    for _ in range(sweeps):
        r = b - A @ x
        e = np.zeros_like(b)
        for patches in parts:
            for idx in patches:
                e[idx] += np.linalg.solve(A[np.ix_(idx, idx)], r[idx])
        x = x + omega * e
    return x


@pytest.mark.parametrize("shape", [(2, 1, (8, 8)), (3, 1, (4, 4, 4)), (3, 2, (4, 4, 4)), (3, 2, (6, 6, 2))])
@pytest.mark.parametrize("sweeps", [1, 2])
def test_schwarz_smoother_matches_dense_patch_solves(shape, sweeps):
    """Alg. AS on two partitions of overlapping 2^d-cell patches against the same
    iteration built from dense submatrices A[idx, idx] and LU solves."""
    d, p, n = shape
    pr = make_problem(d, p, n, 2, seed=3)
    A = dense_matrix(pr.blocks, pr.nbr)
    orc = _solver(pr, smoother="as", omega=0.4, sweeps=sweeps)
    x = orc.smooth(0, pr.b)
    ref = _dense_as(A, pr, pr.b, 0.4, sweeps)
    assert np.abs(x - ref).max() <= 1e-12 * np.abs(ref).max()


def test_schwarz_smoother_on_decoupled_cells_has_closed_form():
    """With every face coupling removed, each patch solve is D^-1 on its cells and every
    cell lies in one patch of each partition: k sweeps give (1 - (1 - 2 omega)^k) D^-1 b."""
    pr = make_problem(3, 2, (4, 4, 4), 2, seed=5)
    blocks = pr.blocks.copy()
    blocks[1:] = 0.0
    omega, k = 0.3, 3
    orc = OracleSolver(pr.d, pr.np_, pr.n, 2, blocks, pr.prolong, omega=omega, sweeps=k, smoother="as")
    x = orc.smooth(0, pr.b)
    C, np_ = blocks.shape[1], pr.np_
    dinv_b = np.concatenate([np.linalg.solve(blocks[0, K], pr.b[K * np_:(K + 1) * np_]) for K in range(C)])
    ref = (1.0 - (1.0 - 2 * omega) ** k) * dinv_b
    assert np.abs(x - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("m", [0, 4])
def test_schwarz_smoothed_kcycle_matches_dense_lu(m):
    pr = workload("sipg3d_p2_8cube").make(0)
    A = dense_matrix(pr.blocks, pr.nbr)
    xs = np.linalg.solve(A, pr.b)
    x, info = _solver(pr, smoother="as", omega=0.5, sweeps=2, async_smooth=m).solve(pr.b, rtol=1e-10)
    assert info["status"] == ORC_OK
    assert np.linalg.norm(pr.b - A @ x) <= 1e-10 * np.linalg.norm(pr.b)
    assert np.linalg.norm(x - xs) <= 1e-8 * np.linalg.norm(xs)


def test_schwarz_openmp_build_gives_bitwise_the_serial_results():
    import oracle
    oracle.threads(4)
    pr = make_problem(3, 2, (8, 8, 8), 3, seed=4)
    out = [_solver(pr, smoother="as", omega=0.5, sweeps=2, openmp=o).solve(pr.b, rtol=1e-10)[0]
           for o in (False, True)]
    assert np.array_equal(out[0], out[1])
