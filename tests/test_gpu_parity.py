"""Parity of the CUDA path (through the C interface) with the CPU oracle.

Tolerances: FP64 kernels agree with the oracle to rounding (1e-12 relative to the largest
entry); FP32 kernels to 1e-5; whole solves reach a true FP64 relative residual <= 1e-10
and a solution within 1e-8 (relative, 2-norm) of the oracle's solution.
"""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2512_08728_gb300 as pkg
from oracle import OracleSolver, grad_lognu
from workloads import dense_matrix, make_problem, workload

pytestmark = pytest.mark.gpu

# GPU solves whose true residual the oracle re-evaluates against 1e-10 stop at 9e-11.  The
# GPU tests convergence on a compensated FP64 residual; the oracle evaluates the same
# residual with plain FP64 sums.  The two readings differ by rounding (measured 1.3e-13
# relative), so a solve stopped exactly at 1e-10 can read just above it in the oracle.
RTOL_GPU = 9e-11

SMALL = ["sipg2d_p1_16x16", "sipg3d_p1_8x4x4", "sipg2d_p2_32x16", "sipg3d_p2_8cube",
         "sipg3d_p3_8cube_zstretch"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _problem(name, seed=0):
    if name == "ragged_3d_p2":
        return make_problem(3, 2, (6, 6, 2), 2, seed=seed)
    if name == "sipg2d_p1_32x32_5lev":   # levels 0..3 iterate: deep coarse recursion
        return make_problem(2, 1, (32, 32), 5, seed=seed)
    return workload(name).make(seed)


@pytest.mark.parametrize("name", SMALL + ["ragged_3d_p2"])
def test_operator_galerkin_and_transfers(name):
    pr = _problem(name)
    orc = OracleSolver.from_problem(pr)
    s = pkg.KCycleSolver(pr, precision="mixed")
    rng = np.random.default_rng(1)
    for lev in range(pr.nlevels):
        assert _rel(s.blocks(lev), orc.blocks(lev)) < 1e-13
        x = rng.standard_normal(orc.ndof(lev))
        y = orc.apply(lev, x)
        assert _rel(s.apply(lev, x, op=0), y) < 1e-13
        assert _rel(s.apply(lev, x, op=1), y) < 2e-6
        if lev + 1 < pr.nlevels:
            r = rng.standard_normal(orc.ndof(lev))
            zc = rng.standard_normal(orc.ndof(lev + 1))
            assert _rel(s.restrict(lev, r), orc.restrict(lev, r)) < 1e-5
            assert _rel(s.prolong(lev, zc), orc.prolong(lev, zc)) < 1e-5
    s.close()


@pytest.mark.parametrize("name", SMALL + ["ragged_3d_p2"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 3e-5), ("mixed_bf16", 2e-2)])
def test_block_jacobi_smoother(name, precision, tol):
    pr = _problem(name)
    orc = OracleSolver.from_problem(pr)
    s = pkg.KCycleSolver(pr, precision=precision)
    rng = np.random.default_rng(2)
    for lev in range(pr.nlevels - 1):
        r = rng.standard_normal(orc.ndof(lev))
        assert _rel(s.smooth(lev, r), orc.smooth(lev, r)) < tol
    s.close()


@pytest.mark.parametrize("name", SMALL)
def test_fp64_transfers_and_coarse_solve(name):
    pr = _problem(name)
    orc = OracleSolver.from_problem(pr)
    s = pkg.KCycleSolver(pr, precision="fp64")
    rng = np.random.default_rng(3)
    for lev in range(pr.nlevels - 1):
        r = rng.standard_normal(orc.ndof(lev))
        zc = rng.standard_normal(orc.ndof(lev + 1))
        assert _rel(s.restrict(lev, r), orc.restrict(lev, r)) < 1e-13
        assert _rel(s.prolong(lev, zc), orc.prolong(lev, zc)) < 1e-13
    rc = rng.standard_normal(orc.ndof(pr.nlevels - 1))
    assert _rel(s.coarse_solve(rc), orc.coarse_solve(rc)) < 1e-9
    s.close()


@pytest.mark.parametrize("name", ["sipg2d_p1_16x16", "sipg3d_p2_8cube", "ragged_3d_p2"])
def test_residual_minimization_sequence(name):
    """Alg. 1 on the GPU (classical Gram-Schmidt with a reorthogonalisation test) against
    the oracle's modified Gram-Schmidt, on the same corrections: smoother outputs, coarse
    corrections and random vectors, including a linearly dependent one (discarded)."""
    pr = _problem(name)
    orc = OracleSolver.from_problem(pr)
    s = pkg.KCycleSolver(pr, precision="fp64")
    rng = np.random.default_rng(4)
    x0 = rng.uniform(-1, 1, pr.ndof)
    orc.rm_begin(0, pr.b, x0)
    r = pr.b - orc.apply(0, x0)
    zs = []
    for k in range(24):
        kind = k % 4
        if kind == 0:
            z = orc.smooth(0, r)
        elif kind == 1:
            z = orc.prolong(0, orc.restrict(0, r))
        elif kind == 2:
            z = rng.uniform(-1, 1, pr.ndof)
        else:
            z = 2.0 * zs[-1]                  # dependent: must be discarded
        zs.append(z)
        rc, xo, r, lo = orc.rm_call(0, z)
    xg, rg, lg = s.rm_sequence(0, pr.b, x0, np.stack(zs))
    assert lg == lo
    # rounding of the two recursions (incremental on the GPU, from scratch in the oracle)
    # scales with the initial residual b - A x0, which a random x0 makes large
    scale = np.linalg.norm(pr.b - orc.apply(0, x0))
    assert np.linalg.norm(rg - r) <= 1e-10 * scale
    assert np.linalg.norm(xg - xo) <= 1e-7 * np.linalg.norm(xo)
    s.close()


def _check_solution(pr, x, info, x_or, tol_err=1e-8):
    # true residual evaluated by the oracle's operator, independent of the GPU
    orc = OracleSolver.from_problem(pr)
    rel = np.linalg.norm(pr.b - orc.apply(0, x)) / np.linalg.norm(pr.b)
    assert rel <= 1e-10, rel
    assert info["rel_res"] <= 1e-10
    assert np.linalg.norm(x - x_or) <= tol_err * np.linalg.norm(x_or)


@pytest.mark.parametrize("name", SMALL + ["ragged_3d_p2", "sipg2d_p1_32x32_5lev"])
@pytest.mark.parametrize("use_graph,persistent", [(False, False), (True, False), (False, True),
                                                  (True, True)])
def test_fp64_solve_matches_oracle(name, use_graph, persistent):
    pr = _problem(name)
    x_or, info_or = OracleSolver.from_problem(pr).solve(pr.b, rtol=1e-10, maxiter=400)
    assert info_or["status"] == 0
    s = pkg.KCycleSolver(pr, precision="fp64", use_graph=use_graph, coarse_persistent=persistent)
    x, info = s.solve(pr.b, rtol=RTOL_GPU, maxiter=400)
    s.close()
    assert info["status"] == 0, info
    _check_solution(pr, x, info, x_or)
    # the residual history is monotone within runs of RM calls
    h, t = info["hist"], info["hist_type"]
    assert np.all(np.diff(h)[t[1:] != 4] <= 1e-12 * h[0])


@pytest.mark.parametrize("name", SMALL + ["ragged_3d_p2", "sipg2d_p1_32x32_5lev"])
@pytest.mark.parametrize("precision", ["mixed", "mixed_bf16"])
@pytest.mark.parametrize("persistent", [False, True])
def test_mixed_precision_solve_matches_fp64_oracle(name, precision, persistent):
    pr = _problem(name)
    x_or, _ = OracleSolver.from_problem(pr).solve(pr.b, rtol=1e-10, maxiter=400)
    s = pkg.KCycleSolver(pr, precision=precision, use_graph=True, coarse_persistent=persistent)
    x, info = s.solve(pr.b, rtol=RTOL_GPU, maxiter=2000)
    s.close()
    assert info["status"] == 0, info
    _check_solution(pr, x, info, x_or)
    assert info["refinements"] >= 1


@pytest.mark.parametrize("persistent", [False, True])
def test_graph_and_eager_are_bitwise_identical_and_repeatable(persistent):
    pr = make_problem(3, 2, (8, 8, 8), 3, seed=5)
    out = []
    for g in (False, True, True):
        s = pkg.KCycleSolver(pr, precision="fp64", use_graph=g, coarse_persistent=persistent)
        x, info = s.solve(pr.b, rtol=1e-10)
        x2, _ = s.solve(pr.b, rtol=1e-10)
        s.close()
        assert np.array_equal(x, x2)
        out.append(x)
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[1], out[2])


def test_device_and_host_inputs_agree():
    pr = workload("sipg3d_p1_8x4x4").make(0)
    s = pkg.KCycleSolver(pr, precision="fp64")
    xh, _ = s.solve(pr.b, rtol=1e-10)
    xd, _ = s.solve(torch.from_numpy(pr.b).cuda(), rtol=1e-10)
    s.close()
    assert np.array_equal(xh, xd.cpu().numpy())


def test_degenerate_inputs():
    pr = workload("sipg2d_p1_16x16").make(0)
    s = pkg.KCycleSolver(pr, precision="fp64")
    x, info = s.solve(np.zeros(pr.ndof), rtol=1e-10)          # b = 0: x = 0 at once
    assert info["status"] == 0 and info["iters"] == 0 and not np.any(x)
    xs, _ = s.solve(pr.b, rtol=1e-10)
    x, info = s.solve(pr.b, x0=xs, rtol=0.0, atol=1e-6)        # x0 already converged
    assert info["status"] == 0 and info["iters"] == 0 and np.array_equal(x, xs)
    x, info = s.solve(pr.b, rtol=1e-10, maxiter=0)              # no iterations allowed
    assert info["status"] == 1 and np.array_equal(x, np.zeros(pr.ndof))
    x, info = s.solve(pr.b, rtol=1e-14, maxiter=2)              # not converged, no worse
    assert info["status"] == 1 and info["rel_res"] < 1.0
    bad = pr.b.copy()
    bad[7] = np.nan
    with pytest.raises(pkg.KcmgError) as e:
        s.solve(bad, rtol=1e-10)
    assert e.value.status == 3
    s.close()


def test_setup_rejects_bad_arguments():
    pr = workload("sipg2d_p1_16x16").make(0)
    p = pkg.kcmg_default_params(pr.d, pr.np_, (16, 10), 3)      # 10 not divisible by 4
    with pytest.raises(pkg.KcmgError) as e:
        pkg.kcmg_setup(p, pr.blocks, pr.prolong)
    assert e.value.status == 5
    blocks = pr.blocks.copy()
    blocks[0, 3] = 0.0                                          # singular diagonal block
    p = pkg.kcmg_default_params(pr.d, pr.np_, pr.n, 3)
    with pytest.raises(pkg.KcmgError) as e:
        pkg.kcmg_setup(p, blocks, pr.prolong)
    assert e.value.status == 4


def test_persistent_and_per_kernel_coarse_cycles_agree():
    """Both coarse-cycle implementations run the same algorithm; they sum reductions in
    different orders.  Near the attainable accuracy the adaptive level criteria and the
    restarts turn that rounding into different trajectories, so cycle counts are compared
    only loosely; both converge and the solutions agree to the solve tolerance."""
    pr = make_problem(3, 2, (16, 16, 8), 4, seed=2)
    res = []
    for persistent in (False, True):
        s = pkg.KCycleSolver(pr, precision="fp64", coarse_persistent=persistent)
        x, info = s.solve(pr.b, rtol=RTOL_GPU, maxiter=400)
        s.close()
        assert info["status"] == 0
        res.append((x, info))
    (x0, i0), (x1, i1) = res
    assert np.linalg.norm(x0 - x1) <= 1e-8 * np.linalg.norm(x0)
    assert max(i0["iters"], i1["iters"]) <= 2 * min(i0["iters"], i1["iters"])


def test_adjoint_solve():
    pr = workload("sipg3d_p1_8x4x4").make(0)
    s = pkg.KCycleSolver(pr, precision="fp64")
    x, _ = s.solve(pr.b, rtol=1e-10)
    lam, info = s.solve(pr.b, rtol=1e-10, adjoint=True)        # symmetric: same hierarchy
    assert np.array_equal(x, lam) and info["status"] == 0
    s.close()
    blocks = pr.blocks.copy()
    rng = np.random.default_rng(4)
    for sl in range(1, blocks.shape[0]):
        blocks[sl] *= 1.0 + 0.2 * rng.uniform(-1, 1, blocks.shape[1])[:, None, None]
    A = dense_matrix(blocks, pr.nbr)
    pr2 = make_problem(3, 1, (8, 4, 4), 3)
    pr2.blocks = blocks
    s = pkg.KCycleSolver(pr2, precision="fp64")
    lam, info = s.solve(pr.b, rtol=1e-11, adjoint=True)
    s.close()
    ref = np.linalg.solve(A.T, pr.b)
    assert info["status"] == 0
    assert np.linalg.norm(lam - ref) <= 1e-8 * np.linalg.norm(ref)


def test_gradient_kernel_matches_oracle():
    pr = make_problem(3, 2, (8, 8, 4), 2, nu_kind="lognormal", seed=3)
    s = pkg.KCycleSolver(pr, precision="fp64")
    rng = np.random.default_rng(6)
    lam, u = rng.standard_normal(pr.ndof), rng.standard_normal(pr.ndof)
    g = s.grad_lognu(pr.nu, pr.ref, lam, u)
    s.close()
    assert _rel(g, grad_lognu(pr, pr.nu, lam, u)) < 1e-12


# ------------------------------------------------------------------ Alg. AsyncMG on the GPU
@pytest.mark.parametrize("name", SMALL + ["ragged_3d_p2", "sipg2d_p1_32x32_5lev"])
@pytest.mark.parametrize("m", [1, 3])
@pytest.mark.parametrize("use_graph,persistent", [(False, False), (True, False), (True, True)])
def test_task_parallel_cycle_matches_oracle(name, m, use_graph, persistent):
    """Level 0 as Alg. AsyncMG with m smoother steps per cycle; the coarse path runs on a
    second stream.  The solution must match the oracle's AsyncMG solve."""
    pr = _problem(name)
    x_or, info_or = OracleSolver.from_problem(pr, async_smooth=m).solve(pr.b, rtol=1e-10, maxiter=2000)
    assert info_or["status"] == 0
    s = pkg.KCycleSolver(pr, precision="fp64", use_graph=use_graph, coarse_persistent=persistent,
                         async_smooth=m)
    x, info = s.solve(pr.b, rtol=RTOL_GPU, maxiter=2000)
    s.close()
    assert info["status"] == 0, info
    _check_solution(pr, x, info, x_or)


@pytest.mark.parametrize("m", [1, 2, 4])
@pytest.mark.parametrize("persistent", [False, True])
def test_task_parallel_first_cycles_follow_the_oracle(m, persistent):
    """The residual history of the first cycles (m smoother RMs, then the coarse RM from
    the cycle-start residual) agrees with the oracle's, entry by entry."""
    pr = make_problem(3, 2, (8, 8, 8), 3, seed=9)
    _, io = OracleSolver.from_problem(pr, async_smooth=m).solve(pr.b, rtol=1e-14, maxiter=3)
    s = pkg.KCycleSolver(pr, precision="fp64", use_graph=True, coarse_persistent=persistent,
                         async_smooth=m)
    _, info = s.solve(pr.b, rtol=1e-14, maxiter=3)
    s.close()
    n = 1 + 3 * (m + 1)
    assert list(info["hist_type"][:n]) == list(io["hist_type"][:n])
    assert list(info["hist_type"][1:m + 2]) == [1] * m + [2]
    h, ho = info["hist"][:n], io["hist"][:n]
    assert np.all(np.abs(h - ho) <= 1e-9 * ho[0]), (h, ho)


@pytest.mark.parametrize("precision", ["mixed", "mixed_bf16"])
def test_task_parallel_mixed_precision(precision):
    pr = _problem("sipg3d_p2_8cube")
    x_or, _ = OracleSolver.from_problem(pr, async_smooth=2).solve(pr.b, rtol=1e-10, maxiter=2000)
    s = pkg.KCycleSolver(pr, precision=precision, use_graph=True, async_smooth=2)
    x, info = s.solve(pr.b, rtol=RTOL_GPU, maxiter=2000)
    s.close()
    assert info["status"] == 0, info
    _check_solution(pr, x, info, x_or)


def test_task_parallel_graph_and_eager_are_bitwise_identical():
    pr = make_problem(3, 2, (8, 8, 8), 3, seed=5)
    out = []
    for g in (False, True):
        s = pkg.KCycleSolver(pr, precision="fp64", use_graph=g, async_smooth=3)
        x, _ = s.solve(pr.b, rtol=1e-10)
        s.close()
        out.append(x)
    assert np.array_equal(out[0], out[1])


# ------------------------------------------------------------------ the benchmark's level layout
def _layout_solve(pr, m, rows_max, monkeypatch, lmax=200, rtol=RTOL_GPU):
    """Solve with the persistent coarse kernel taking the levels from the first one with at
    most rows_max rows (set through KCMG_PERSISTENT_ROWS at setup); the levels above it run
    one kernel per step under nested conditional graph nodes."""
    monkeypatch.setenv("KCMG_PERSISTENT_ROWS", str(rows_max))
    s = pkg.KCycleSolver(pr, precision="fp64", use_graph=True, coarse_persistent=True,
                         async_smooth=m, lmax=lmax)
    monkeypatch.delenv("KCMG_PERSISTENT_ROWS")
    x, info = s.solve(pr.b, rtol=rtol, maxiter=2000)
    rep = s.kernel_report()
    s.close()
    return x, info, rep


@pytest.mark.parametrize("m", [0, 8])
def test_benchmark_level_layout_matches_oracle(m, monkeypatch):
    """The 64^3 benchmark runs level 1 as full-occupancy kernels under a nested conditional
    node and levels 2-3 in the persistent kernel, inside the task-parallel (m = 8, Alg.
    AsyncMG) or multiplicative (m = 0, Alg. 2) level-0 cycle.  The same layout on 16^3
    cells, p = 2, 5 levels (l1 5,120 rows nested; l2 640 and l3 80 rows persistent; l4
    direct), against the oracle's solve of the same cycle."""
    pr = make_problem(3, 2, (16, 16, 16), 5, seed=3)
    x, info, rep = _layout_solve(pr, m, 1000, monkeypatch)
    assert info["status"] == 0, info
    lv = rep["coarse_level_ms"]
    assert lv[1] == 0.0 and lv[2] > 0.0 and lv[3] > 0.0     # the layout really ran
    x_or, io = OracleSolver.from_problem(pr, async_smooth=m, lmax=200, openmp=True).solve(
        pr.b, rtol=1e-10, maxiter=2000)
    assert io["status"] == 0
    _check_solution(pr, x, info, x_or)


def test_benchmark_level_layout_32cube_task_parallel_matches_oracle(monkeypatch):
    """32^3 cells, p = 2 (327,680 DOFs), 5 levels, Alg. AsyncMG with m = 8 and lmax = 200 as
    the benchmark: level 1 (40,960 rows) nested, levels 2-3 persistent, level 4 direct.

    Both sides solve to 3e-11.  At this size (condition number near 1e7) two iterates that
    both meet a relative residual of 1e-10 can differ by more than 1e-8: measured 1.3e-8.
    The difference is bounded by the sum of their errors, each at most ||A^-1|| times its
    residual, so a tighter stop on both sides keeps it inside the 1e-8 bound."""
    pr = make_problem(3, 2, (32, 32, 32), 5, seed=0)
    x, info, rep = _layout_solve(pr, 8, 10000, monkeypatch, rtol=3e-11)
    assert info["status"] == 0, info
    lv = rep["coarse_level_ms"]
    assert lv[1] == 0.0 and lv[2] > 0.0
    x_or, io = OracleSolver.from_problem(pr, async_smooth=8, lmax=200, openmp=True).solve(
        pr.b, rtol=3e-11, maxiter=2000)
    assert io["status"] == 0
    _check_solution(pr, x, info, x_or)


def test_benchmark_workload_at_full_size():
    """The benchmark's workload at full size in its timed launch configuration: 64^3 cells,
    p = 2 (2,621,440 DOFs), 5 levels, FP64, Alg. AsyncMG with m = 12, lmax 400, CUDA graph,
    persistent coarse cycle.
    - Every row of the level-0 operator and of one level-0 smoothing step against the
      oracle.
    - The first cycle's residual history (12 smoother RMs, then the coarse RM) against the
      oracle's first cycle, entry by entry.
    - The whole solve's true residual evaluated by the oracle's FP64 operator.  The oracle's
      own solve of this size takes minutes on the host, so the solution is checked through
      its residual, which bounds it at any size."""
    pr = workload("sipg3d_p2_64cube").make(0)
    m = 12
    orc = OracleSolver.from_problem(pr, async_smooth=m, lmax=400, openmp=True)
    s = pkg.KCycleSolver(pr, precision="fp64", use_graph=True, coarse_persistent=True,
                         async_smooth=m, lmax=400)
    rng = np.random.default_rng(11)
    xr = rng.standard_normal(pr.ndof)
    assert _rel(s.apply(0, xr), orc.apply(0, xr)) < 1e-13
    rr = rng.standard_normal(pr.ndof)
    assert _rel(s.smooth(0, rr), orc.smooth(0, rr)) < 1e-12
    _, io = orc.solve(pr.b, rtol=1e-14, maxiter=1)
    _, i1 = s.solve(pr.b, rtol=1e-14, maxiter=1)
    n = m + 2
    assert list(i1["hist_type"][:n]) == list(io["hist_type"][:n])
    h, ho = i1["hist"][:n], io["hist"][:n]
    assert np.all(np.abs(h - ho) <= 1e-9 * ho[0]), (h, ho)
    x, info = s.solve(pr.b, rtol=RTOL_GPU, maxiter=4000)
    s.close()
    assert info["status"] == 0, info
    rel = np.linalg.norm(pr.b - orc.apply(0, x)) / np.linalg.norm(pr.b)
    assert rel <= 1e-10, rel


# ------------------------------------------------------------------ FP64 refinement, FP32 inner solve
_IR_CASES = ([(n, "ir32", 0, True) for n in SMALL + ["ragged_3d_p2", "sipg2d_p1_32x32_5lev"]]
             + [(n, "ir32", m, pers) for n in ("sipg3d_p2_8cube", "ragged_3d_p2", "sipg2d_p1_32x32_5lev")
                for m, pers in ((0, False), (3, True))]
             + [(n, "ir32_bf16", 0, True) for n in ("sipg2d_p1_16x16", "sipg3d_p2_8cube",
                                                   "sipg3d_p3_8cube_zstretch")])


@pytest.mark.parametrize("name,precision,m,persistent", _IR_CASES)
def test_iterative_refinement_solve_matches_fp64_oracle(name, precision, m, persistent):
    """FP64 outer refinement around a K-cycle run entirely in FP32 (operators, sweeps,
    transfers, bases) with FP64 Gram reductions and coarsest solve: the FP64 true residual
    and the distance to the oracle's FP64 solution meet the FP64 bounds."""
    pr = _problem(name)
    x_or, _ = OracleSolver.from_problem(pr).solve(pr.b, rtol=1e-10, maxiter=400)
    s = pkg.KCycleSolver(pr, precision=precision, use_graph=True, coarse_persistent=persistent,
                         async_smooth=m)
    x, info = s.solve(pr.b, rtol=RTOL_GPU, maxiter=4000)
    s.close()
    assert info["status"] == 0, info
    _check_solution(pr, x, info, x_or)
    assert info["refinements"] >= 1
    h, t = info["hist"], info["hist_type"]
    assert t[0] == 0 and np.all(t[1:] == 6) and len(h) == info["refinements"] + 1
    assert np.all(np.diff(h) < 0)                 # every accepted step lowers the residual


@pytest.mark.parametrize("name", ["sipg2d_p1_16x16", "sipg3d_p2_8cube", "ragged_3d_p2"])
def test_iterative_refinement_components_in_fp32(name):
    """The inner solve's kernels on FP32 vectors against the oracle: operator, sweeps,
    transfers (FP32 rounding), and Alg. 1 on FP32 bases."""
    pr = _problem(name)
    orc = OracleSolver.from_problem(pr)
    s = pkg.KCycleSolver(pr, precision="ir32")
    rng = np.random.default_rng(7)
    for lev in range(pr.nlevels - 1):
        x = rng.standard_normal(orc.ndof(lev))
        assert _rel(s.apply(lev, x, op=1), orc.apply(lev, x)) < 2e-6
        assert _rel(s.smooth(lev, x), orc.smooth(lev, x)) < 3e-5
        zc = rng.standard_normal(orc.ndof(lev + 1))
        assert _rel(s.restrict(lev, x), orc.restrict(lev, x)) < 2e-6
        assert _rel(s.prolong(lev, zc), orc.prolong(lev, zc)) < 2e-6
    x0 = rng.uniform(-1, 1, pr.ndof)
    orc.rm_begin(0, pr.b, x0)
    r = pr.b - orc.apply(0, x0)
    zs = []
    for k in range(8):
        z = orc.smooth(0, r) if k % 2 == 0 else orc.prolong(0, orc.restrict(0, r))
        zs.append(z)
        _, xo, r, lo = orc.rm_call(0, z)
    xg, rg, lg = s.rm_sequence(0, pr.b, x0, np.stack(zs))
    assert lg == lo
    scale = np.linalg.norm(pr.b - orc.apply(0, x0))
    assert np.linalg.norm(rg - r) <= 1e-5 * scale
    s.close()


def test_iterative_refinement_degenerate_inputs():
    pr = workload("sipg2d_p1_16x16").make(0)
    s = pkg.KCycleSolver(pr, precision="ir32")
    x, info = s.solve(np.zeros(pr.ndof), rtol=1e-10)          # b = 0: x = 0 at once
    assert info["status"] == 0 and info["iters"] == 0 and not np.any(x)
    x, info = s.solve(pr.b, rtol=1e-10, maxiter=0)              # no cycles allowed
    assert info["status"] == 1 and np.array_equal(x, np.zeros(pr.ndof))
    xs, _ = s.solve(pr.b, rtol=1e-10)
    x, info = s.solve(pr.b, x0=xs, rtol=0.0, atol=1e-6)         # x0 already converged
    assert info["status"] == 0 and info["refinements"] == 0 and np.array_equal(x, xs)
    with pytest.raises(pkg.KcmgError) as e:                    # batched solves: FP64/mixed only
        s.solve(np.zeros((pr.ndof, 2)), rtol=1e-10)
    assert e.value.status == 5
    s.close()


# ------------------------------------------------------------------ Alg. AS (additive Schwarz)
AS_KW = dict(smoother="as", omega=0.5, sweeps=2)


@pytest.mark.parametrize("name", SMALL + ["ragged_3d_p2"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 3e-5), ("mixed_bf16", 2e-2)])
def test_schwarz_smoother(name, precision, tol):
    """Alg. AS on the two partitions of overlapping 2^d-cell patches, every iterated level,
    against the oracle's Alg. AS (dense local inverses in the smoother's precision)."""
    pr = _problem(name)
    orc = OracleSolver.from_problem(pr, **AS_KW)
    s = pkg.KCycleSolver(pr, precision=precision, **AS_KW)
    rng = np.random.default_rng(12)
    for lev in range(pr.nlevels - 1):
        r = rng.standard_normal(orc.ndof(lev))
        assert _rel(s.smooth(lev, r), orc.smooth(lev, r)) < tol
    s.close()


@pytest.mark.parametrize("name", SMALL + ["ragged_3d_p2", "sipg2d_p1_32x32_5lev"])
@pytest.mark.parametrize("precision", ["fp64", "mixed_bf16"])
@pytest.mark.parametrize("m,persistent", [(0, True), (0, False), (3, True)])
def test_schwarz_smoothed_solve_matches_oracle(name, precision, m, persistent):
    pr = _problem(name)
    x_or, io = OracleSolver.from_problem(pr, async_smooth=m, **AS_KW).solve(pr.b, rtol=1e-10, maxiter=2000)
    assert io["status"] == 0
    s = pkg.KCycleSolver(pr, precision=precision, use_graph=True, coarse_persistent=persistent,
                         async_smooth=m, **AS_KW)
    x, info = s.solve(pr.b, rtol=RTOL_GPU, maxiter=2000)
    s.close()
    assert info["status"] == 0, info
    _check_solution(pr, x, info, x_or)


def test_schwarz_smoother_in_the_refinement_form():
    pr = _problem("sipg3d_p2_8cube")
    x_or, _ = OracleSolver.from_problem(pr, **AS_KW).solve(pr.b, rtol=1e-10, maxiter=400)
    s = pkg.KCycleSolver(pr, precision="ir32", async_smooth=3, **AS_KW)
    x, info = s.solve(pr.b, rtol=RTOL_GPU, maxiter=2000)
    s.close()
    assert info["status"] == 0, info
    _check_solution(pr, x, info, x_or)


# ------------------------------------------------------------------ matrix-free fine coupling
@pytest.mark.parametrize("name", ["sipg2d_p1_16x16", "sipg3d_p2_8cube", "ragged_3d_p2", "sipg3d_p3_8cube_zstretch"])
@pytest.mark.parametrize("precision,tol", [("mixed", 3e-5), ("mixed_bf16", 2e-2)])
def test_matrix_free_fine_sweeps_match_oracle(name, precision, tol):
    """Level-0 FP32 sweeps with the off-diagonal coupling applied from the coefficient field
    and the face reference matrices (gamma_F F_k^{RL}, gamma_F F_k^{LR}) instead of stored
    blocks: against the oracle's Alg. BJ and against the stored-block sweeps."""
    pr = _problem(name)
    orc = OracleSolver.from_problem(pr)
    s_mf = pkg.KCycleSolver(pr, precision=precision, matrix_free=True)
    s_st = pkg.KCycleSolver(pr, precision=precision)
    rng = np.random.default_rng(21)
    for lev in range(pr.nlevels - 1):
        r = rng.standard_normal(orc.ndof(lev))
        z_mf, z_st = s_mf.smooth(lev, r), s_st.smooth(lev, r)
        assert _rel(z_mf, orc.smooth(lev, r)) < tol
        assert _rel(z_mf, z_st) < (2e-6 if precision == "mixed" else 2e-3)
    s_mf.close()
    s_st.close()


@pytest.mark.parametrize("name", ["sipg3d_p2_8cube", "ragged_3d_p2", "sipg2d_p1_32x32_5lev"])
@pytest.mark.parametrize("m", [0, 3])
def test_matrix_free_fine_sweeps_solve_matches_oracle(name, m):
    pr = _problem(name)
    x_or, _ = OracleSolver.from_problem(pr, async_smooth=m).solve(pr.b, rtol=1e-10, maxiter=2000)
    s = pkg.KCycleSolver(pr, precision="mixed_bf16", matrix_free=True, async_smooth=m)
    x, info = s.solve(pr.b, rtol=RTOL_GPU, maxiter=2000)
    s.close()
    assert info["status"] == 0, info
    _check_solution(pr, x, info, x_or)


def test_matrix_free_setup_rejects_a_coefficient_that_does_not_match():
    pr = _problem("sipg3d_p2_8cube")
    shell = dataclasses.replace(pr, nu=pr.nu * np.where(np.arange(pr.ncells) == 5, 1.5, 1.0))
    with pytest.raises(pkg.KcmgError) as e:
        pkg.KCycleSolver(shell, precision="mixed", matrix_free=True)
    assert e.value.status == 5
    with pytest.raises(pkg.KcmgError) as e:                    # FP64 smoother: not served
        pkg.KCycleSolver(pr, precision="fp64", matrix_free=True)
    assert e.value.status == 5
