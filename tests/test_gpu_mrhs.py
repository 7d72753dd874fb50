"""Parity of the batched multi-right-hand-side path (through the C interface) with the
oracle, column by column.

Each column of a batched solve is an independent K-cycle that shares operator
applications with the others, so each column must match the oracle's single solve of
that column: a true relative residual <= 1e-10 and a solution within 1e-8 (relative).
Batched kernels: the FP64 block SpMM agrees with the oracle to rounding; the block-Jacobi
smoother agrees to rounding in FP64.  On the tensor cores it agrees to about TF32
precision: 2^-11 per product for one product, or FP32-level with the three-product
split.  BF16-stored inverses give about 2^-9.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2512_08728_gb300 as pkg
from oracle import OracleSolver
from workloads import make_problem, workload

pytestmark = pytest.mark.gpu

# batched solves whose columns the oracle re-evaluates against 1e-10 stop at 9e-11: the
# GPU confirms each column on a compensated FP64 residual, the oracle evaluates it with
# plain FP64 sums, and the two readings differ by rounding
RTOL_GPU = 9e-11


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _problem(name, seed=0, nrhs=1):
    if name == "ragged_3d_p2":
        return make_problem(3, 2, (6, 6, 2), 2, seed=seed, nrhs=nrhs)
    w = workload(name)
    return make_problem(w.d, w.p, w.n, w.nlevels, length=w.length, nu_kind=w.nu_kind,
                        nu_inside=w.nu_inside, seed=seed, nrhs=nrhs)


CASES = ["sipg2d_p1_16x16", "sipg3d_p1_8x4x4", "sipg2d_p2_32x16", "sipg3d_p2_8cube",
         "sipg3d_p3_8cube_zstretch", "ragged_3d_p2"]


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("nrhs", [32, 5])
def test_batched_operator_matches_oracle(name, nrhs):
    pr = _problem(name)
    orc = OracleSolver.from_problem(pr)
    s = pkg.KCycleSolver(pr, precision="fp64")
    rng = np.random.default_rng(2)
    for lev in range(pr.nlevels - 1):
        X = rng.standard_normal((orc.ndof(lev), nrhs))
        Y = s.apply_multi(lev, X)
        ref = np.stack([orc.apply(lev, X[:, j]) for j in range(nrhs)], axis=1)
        assert _rel(Y, ref) < 1e-13
    s.close()


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("precision,tc_tf32_only,tol", [("fp64", 0, 1e-12), ("mixed", 0, 2e-5),
                                                        ("mixed", 1, 5e-3),
                                                        ("mixed_bf16", 0, 2e-2)])
@pytest.mark.parametrize("nrhs", [32, 5])
def test_batched_smoother_matches_oracle(name, precision, tc_tf32_only, tol, nrhs):
    """Also checks the tensor-core fragment layout: a wrong lane mapping gives O(1) errors."""
    pr = _problem(name)
    orc = OracleSolver.from_problem(pr)
    s = pkg.KCycleSolver(pr, precision=precision, tc_tf32_only=tc_tf32_only)
    rng = np.random.default_rng(3)
    for lev in range(pr.nlevels - 1):
        Rm = rng.standard_normal((orc.ndof(lev), nrhs))
        Z = s.smooth_multi(lev, Rm)
        ref = np.stack([orc.smooth(lev, Rm[:, j]) for j in range(nrhs)], axis=1)
        assert _rel(Z, ref) < tol, (lev, _rel(Z, ref))
    s.close()


def _check_columns(pr, X, info, rtol=1e-10, tol_err=1e-8):
    orc = OracleSolver.from_problem(pr)
    B = pr.b
    for j in range(B.shape[1]):
        x_or, io = orc.solve(B[:, j], rtol=1e-10, maxiter=600)
        assert io["status"] == 0
        # the oracle's plain FP64 residual of x carries its own rounding (the solver's
        # stopping test uses a compensated residual): allow 10 % on the re-evaluation
        rel = np.linalg.norm(B[:, j] - orc.apply(0, X[:, j])) / np.linalg.norm(B[:, j])
        assert rel <= 1.1 * rtol, (j, rel)
        assert np.linalg.norm(X[:, j] - x_or) <= tol_err * np.linalg.norm(x_or), j
    assert info["rel_res"] <= rtol


@pytest.mark.parametrize("name,nrhs", [("sipg2d_p1_16x16", 32), ("sipg3d_p2_8cube", 8),
                                       ("ragged_3d_p2", 5), ("sipg3d_p3_8cube_zstretch", 3),
                                       ("sipg2d_p2_32x16", 12)])
@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_bf16"])
def test_batched_solve_matches_oracle_per_column(name, nrhs, precision):
    pr = _problem(name, nrhs=nrhs)
    s = pkg.KCycleSolver(pr, precision=precision)
    X, info = s.solve(pr.b, rtol=RTOL_GPU, maxiter=2000)
    s.close()
    assert info["status"] == 0, info
    assert X.shape == pr.b.shape
    _check_columns(pr, X, info)


def test_batched_columns_equal_single_solves_and_device_inputs():
    pr = _problem("sipg3d_p2_8cube", seed=4, nrhs=6)
    s = pkg.KCycleSolver(pr, precision="mixed")
    Xh, info_h = s.solve(pr.b, rtol=RTOL_GPU, maxiter=2000)
    Bd = torch.from_numpy(pr.b).cuda()
    Xd, info_d = s.solve(Bd, rtol=RTOL_GPU, maxiter=2000)
    assert info_h["status"] == 0 and info_d["status"] == 0
    # host and device inputs run the same kernels on the same data
    assert np.array_equal(Xh, Xd.cpu().numpy())
    for j in range(pr.b.shape[1]):
        xj, ij = s.solve(np.ascontiguousarray(pr.b[:, j]), rtol=RTOL_GPU, maxiter=2000)
        assert ij["status"] == 0
        assert np.linalg.norm(Xh[:, j] - xj) <= 1e-8 * np.linalg.norm(xj)
    t = s.mrhs_tuning()
    assert t["nrhs"] == 6 and t["spmm_warps"] in (4, 8) and t["lcap0"] >= 6
    s.close()


def test_batched_masks_and_degenerate_columns():
    """A zero column, and a column that starts at its solution (below the absolute
    tolerance), are inactive from the start and keep x0 exactly; the others solve."""
    pr = _problem("sipg3d_p2_8cube", seed=6, nrhs=4)
    B = pr.b.copy()
    B[:, 1] = 0.0
    orc = OracleSolver.from_problem(pr)
    x2, _ = orc.solve(B[:, 2], rtol=1e-12, maxiter=600)
    X0 = np.zeros_like(B)
    X0[:, 2] = x2
    atol = 1e-11 * np.linalg.norm(B, axis=0).max()
    assert np.linalg.norm(B[:, 2] - orc.apply(0, x2)) < atol
    s = pkg.KCycleSolver(pr, precision="fp64")
    X, info = s.solve(B, x0=X0, rtol=1e-10, atol=atol, maxiter=2000)
    assert info["status"] == 0, info
    assert np.all(X[:, 1] == 0.0)
    assert np.array_equal(X[:, 2], x2)
    for j in (0, 3):
        rel = np.linalg.norm(B[:, j] - orc.apply(0, X[:, j])) / np.linalg.norm(B[:, j])
        assert rel <= 1.1e-10
    # nrhs beyond 32 is rejected
    with pytest.raises(pkg.KcmgError):
        s.solve(np.zeros((pr.ndof, 33)), rtol=1e-10)
    s.close()


def test_batched_adjoint_equals_forward_for_symmetric_operator():
    pr = _problem("sipg3d_p1_8x4x4", seed=7, nrhs=4)
    s = pkg.KCycleSolver(pr, precision="fp64")
    X, i1 = s.solve(pr.b, rtol=RTOL_GPU, maxiter=2000)
    L, i2 = s.solve(pr.b, rtol=RTOL_GPU, maxiter=2000, adjoint=True)
    s.close()
    assert i1["status"] == 0 and i2["status"] == 0
    assert np.linalg.norm(X - L) <= 1e-9 * np.linalg.norm(X)


@pytest.mark.parametrize("name,nrhs,m,precision", [("sipg3d_p2_8cube", 6, 3, "fp64"),
                                                   ("sipg2d_p2_32x16", 5, 2, "mixed"),
                                                   ("ragged_3d_p2", 4, 4, "fp64"),
                                                   ("sipg3d_p1_8x4x4", 8, 8, "mixed_bf16")])
def test_batched_task_parallel_cycle_matches_oracle(name, nrhs, m, precision):
    """Level 0 as Alg. AsyncMG in the batched solve: each column against the oracle's
    AsyncMG solve of that column."""
    pr = _problem(name, nrhs=nrhs)
    s = pkg.KCycleSolver(pr, precision=precision, async_smooth=m)
    X, info = s.solve(pr.b, rtol=RTOL_GPU, maxiter=2000)
    s.close()
    assert info["status"] == 0, info
    orc = OracleSolver.from_problem(pr, async_smooth=m)
    for j in range(nrhs):
        x_or, io = orc.solve(pr.b[:, j], rtol=1e-10, maxiter=2000)
        assert io["status"] == 0
        rel = np.linalg.norm(pr.b[:, j] - orc.apply(0, X[:, j])) / np.linalg.norm(pr.b[:, j])
        assert rel <= 1.1e-10, (j, rel)
        assert np.linalg.norm(X[:, j] - x_or) <= 1e-8 * np.linalg.norm(x_or), j


@pytest.mark.parametrize("nrhs", [1, 4])
def test_short_restart_length_with_long_task_parallel_cycle(nrhs):
    """lmax = 4 with m = 8: one cycle appends 9 vectors, more than lmax.  The level-0 basis
    holds lmax plus one cycle, so the cycle fits, and the level restarts after every cycle.
    Restarting every cycle discards the level-0 basis and the solve barely converges; the
    test checks that it runs, keeps its status and reduces the residual."""
    pr = _problem("sipg3d_p2_8cube", seed=3, nrhs=nrhs)
    s = pkg.KCycleSolver(pr, precision="fp64", lmax=4, async_smooth=8)
    B = pr.b if nrhs > 1 else pr.b.reshape(-1)
    X, info = s.solve(B, rtol=1e-10, maxiter=30)
    s.close()
    assert info["status"] in (0, 1), info
    assert info["rel_res"] < 1.0


def _forced_sweep_check(name, precision, tol, nrhs, kind, solve):
    pr = _problem(name)
    orc = OracleSolver.from_problem(pr)
    s = pkg.KCycleSolver(pr, precision=precision)
    rng = np.random.default_rng(8)
    for lev in range(pr.nlevels - 1):
        Rm = rng.standard_normal((orc.ndof(lev), nrhs))
        Z = s.smooth_multi(lev, Rm)
        ref = np.stack([orc.smooth(lev, Rm[:, j]) for j in range(nrhs)], axis=1)
        assert _rel(Z, ref) < tol, (lev, _rel(Z, ref))
    assert s.mrhs_tuning()["sweep_kernel"] == kind
    s.close()
    if not solve:
        return
    # and a whole batched solve on it, column by column against the oracle
    pm = _problem(name, nrhs=nrhs)
    s = pkg.KCycleSolver(pm, precision=precision)
    X, info = s.solve(pm.b, rtol=RTOL_GPU, maxiter=2000)
    assert s.mrhs_tuning()["sweep_kernel"] == kind
    s.close()
    assert info["status"] == 0, info
    _check_columns(pm, X, info)


@pytest.mark.parametrize("name", ["sipg3d_p2_8cube", "ragged_3d_p2", "sipg3d_p3_8cube_zstretch"])
@pytest.mark.parametrize("precision,tol", [("mixed", 2e-5), ("mixed_bf16", 2e-2)])
@pytest.mark.parametrize("nrhs", [32, 6])
def test_bulk_copy_tensor_core_sweep_matches_oracle(name, precision, tol, nrhs, monkeypatch):
    """The tensor-core sweep with every cell's blocks, inverse, residual and neighbour slabs
    staged by double-buffered 1-D bulk copies (forced on every level), against the oracle;
    a batched solve on it at Np = 10 (at Np = 20 the forced kernel runs one warp per SM
    and a solve takes minutes)."""
    monkeypatch.setenv("KCMG_SWEEP", "tcb")
    _forced_sweep_check(name, precision, tol, nrhs, 1.0, solve=name != "sipg3d_p3_8cube_zstretch")


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("precision,tol", [("mixed", 2e-5), ("mixed_bf16", 2e-2)])
@pytest.mark.parametrize("nrhs", [32, 5])
def test_cuda_core_sweep_matches_oracle(name, precision, tol, nrhs, monkeypatch):
    """The register-blocked FP32 sweep on the CUDA cores (forced on every level): every Np of
    the workloads (3, 4, 6, 10, 20: odd Np reads the blocks one entry at a time, Np = 20
    gives a warp one cell), an odd column count (one column at a time) and 32, against the
    oracle's FP64 sweeps; a batched solve on the 3-D p = 2 cases."""
    monkeypatch.setenv("KCMG_SWEEP", "simt")
    _forced_sweep_check(name, precision, tol, nrhs, 2.0,
                        solve=name in ("sipg3d_p2_8cube", "ragged_3d_p2"))
