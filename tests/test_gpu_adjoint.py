"""Adjoint gradients of the solve (torch.autograd.Function with a hand-written backward)
against central finite differences and against the oracle's adjoint gradient."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2512_08728_gb300 as pkg
from oracle import OracleSolver, grad_lognu
from paper_2512_08728_gb300.autograd import KCycleSolve, SolveOptions, SWIPOperator
from workloads import make_problem
from workloads.sipg import assemble

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()


def _setup(n=(8, 8, 8), levels=3, seed=3, rtol=1e-11):
    pr = make_problem(3, 2, n, levels, nu_kind="lognormal", seed=seed)
    # target from a second seeded coefficient field (same law)
    pt = make_problem(3, 2, n, levels, nu_kind="lognormal", seed=seed + 1)
    op = SWIPOperator(pr, options=SolveOptions(rtol=rtol))
    b = torch.from_numpy(pr.b).cuda()
    ut = op.solve(pt.nu, b)
    return pr, op, b, ut


def _check_against_fd(pr, op, b, ut, nfd, seed=0, fd_atol=2e-12, cell_tol=1e-5, h_dir=1e-2):
    """Adjoint gradient vs central finite differences of L(log nu) = 0.5 ||u - u_t||^2.

    Fourth-order central differences with h = 1e-2 (truncation ~h^4 L^(5) / 30): a
    two-point difference with h = 1e-6 amplifies the solve's attainable accuracy
    (~2e-13 ||b||) by 1/(2h), which leaves ~1e-3 of noise in FD itself."""
    log_nu = torch.from_numpy(np.log(pr.nu)).cuda().requires_grad_(True)
    bb = b.clone().requires_grad_(True)
    u = KCycleSolve.apply(bb, log_nu, op)
    L = 0.5 * torch.sum((u - ut) ** 2)
    L.backward()
    g = log_nu.grad.cpu().numpy()
    gb = bb.grad.cpu().numpy()
    u0 = u.detach()
    bnorm = float(torch.linalg.vector_norm(b))
    rng = np.random.default_rng(seed)
    cells = rng.choice(pr.ncells, nfd, replace=False)

    def loss(lognu_np, rhs=b):
        # warm start from u; an absolute stop just above the FP64 floor of the operator
        # (fd_atol ||b||); a solve that ends on the floor must still be within 5x of it
        x = op.solve(np.exp(lognu_np), rhs, x0=u0, rtol=0.0, atol=fd_atol * bnorm, strict=False,
                     maxiter=2000)
        info = op.last_info
        assert info["rel_res"] * info["res0"] <= 5 * fd_atol * bnorm, info
        return 0.5 * float(torch.sum((x - ut) ** 2))

    base = np.log(pr.nu)

    def fd(direction, h=1e-2):
        f = lambda t: loss(base + t * direction)
        return (8 * (f(h) - f(-h)) - (f(2 * h) - f(-2 * h))) / (12 * h)

    fds = []
    for K in cells:
        e = np.zeros_like(base)
        e[K] = 1.0
        fds.append(fd(e))
    fds = np.array(fds)
    assert np.abs(g[cells] - fds).max() <= cell_tol * np.abs(fds).max(), (g[cells], fds)
    # one directional derivative along a random direction over all cells
    d = rng.standard_normal(pr.ncells)
    fdd = fd(d, h_dir)
    assert abs(float(g @ d) - fdd) <= 1e-5 * abs(fdd), (float(g @ d), fdd)
    # dL/db = lambda: L is quadratic in b, so a central difference is exact up to rounding
    i = int(rng.integers(pr.ndof))
    db = torch.zeros_like(b)
    db[i] = float(torch.max(torch.abs(b)))
    lp = loss(base, b + db)
    lm = loss(base, b - db)
    assert abs((lp - lm) / (2 * db[i].item()) - gb[i]) <= 1e-5 * np.abs(gb).max()


def test_gradient_matches_central_differences():
    _check_against_fd(*_setup(), nfd=8)


def test_gradient_fd_32cube_lognormal():
    """The adjoint workload at full size: 32^3 p=2 (327,680 DOFs), 4 levels, log nu ~ N(0,1)
    plus ln 1000 in the ball, target field from the next seed: 6 random cells and one
    random direction over all cells (every cell is checked against the oracle's adjoint
    gradient below)."""
    # The FP64 floor of this operator is near 2e-11 relative, so solves stop at 1e-10.
    # A single cell moves L by ~1e-9 per unit log nu; at h = 1e-2 the solve floor leaves
    # ~5e-4 of noise in those differences, so the cells are checked at 2e-3.  The random
    # direction over all 32,768 cells moves L ~180x more and is checked at 1e-5 (h = 2e-2,
    # truncation ~h^4/30 relative).
    _check_against_fd(*_setup(n=(32, 32, 32), levels=4, seed=0, rtol=1e-10), nfd=6, fd_atol=2e-11,
                      cell_tol=2e-3, h_dir=2e-2)


def _oracle_gradient_check(n, levels, seed, rtol, tol):
    """dL/dlog nu of the GPU path (KCycleSolve forward + hand-written adjoint backward)
    against the oracle's own gradient: the oracle solves the target u_t = A(nu_t)^{-1} b,
    then u = A(nu)^{-1} b and A^T lambda = u - u_t, and evaluates -lambda^T (dA/dlog nu_K) u
    per cell.  Every oracle input is generated data or the oracle's own result."""
    pr = make_problem(3, 2, n, levels, nu_kind="lognormal", seed=seed)
    pt = make_problem(3, 2, n, levels, nu_kind="lognormal", seed=seed + 1)
    kw = dict(async_smooth=8, lmax=200, openmp=True)
    ut, it = OracleSolver.from_problem(pt, **kw).solve(pr.b, rtol=rtol, maxiter=2000)
    assert it["status"] == 0
    uo, iu = OracleSolver.from_problem(pr, **kw).solve(pr.b, rtol=rtol, maxiter=2000)
    assert iu["status"] == 0
    lam, il = OracleSolver.from_problem(pr, transpose=True, **kw).solve(uo - ut, rtol=rtol, maxiter=2000)
    assert il["status"] == 0
    go = grad_lognu(pr, pr.nu, lam, uo)
    op = SWIPOperator(pr, options=SolveOptions(rtol=rtol))
    log_nu = torch.from_numpy(np.log(pr.nu)).cuda().requires_grad_(True)
    u = KCycleSolve.apply(torch.from_numpy(pr.b).cuda(), log_nu, op)
    L = 0.5 * torch.sum((u - torch.from_numpy(ut).cuda()) ** 2)
    L.backward()
    g = log_nu.grad.cpu().numpy()
    err = np.abs(g - go).max() / np.abs(go).max()
    assert err <= tol, err


def test_gradient_matches_oracle_adjoint():
    _oracle_gradient_check((8, 8, 4), 2, 5, 1e-10, 1e-6)


def test_gradient_32cube_lognormal_matches_oracle_adjoint():
    """The adjoint workload at full size: 32^3 p=2 (327,680 DOFs), 4 levels, log nu ~ N(0,1)
    plus ln 1000 in the ball, target field from the next seed: every cell's dL/dlog nu
    within 1e-5 of max |g| of the oracle's adjoint gradient."""
    _oracle_gradient_check((32, 32, 32), 4, 0, 1e-10, 1e-5)
