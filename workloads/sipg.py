"""SIPG discretisation of -div(nu grad u) = f on a Cartesian cell grid (problem input).

The paper solves systems from a symmetric interior penalty (SIP) discontinuous Galerkin
discretisation (Sec. 2, "XDG discretization") of a Poisson problem whose diffusion
coefficient jumps across a spherical interface (Sec. 2, Poisson equation; Sec. 5.1,
benchmark problems).  Cut cells are replaced here by a cell-wise constant coefficient
decided by each cell's centroid, on the unit square/cube.

Discretisation (a reading; the paper gives only "SIP"):
  * basis: L2-orthonormal tensor Legendre polynomials of total degree <= p on each cell,
    Np = C(p+d, d) modes per cell (the N local DOFs of Sec. 2, "XDG discretization");
  * interior faces: weighted averages with weights nu_K'/(nu_K+nu_K'), which equals the
    harmonic mean gamma_F = 2 nu_K nu_K'/(nu_K+nu_K') times the plain arithmetic-average
    SIP face terms with unit coefficient; penalty eta*gamma_F/h_perp, eta = 4(p+1)^2;
  * Dirichlet faces: one-sided terms with nu_K and penalty eta*nu_K/h_perp.
So A = sum_K nu_K V + sum_F gamma_F F_F + sum_{boundary F} nu_K B_F with constant
reference matrices V, F, B; the same matrices give dA/dnu for the adjoint gradient.

Storage (the block-ELL input of the solver): blocks[s][K] is the Np x Np row-major block
coupling test cell K to trial cell nbr(K, s); slot 0 is the diagonal, slots 1..2d the face
neighbours in the order (-x, +x, -y, +y, -z, +z); nbr[K][s-1] = -1 on the boundary (block
zero).  Cells are numbered lexicographically with x fastest; DOF index = K*Np + mode.
"""
from __future__ import annotations

import dataclasses
import math
from itertools import product

import numpy as np
from numpy.polynomial import legendre as npleg


# ----------------------------------------------------------------------------- basis
def modes(d: int, p: int) -> np.ndarray:
    """Multi-indices of the total-degree-<=p tensor Legendre basis, shape (Np, d).

    Ordered by total degree, then by decreasing power of x, then of y."""
    out = []
    for n in range(p + 1):
        for a in product(range(n, -1, -1), repeat=d):
            if sum(a) == n:
                out.append(a)
    return np.array(out, dtype=np.int64).reshape(-1, d)


def _leg(m: int, xi, deriv: int = 0):
    """Orthonormal Legendre polynomial sqrt((2m+1)/2) P_m on [-1, 1] (or a derivative)."""
    c = np.zeros(m + 1)
    c[m] = math.sqrt((2 * m + 1) / 2.0)
    if deriv:
        c = npleg.legder(c, deriv)
    return npleg.legval(xi, c)


def _ref_1d(p: int):
    """1-D reference data on [-1, 1]: stiffness, traces, and child projections."""
    xg, wg = npleg.leggauss(p + 2)
    D1 = np.array([[np.sum(wg * _leg(m, xg, 1) * _leg(n, xg, 1)) for n in range(p + 1)]
                   for m in range(p + 1)])
    tp = np.array([_leg(m, 1.0) for m in range(p + 1)])
    tm = np.array([_leg(m, -1.0) for m in range(p + 1)])
    dp = np.array([_leg(m, 1.0, 1) for m in range(p + 1)])
    dm = np.array([_leg(m, -1.0, 1) for m in range(p + 1)])
    # child c in {0,1} covers coarse coordinate [-1,0] or [0,1]; xi_coarse = (eta + s)/2.
    # Q_c[a][i] = int_child phi_i psi_a dx with both bases orthonormal on their own cell.
    Q = np.zeros((2, p + 1, p + 1))
    for c, s in ((0, -1.0), (1, 1.0)):
        for a in range(p + 1):
            for i in range(p + 1):
                Q[c, a, i] = np.sum(wg * _leg(i, (xg + s) / 2.0) * _leg(a, xg)) / math.sqrt(2.0)
    return D1, tp, tm, dp, dm, Q


def reference_matrices(d: int, p: int, h, eta: float):
    """Constant matrices of the SWIP form on cells of size h (length-d).

    Returns dict with
      V        (Np, Np)         volume stiffness  int grad phi_b . grad phi_a
      F        (d, 4, Np, Np)   interior face, unit gamma: [LL, LR, RL, RR] where L is the
                                cell on the low side of the face and R the high side;
                                F[k, 1][b, a] = test L mode b, trial R mode a
      B        (d, 2, Np, Np)   Dirichlet face, unit nu: [low face, high face] of a cell
    Row index = test mode, column index = trial mode.
    """
    md = modes(d, p)
    Np = md.shape[0]
    D1, tp, tm, dp, dm, _ = _ref_1d(p)
    h = np.asarray(h, dtype=np.float64)
    V = np.zeros((Np, Np))
    F = np.zeros((d, 4, Np, Np))
    B = np.zeros((d, 2, Np, Np))
    for k in range(d):
        others = [j for j in range(d) if j != k]
        E = np.ones((Np, Np))
        for j in others:
            E *= (md[:, None, j] == md[None, :, j])
        bk = md[:, None, k]  # test index along k (rows)
        ak = md[None, :, k]  # trial index along k (cols)
        g = 2.0 / h[k]
        sg = eta / h[k]
        V += g * g * D1[bk, ak] * E
        F[k, 0] = E * (-0.5 * g * g * (dp[ak] * tp[bk] + dp[bk] * tp[ak]) + sg * g * tp[ak] * tp[bk])
        F[k, 1] = E * (-0.5 * g * g * dm[ak] * tp[bk] + 0.5 * g * g * dp[bk] * tm[ak] - sg * g * tm[ak] * tp[bk])
        F[k, 2] = E * (0.5 * g * g * dp[ak] * tm[bk] - 0.5 * g * g * dm[bk] * tp[ak] - sg * g * tp[ak] * tm[bk])
        F[k, 3] = E * (0.5 * g * g * (dm[ak] * tm[bk] + dm[bk] * tm[ak]) + sg * g * tm[ak] * tm[bk])
        B[k, 0] = E * (g * g * (dm[ak] * tm[bk] + dm[bk] * tm[ak]) + sg * g * tm[ak] * tm[bk])
        B[k, 1] = E * (-g * g * (dp[ak] * tp[bk] + dp[bk] * tp[ak]) + sg * g * tp[ak] * tp[bk])
    # make the form bitwise symmetric: a(u, v) = a(v, u) holds exactly in the stored blocks
    sym = lambda M: 0.5 * (M + M.T)
    V = sym(V)
    for k in range(d):
        F[k, 0], F[k, 3] = sym(F[k, 0]), sym(F[k, 3])
        F[k, 1] = F[k, 2].T.copy()
        B[k, 0], B[k, 1] = sym(B[k, 0]), sym(B[k, 1])
    return {"V": V, "F": F, "B": B}


def prolongation_matrices(d: int, p: int) -> np.ndarray:
    """P[k] (Np x Np): coarse modes -> modes of child k of a 2^d agglomerated cell.

    Child k = cx + 2 cy + 4 cz, c in {0,1} the low/high half in each direction.  P[k][a][i]
    is the coefficient of child mode a in coarse mode i restricted to child k (exact
    injection of nested polynomial spaces = L2 projection); sum_k P[k]^T P[k] = I."""
    md = modes(d, p)
    Np = md.shape[0]
    _, _, _, _, _, Q = _ref_1d(p)
    P = np.ones((2 ** d, Np, Np))
    for k in range(2 ** d):
        for j in range(d):
            c = (k >> j) & 1
            P[k] *= Q[c][md[:, None, j], md[None, :, j]]
    return P


# ----------------------------------------------------------------------------- mesh
def _cell_index_grid(n):
    d = len(n)
    idx = np.indices(tuple(reversed(n))).reshape(d, -1)[::-1]  # idx[k] = i_k, x fastest
    return idx


def neighbours(n) -> np.ndarray:
    """nbr[K][2k] = cell at -e_k, nbr[K][2k+1] = cell at +e_k, -1 outside."""
    n = tuple(int(v) for v in n)
    d = len(n)
    idx = _cell_index_grid(n)
    C = int(np.prod(n))
    stride = np.cumprod((1,) + n[:-1])
    K = np.arange(C)
    nbr = np.full((C, 2 * d), -1, dtype=np.int32)
    for k in range(d):
        lo = idx[k] > 0
        hi = idx[k] < n[k] - 1
        nbr[lo, 2 * k] = (K - stride[k])[lo]
        nbr[hi, 2 * k + 1] = (K + stride[k])[hi]
    return nbr


def centroids(n, h) -> np.ndarray:
    idx = _cell_index_grid(n)
    return np.stack([(idx[k] + 0.5) * h[k] for k in range(len(n))], axis=1)


def nu_field(n, ref_centroid, kind: str, rng=None, inside=1000.0, radius=0.3,
             centre=0.5) -> np.ndarray:
    """Cell-wise coefficient.  ref_centroid: centroids in unit-cube reference coordinates.

    kind 'jump':      nu = inside for cells whose centroid lies within radius of centre.
    kind 'lognormal': log nu ~ N(0,1) iid per cell (from rng) + log(inside) inside."""
    r2 = np.sum((ref_centroid - centre) ** 2, axis=1)
    ins = r2 < radius * radius
    if kind == "jump":
        return np.where(ins, inside, 1.0).astype(np.float64)
    if kind == "lognormal":
        lg = rng.standard_normal(ref_centroid.shape[0]) + np.where(ins, math.log(inside), 0.0)
        return np.exp(lg)
    raise ValueError(kind)


def harmonic(a, b):
    """2ab/(a+b), evaluated so that harmonic(a, b) == harmonic(b, a) bitwise."""
    return 2.0 * (a * b) / (a + b)


def assemble(n, p: int, h, nu: np.ndarray, eta: float, ref=None):
    """Block-ELL matrix of the SWIP form: blocks (2d+1, C, Np, Np), nbr (C, 2d)."""
    n = tuple(int(v) for v in n)
    d = len(n)
    if ref is None:
        ref = reference_matrices(d, p, h, eta)
    V, F, B = ref["V"], ref["F"], ref["B"]
    Np = V.shape[0]
    C = int(np.prod(n))
    nbr = neighbours(n)
    blocks = np.zeros((2 * d + 1, C, Np, Np))
    blocks[0] = nu[:, None, None] * V[None]
    for k in range(d):
        lo, hi = nbr[:, 2 * k], nbr[:, 2 * k + 1]
        has_lo, has_hi = lo >= 0, hi >= 0
        g_lo = np.where(has_lo, harmonic(nu, nu[np.maximum(lo, 0)]), 0.0)
        g_hi = np.where(has_hi, harmonic(nu, nu[np.maximum(hi, 0)]), 0.0)
        # high face of K: K is the low-side cell L; low face of K: K is the high-side R
        blocks[0] += (g_hi[:, None, None] * F[k, 0][None]
                      + np.where(has_hi, 0.0, nu)[:, None, None] * B[k, 1][None]
                      + g_lo[:, None, None] * F[k, 3][None]
                      + np.where(has_lo, 0.0, nu)[:, None, None] * B[k, 0][None])
        blocks[1 + 2 * k] = g_lo[:, None, None] * F[k, 2][None]   # test R=K, trial L=-e_k nbr
        blocks[2 + 2 * k] = g_hi[:, None, None] * F[k, 1][None]   # test L=K, trial R=+e_k nbr
    return blocks, nbr


def dense_matrix(blocks: np.ndarray, nbr: np.ndarray) -> np.ndarray:
    """Expand a block-ELL matrix into a dense (N, N) array (small meshes only)."""
    S, C, Np, _ = blocks.shape
    A = np.zeros((C * Np, C * Np))
    for K in range(C):
        A[K * Np:(K + 1) * Np, K * Np:(K + 1) * Np] += blocks[0, K]
        for s in range(1, S):
            J = nbr[K, s - 1]
            if J >= 0:
                A[K * Np:(K + 1) * Np, J * Np:(J + 1) * Np] += blocks[s, K]
    return A


def eval_field(u: np.ndarray, n, p: int, h, pts: np.ndarray) -> np.ndarray:
    """Evaluate the DG field with coefficients u (C*Np) at physical points pts (m, d)."""
    n = tuple(int(v) for v in n)
    d = len(n)
    md = modes(d, p)
    Np = md.shape[0]
    h = np.asarray(h, dtype=np.float64)
    cidx = np.minimum((pts / h).astype(np.int64), np.array(n) - 1)
    stride = np.cumprod((1,) + n[:-1])
    K = (cidx * stride).sum(axis=1)
    xi = (pts - (cidx + 0.5) * h) / (0.5 * h)
    val = np.ones((pts.shape[0], Np)) * np.prod(np.sqrt(2.0 / h))
    for a in range(Np):
        for j in range(d):
            val[:, a] *= _leg(int(md[a, j]), xi[:, j])
    return np.sum(val * u.reshape(-1, Np)[K], axis=1)


# ----------------------------------------------------------------------------- problem
@dataclasses.dataclass
class Problem:
    """A fine operator with its agglomeration hierarchy and right-hand side(s)."""
    d: int
    p: int
    n: tuple            # cells per direction
    h: np.ndarray       # cell size per direction
    nlevels: int
    eta: float
    nu: np.ndarray      # (C,)
    blocks: np.ndarray  # (2d+1, C, Np, Np) float64
    nbr: np.ndarray     # (C, 2d) int32
    prolong: np.ndarray  # (2^d, Np, Np)
    ref: dict           # reference matrices V, F, B
    b: np.ndarray       # (C*Np,) or (C*Np, nrhs) with the right-hand sides fastest

    @property
    def np_(self) -> int:
        return self.blocks.shape[2]

    @property
    def ncells(self) -> int:
        return self.blocks.shape[1]

    @property
    def ndof(self) -> int:
        return self.ncells * self.np_

    @property
    def nrhs(self) -> int:
        return 1 if self.b.ndim == 1 else self.b.shape[1]


def make_problem(d: int, p: int, n, nlevels: int, *, length=None, nu_kind="jump",
                 nu_inside=1000.0, radius=0.3, seed=0, nrhs=1, eta=None) -> Problem:
    """Build a seeded problem.  length: domain extent per direction (default unit cube).

    The coefficient ball is placed in unit-cube reference coordinates, so stretched
    domains see an ellipsoid.  b ~ U[-1,1] iid per DOF (and per right-hand side)."""
    n = tuple(int(v) for v in n)
    if len(n) != d:
        raise ValueError("n must have d entries")
    for v in n:
        if v % (1 << (nlevels - 1)):
            raise ValueError(f"{n} cells do not agglomerate over {nlevels} levels")
    length = np.ones(d) if length is None else np.asarray(length, dtype=np.float64)
    h = length / np.array(n)
    if eta is None:
        eta = 4.0 * (p + 1) ** 2
    rng = np.random.default_rng(seed)
    ref_c = centroids(n, 1.0 / np.array(n, dtype=np.float64))
    nu = nu_field(n, ref_c, nu_kind, rng=rng, inside=nu_inside, radius=radius)
    ref = reference_matrices(d, p, h, eta)
    blocks, nbr = assemble(n, p, h, nu, eta, ref)
    Np = blocks.shape[2]
    N = blocks.shape[1] * Np
    b = rng.uniform(-1.0, 1.0, size=N if nrhs == 1 else (N, nrhs))
    return Problem(d=d, p=p, n=n, h=h, nlevels=nlevels, eta=float(eta), nu=nu,
                   blocks=blocks, nbr=nbr, prolong=prolongation_matrices(d, p), ref=ref, b=b)


def project(fun, n, p: int, h, q: int | None = None) -> np.ndarray:
    """L2 projection of fun(points (m, d)) -> (m,) onto the DG space (C*Np coefficients).

    Uses a tensor Gauss rule with q points per direction (exact for polynomials of degree
    <= 2q-1-p in each direction)."""
    n = tuple(int(v) for v in n)
    d = len(n)
    md = modes(d, p)
    Np = md.shape[0]
    h = np.asarray(h, dtype=np.float64)
    q = q or p + 3
    xg, wg = npleg.leggauss(q)
    XI = np.stack(np.meshgrid(*([xg] * d), indexing="ij"), axis=-1).reshape(-1, d)
    W = np.prod(np.stack(np.meshgrid(*([wg] * d), indexing="ij"), axis=-1).reshape(-1, d), axis=1)
    phi = np.ones((XI.shape[0], Np)) * np.prod(np.sqrt(2.0 / h))
    for a in range(Np):
        for j in range(d):
            phi[:, a] *= _leg(int(md[a, j]), XI[:, j])
    jac = np.prod(h / 2.0)
    ctr = centroids(n, h)
    out = np.zeros((ctr.shape[0], Np))
    for K in range(ctr.shape[0]):
        pts = ctr[K] + XI * (h / 2.0)
        out[K] = (W * fun(pts)) @ phi * jac
    return out.reshape(-1)
