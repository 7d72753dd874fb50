"""Pins of the seeded problem generator (inputs shared by the oracle and the CUDA path)."""
import numpy as np
import pytest

from workloads import (dense_matrix, eval_field, make_problem, neighbours, project,
                       prolongation_matrices, workload)
from workloads.sipg import _cell_index_grid, assemble


@pytest.mark.parametrize("name", ["sipg2d_p1_16x16", "sipg3d_p1_8x4x4", "sipg2d_p2_32x16"])
def test_symmetric_positive_definite(name):
    pr = workload(name).make(0)
    A = dense_matrix(pr.blocks, pr.nbr)
    assert np.array_equal(A, A.T)            # bitwise symmetric by construction
    np.linalg.cholesky(A)                    # SPD: the factorisation exists


def test_stretched_p3_spd():
    pr = make_problem(3, 3, (4, 4, 4), 2, length=(1, 1, 10), nu_inside=1e4)
    np.linalg.cholesky(dense_matrix(pr.blocks, pr.nbr))


@pytest.mark.parametrize("d,p,n,u,f", [
    (2, 2, (8, 8), lambda X: X[:, 0] ** 2, lambda X: -2.0 + 0 * X[:, 0]),
    (3, 2, (6, 6, 6), lambda X: X[:, 0] * X[:, 1] + X[:, 2] ** 2, lambda X: -2.0 + 0 * X[:, 0]),
    (2, 1, (8, 8), lambda X: 3 * X[:, 0] - X[:, 1], lambda X: 0 * X[:, 0]),
    (3, 3, (4, 4, 4), lambda X: X[:, 0] ** 3 - X[:, 1] * X[:, 2] ** 2,
     lambda X: -(6 * X[:, 0] - 2 * X[:, 1])),
])
def test_consistency_on_interior_cells(d, p, n, u, f):
    """SIP is consistent: a polynomial solution of degree <= p satisfies the discrete
    equations exactly on cells away from the (non-homogeneous) boundary."""
    h = np.ones(d) / np.array(n)
    nu = np.full(int(np.prod(n)), 2.5)
    blocks, nbr = assemble(n, p, h, nu, 4.0 * (p + 1) ** 2)
    A = dense_matrix(blocks, nbr)
    uh = project(u, n, p, h)
    r = A @ uh - 2.5 * project(f, n, p, h)    # -div(nu grad u) = nu * f here
    interior = (nbr >= 0).all(axis=1)
    Np = blocks.shape[2]
    assert np.abs(r.reshape(-1, Np)[interior]).max() < 1e-10 * np.abs(A @ uh).max()


def test_weighted_average_matches_harmonic_mean():
    """Across a coefficient jump the face block equals the unit-coefficient face block
    scaled by the harmonic mean 2 a b/(a+b) (weighted-average SIP)."""
    n, p, h = (2, 1), 2, np.array([0.5, 1.0])
    nu = np.array([1.0, 1000.0])
    blocks, nbr = assemble(n, p, h, nu, 36.0)
    blocks1, _ = assemble(n, p, h, np.ones(2), 36.0)
    gam = 2 * 1000.0 / 1001.0
    assert np.allclose(blocks[2, 0], gam * blocks1[2, 0], rtol=1e-14, atol=0)


@pytest.mark.parametrize("d,p", [(2, 1), (2, 2), (3, 2), (3, 3)])
def test_prolongation_orthonormal(d, p):
    P = prolongation_matrices(d, p)
    assert np.abs(sum(P[k].T @ P[k] for k in range(2 ** d)) - np.eye(P.shape[1])).max() < 1e-14


@pytest.mark.parametrize("d,p", [(2, 1), (2, 3), (3, 2)])
def test_prolongation_reproduces_polynomials(d, p):
    nc, nf = (2,) * d, (4,) * d
    hc, hf = np.ones(d) / 2, np.ones(d) / 4
    fun = lambda X: 1 + X[:, 0] - 0.5 * X[:, -1] ** min(p, 2) + (X[:, 0] * X[:, 1] ** (p - 1) if p > 1 else 0)
    uc = project(fun, nc, p, hc)
    P = prolongation_matrices(d, p)
    Np = P.shape[1]
    idx = _cell_index_grid(nf)
    uf = np.zeros(int(np.prod(nf)) * Np)
    for K in range(int(np.prod(nf))):
        c = [idx[j][K] // 2 for j in range(d)]
        k = sum(((idx[j][K] % 2) << j) for j in range(d))
        J = sum(c[j] * int(np.prod(nc[:j])) for j in range(d))
        uf[K * Np:(K + 1) * Np] = P[k] @ uc[J * Np:(J + 1) * Np]
    pts = np.random.default_rng(0).uniform(0, 1, (300, d))
    assert np.abs(eval_field(uf, nf, p, hf, pts) - fun(pts)).max() < 1e-12


def test_layout_and_boundary_blocks():
    pr = workload("sipg3d_p1_8x4x4").make(0)
    nbr = neighbours(pr.n)
    assert np.array_equal(nbr, pr.nbr)
    # K = ix + 8*(iy + 4*iz); -x neighbour of ix=0 is missing, +y of iy=3 too
    K = 0 + 8 * (3 + 4 * 2)
    assert nbr[K, 0] == -1 and nbr[K, 1] == K + 1 and nbr[K, 3] == -1 and nbr[K, 2] == K - 8
    assert nbr[K, 4] == K - 32 and nbr[K, 5] == K + 32
    for s in range(1, 7):
        assert np.all(pr.blocks[s][pr.nbr[:, s - 1] < 0] == 0.0)


def test_seeded_inputs():
    a = workload("sipg2d_p1_16x16").make(0)
    b = workload("sipg2d_p1_16x16").make(0)
    c = workload("sipg2d_p1_16x16").make(1)
    assert np.array_equal(a.b, b.b) and not np.array_equal(a.b, c.b)
    assert a.b.min() >= -1 and a.b.max() <= 1
    # coefficient: 1000 exactly in cells whose centroid is within 0.3 of the centre
    ctr = (np.stack(np.meshgrid(np.arange(16), np.arange(16), indexing="xy"), -1).reshape(-1, 2) + 0.5) / 16
    inside = ((ctr - 0.5) ** 2).sum(1) < 0.09
    assert np.array_equal(a.nu, np.where(inside, 1000.0, 1.0))


def test_sizes_of_paper_shaped_workloads():
    assert workload("sipg3d_p2_64cube").ndof == 2621440
    assert workload("sipg3d_p3_48cube_zstretch").ndof == 2211840
    assert workload("sipg3d_p2_32cube_lognormal").ndof == 327680
    assert workload("sipg2d_p1_16x16").ndof == 768
