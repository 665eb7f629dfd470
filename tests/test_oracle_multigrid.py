"""Pins for the oracle's two-level multigrid: the Galerkin coarse operator of
the Laplacian in closed form, GMRES against a direct solve, the two-grid
cycle as a convergent symmetric preconditioner, the chirality-split adaptive
prolongator for Wilson (orthonormal, commuting with g5, a g5-Hermitian
coarse operator) and multigrid-preconditioned solves that match dense
solves in fewer iterations."""
import numpy as np
import pytest

import oracle.estimator as OE
from oracle import deflation as D
from oracle import multigrid as MG
from oracle import operators as ops
from paper_2106_01275_gb300 import inputs


def _lap(dims, m2):
    return lambda x: np.asarray(ops.laplacian_apply(np.asarray(x).reshape(-1), dims, m2)).reshape(-1)


@pytest.mark.parametrize("dims", [[4, 4, 4, 4], [8, 4, 4, 4], [4, 8, 4, 8]])
def test_laplacian_galerkin_operator_closed_form(dims):
    """Normalised block indicators (2^4 blocks): each block keeps 16 (8 + m^2)
    diagonal terms and loses its 64 inner hops, each face carries 8 hops, so
    P^T A P = (4 + m^2) - (1/2) sum_mu (S_mu + S_mu^{-1}) on the coarse lattice,
    i.e. half the coarse Laplacian with mass 2 m^2."""
    m2 = 0.3
    P = MG.prolongator_constant(dims, 2)
    Ac = MG.coarse_operator(_lap(dims, m2), P)
    cd = [d // 2 for d in dims]
    want = 0.5 * D.dense_matrix(OE.Laplacian(cd, 2 * m2))
    assert np.allclose(Ac, want, atol=1e-13)
    assert np.allclose(P.T @ P, np.eye(P.shape[1]))


def test_laplacian_galerkin_operator_block_side_4():
    """Blocks of b^4 sites in general: per block b^4 (8 + m^2) diagonal terms,
    8 b^3 (b - 1) inner hops, b^3 hops through each face, so
    P^T A P = (8 / b + m^2) - (1 / b) sum_mu (S_mu + S_mu^{-1}) = (1 / b) A_coarse(b m^2)."""
    dims, m2, b = [8, 8, 4, 8], 0.2, 4
    Ac = MG.coarse_operator(_lap(dims, m2), MG.prolongator_constant(dims, b))
    want = D.dense_matrix(OE.Laplacian([d // b for d in dims], b * m2)) / b
    assert np.allclose(Ac, want, atol=1e-13)


def test_gmres_against_a_direct_solve():
    """Full GMRES ends in n steps at the exact solution; restarted GMRES
    converges when the spectrum stays clear of the origin (and stagnates
    when it does not: eigenvalues in a disk of radius ~ sqrt(40) about 4)."""
    rng = np.random.default_rng(1)
    A = np.eye(40) * 4 + rng.standard_normal((40, 40))
    b = rng.standard_normal(40)
    x, its, rel = MG.gmres(lambda v: A @ v, b, tol=1e-12, restart=40)
    assert its <= 40 and rel <= 1e-12 and np.allclose(x, np.linalg.solve(A, b), atol=1e-10)
    _, _, rel15 = MG.gmres(lambda v: A @ v, b, tol=1e-12, restart=15, maxit=300)
    assert rel15 > 1e-3
    A2 = np.eye(40) * 10 + rng.standard_normal((40, 40))
    x, its, rel = MG.gmres(lambda v: A2 @ v, b, tol=1e-12, restart=15)
    assert rel <= 1e-12 and np.allclose(x, np.linalg.solve(A2, b), atol=1e-10)
    Ac = A + 1j * rng.standard_normal((40, 40))
    bc = b + 1j * rng.standard_normal(40)
    x, its, rel = MG.gmres(lambda v: Ac @ v, bc, tol=1e-12, restart=40, precond=lambda r: r / 4.0)
    assert rel <= 1e-12 and np.allclose(x, np.linalg.solve(Ac, bc), atol=1e-10)


def test_two_grid_cycle_is_a_convergent_symmetric_preconditioner():
    """Symmetric smoothing around a Galerkin correction: M is symmetric
    positive definite and the error propagator I - M A contracts."""
    dims, m2 = [4, 4, 4, 4], 0.01
    N = 256
    A_apply = _lap(dims, m2)
    M = MG.TwoGrid(A_apply, np.full(N, 8 + m2), MG.prolongator_constant(dims, 2), nu=2, omega=0.8)
    Md = np.stack([M(np.eye(N)[:, j]) for j in range(N)], axis=1)
    A = D.dense_matrix(OE.Laplacian(dims, m2))
    assert np.allclose(Md, Md.T, atol=1e-12)
    assert np.linalg.eigvalsh(0.5 * (Md + Md.T)).min() > 0
    rho = np.abs(np.linalg.eigvals(np.eye(N) - Md @ A)).max()
    assert rho < 0.6, rho


def test_laplacian_multigrid_solve():
    """8^4, m^2 = 0.001: the two-grid preconditioned GMRES matches CG's
    solution and needs far fewer iterations than unpreconditioned GMRES."""
    dims, m2 = [8, 8, 8, 8], 0.001
    N = 4096
    A_apply = _lap(dims, m2)
    b = np.random.default_rng(2).standard_normal(N)
    M = MG.TwoGrid(A_apply, np.full(N, 8 + m2), MG.prolongator_constant(dims, 2))
    x, its_mg, rel = MG.gmres(A_apply, b, tol=1e-10, restart=40, precond=M)
    _, its_plain, _ = MG.gmres(A_apply, b, tol=1e-10, restart=40)
    xc, _, _ = OE.Laplacian(dims, m2).solve(b, 1e-12)
    assert rel <= 1e-10 and np.allclose(x, np.asarray(xc).reshape(-1), rtol=0, atol=1e-7 * np.abs(xc).max())
    assert its_mg * 3 <= its_plain, (its_mg, its_plain)


def test_wilson_adaptive_prolongator_and_solve():
    dims, kappa = [2, 2, 4, 4], 0.124
    N = int(np.prod(dims))
    U = inputs.gauge_links(dims, 5, eps=0.3)
    op = OE.Wilson(dims, U, kappa)
    A_apply = lambda x: np.asarray(op.apply(np.asarray(x).reshape(N, 12))).reshape(-1)
    n = 12 * N
    V = MG.near_null_vectors(A_apply, np.ones(n), n, 4, 20, 7, np.complex128)
    P = MG.prolongator_adaptive(V, dims, 2, 12)
    assert np.allclose(P.conj().T @ P, np.eye(P.shape[1]), atol=1e-12)
    g5 = np.tile(np.repeat([1.0, 1.0, -1.0, -1.0], 3), N)
    G5c = np.tile(np.repeat([1.0, -1.0], 4), P.shape[1] // 8)          # chirality of each coarse column
    assert np.allclose(g5[:, None] * P, P * G5c[None, :])
    M = MG.TwoGrid(A_apply, np.ones(n), P, nu=2, omega=0.8)
    assert np.allclose(G5c[:, None] * M.Ac * G5c[None, :], M.Ac.conj().T, atol=1e-12)
    # the near-null vectors are smooth: A damps them far more than random vectors
    rng = np.random.default_rng(3)
    Rv = rng.standard_normal((n, 4)) + 1j * rng.standard_normal((n, 4))
    ratio = lambda X: np.mean([np.linalg.norm(A_apply(X[:, k])) / np.linalg.norm(X[:, k]) for k in range(4)])
    assert ratio(V) < 0.5 * ratio(Rv)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x, its_mg, rel = MG.gmres(A_apply, b, tol=1e-10, restart=40, precond=M)
    _, its_plain, _ = MG.gmres(A_apply, b, tol=1e-10, restart=40)
    A = D.dense_matrix(op)
    assert rel <= 1e-10 and np.allclose(x, np.linalg.solve(A, b), atol=1e-8)
    assert its_mg < its_plain, (its_mg, its_plain)


def test_block_side_must_divide():
    with pytest.raises(ValueError):
        MG.prolongator_constant([4, 4, 6, 4], 4)
