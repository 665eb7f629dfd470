"""Pins for the oracle's clover term (Sheikholeslami-Wohlert): the clover
leaves against a generic path walker, a uniform abelian flux (closed form
F = sin phi), gauge covariance, antisymmetry in (mu, nu), the sigma algebra,
free field and c_sw = 0 reduce to Wilson, g5-hermiticity and the adjoint by
dense matrices, per-site Hermitian blocks that split by chirality."""
import numpy as np
import pytest

from oracle import clover as CL
from oracle import operators as ops
from oracle import deflation as D
import oracle.estimator as OE
from oracle.lattice import coords, index_of, volume
from paper_2106_01275_gb300 import inputs


def _walk(U, dims, x, steps):
    """Parallel transporter along a path of steps (+mu or -mu, as (mu, +1/-1))
    from site coordinates x: U_mu(y) for a step forward, U_mu(y - mu)^H back."""
    y = np.array(x)
    M = np.eye(3, dtype=np.complex128)
    for mu, s in steps:
        e = np.zeros(4, dtype=np.int64)
        e[mu] = 1
        if s > 0:
            M = M @ U[index_of(y[None], dims)[0], mu]
            y = y + e
        else:
            y = y - e
            M = M @ np.conj(U[index_of(y[None], dims)[0], mu]).T
    assert np.array_equal(np.mod(y, dims), np.mod(x, dims))      # a closed loop
    return M


def test_leaves_are_the_four_plaquettes_at_x():
    dims = [3, 4, 2, 5]
    U = inputs.gauge_links(dims, 3, eps=0.8)
    xs = coords(dims)
    for mu, nu in [(0, 1), (1, 3), (2, 3), (3, 0)]:
        Q = CL.clover_leaves(U, dims, mu, nu)
        for i in (0, 7, 61, volume(dims) - 1):
            x = xs[i]
            want = (_walk(U, dims, x, [(mu, 1), (nu, 1), (mu, -1), (nu, -1)])
                    + _walk(U, dims, x, [(nu, 1), (mu, -1), (nu, -1), (mu, 1)])
                    + _walk(U, dims, x, [(mu, -1), (nu, -1), (mu, 1), (nu, 1)])
                    + _walk(U, dims, x, [(nu, -1), (mu, 1), (nu, 1), (mu, -1)]))
            assert np.allclose(Q[i], want, atol=1e-13)


@pytest.mark.parametrize("plane,dims,n", [((0, 1), [4, 6, 2, 2], 1), ((2, 3), [2, 2, 3, 4], 2)])
def test_uniform_abelian_flux_closed_form(plane, dims, n):
    U, phi = CL.uniform_abelian_links(dims, n, plane)
    mu, nu = plane
    I3 = np.eye(3)
    for a in range(4):
        for b in range(4):
            if a == b:
                continue
            F = CL.field_strength(U, dims, a, b)
            if (a, b) == (mu, nu):
                want = np.sin(phi)
            elif (a, b) == (nu, mu):
                want = -np.sin(phi)
            else:
                want = 0.0
            assert np.allclose(F, want * I3, atol=1e-13), (a, b)
    Q = CL.clover_leaves(U, dims, mu, nu)
    assert np.allclose(Q, 4 * np.exp(1j * phi) * I3, atol=1e-13)
    kappa, csw = 0.13, 1.7
    C = CL.clover_blocks(U, dims, kappa, csw)
    want = -kappa * csw * np.sin(phi) * np.kron(CL.sigma(mu, nu), I3)
    assert np.allclose(C, want[None], atol=1e-13)


def test_sigma_algebra():
    _, g5 = ops.gammas()
    for mu in range(4):
        for nu in range(4):
            s = CL.sigma(mu, nu)
            assert np.allclose(s, s.conj().T)
            assert np.allclose(s, -CL.sigma(nu, mu))
            assert np.allclose(s @ g5, g5 @ s)
            if mu != nu:
                assert np.allclose(s @ s, np.eye(4))                 # (i g_mu g_nu)^2 = 1 for mu != nu


def test_gauge_covariance():
    dims = [2, 3, 2, 4]
    N = volume(dims)
    U = inputs.gauge_links(dims, 5, eps=0.7)
    g = inputs.random_su3(N, 6)
    fwd, _ = ops.neighbour_tables(dims)
    Ug = np.stack([g @ U[:, mu] @ np.conj(np.swapaxes(g[fwd[mu]], -1, -2)) for mu in range(4)], axis=1)
    for mu, nu in [(0, 1), (0, 3), (1, 2)]:
        F, Fg = CL.field_strength(U, dims, mu, nu), CL.field_strength(Ug, dims, mu, nu)
        assert np.allclose(Fg, g @ F @ np.conj(np.swapaxes(g, -1, -2)), atol=1e-12)
    rng = np.random.default_rng(1)
    psi = rng.standard_normal((N, 4, 3)) + 1j * rng.standard_normal((N, 4, 3))
    gpsi = np.einsum('nab,nsb->nsa', g, psi)
    lhs = CL.clover_apply(gpsi, Ug, 0.12, 1.3, dims)
    rhs = np.einsum('nab,nsb->nsa', g, CL.clover_apply(psi, U, 0.12, 1.3, dims))
    assert np.allclose(lhs, rhs, atol=1e-12)


def test_antisymmetry_and_hermitian_field():
    dims = [2, 2, 3, 2]
    U = inputs.gauge_links(dims, 8, eps=0.9)
    for mu, nu in [(0, 1), (1, 3), (2, 0)]:
        F = CL.field_strength(U, dims, mu, nu)
        assert np.allclose(F, np.conj(np.swapaxes(F, -1, -2)), atol=1e-14)
        assert np.allclose(CL.field_strength(U, dims, nu, mu), -F, atol=1e-14)
    assert np.allclose(CL.field_strength(U, dims, 1, 1), 0.0, atol=1e-14)


def test_reduces_to_wilson():
    dims = [2, 2, 2, 4]
    N = volume(dims)
    rng = np.random.default_rng(2)
    psi = rng.standard_normal((N, 4, 3)) + 1j * rng.standard_normal((N, 4, 3))
    Ufree = inputs.unit_links(dims)
    assert np.abs(CL.clover_blocks(Ufree, dims, 0.12, 1.9)).max() == 0.0
    assert np.allclose(CL.clover_apply(psi, Ufree, 0.12, 1.9, dims), ops.wilson_apply(psi, Ufree, 0.12, dims))
    U = inputs.gauge_links(dims, 9)
    assert np.allclose(CL.clover_apply(psi, U, 0.12, 0.0, dims), ops.wilson_apply(psi, U, 0.12, dims))


def test_gamma5_hermiticity_adjoint_and_blocks_dense():
    dims = [2, 2, 2, 4]
    N = volume(dims)
    U = inputs.gauge_links(dims, 10, eps=0.8)
    op = CL.WilsonClover(dims, U, 0.125, 1.6)
    A = D.dense_matrix(op)
    G5 = np.kron(np.eye(N), np.kron(np.diag([1.0, 1.0, -1.0, -1.0]), np.eye(3)))
    assert np.allclose(G5 @ A @ G5, A.conj().T, atol=1e-13)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(12 * N) + 1j * rng.standard_normal(12 * N)
    assert np.allclose(op.apply_dagger(x).reshape(-1), A.conj().T @ x, atol=1e-12)
    Aw = D.dense_matrix(OE.Wilson(dims, U, 0.125))
    C = CL.clover_blocks(U, dims, 0.125, 1.6)
    diff = A - Aw                                                  # only the site blocks differ
    for i in range(N):
        blk = diff[12 * i:12 * i + 12, 12 * i:12 * i + 12]
        assert np.allclose(blk, C[i], atol=1e-14)
        assert np.allclose(blk, blk.conj().T, atol=1e-14)
        assert np.allclose(blk[:6, 6:], 0.0, atol=1e-14) and np.allclose(blk[6:, :6], 0.0, atol=1e-14)
        diff[12 * i:12 * i + 12, 12 * i:12 * i + 12] = 0.0
    assert np.abs(diff).max() < 1e-14
    b = rng.standard_normal(12 * N) + 1j * rng.standard_normal(12 * N)
    xs, _, rel = op.solve(b, 1e-12)
    assert np.allclose(A @ xs.reshape(-1), b, atol=1e-9)
