"""Pins for the oracle's even-odd preconditioning (the Schur complement on
the even sites of both operators)."""
import numpy as np
import pytest

import oracle.estimator as OE
from oracle import deflation as D
from oracle import evenodd as EO
from paper_2106_01275_gb300 import inputs


def _dense(apply, n, dt):
    A = np.zeros((n, n), dtype=dt)
    for j in range(n):
        e = np.zeros(n, dtype=dt)
        e[j] = 1.0
        A[:, j] = np.asarray(apply(e)).reshape(-1)
    return A


def test_laplacian_schur_is_the_block_formula_and_solves_the_system():
    """S applied matrix-free equals A_ee - A_eo A_oo^{-1} A_oe built from the
    dense A by index blocks; the even solve plus reconstruction is A^{-1} b."""
    dims, m2 = [4, 4, 2, 2], 0.1
    eo = EO.LaplacianEO(dims, m2)
    A = D.dense_matrix(OE.Laplacian(dims, m2))
    ev, od = eo.ev, eo.od
    S_block = A[np.ix_(ev, ev)] - A[np.ix_(ev, od)] @ np.linalg.inv(A[np.ix_(od, od)]) @ A[np.ix_(od, ev)]
    S = _dense(eo.schur, ev.size, np.float64)
    assert np.allclose(S, S_block, atol=1e-13)
    assert np.allclose(A[np.ix_(ev, od)], -_dense(eo.hop_eo, od.size, np.float64))       # bipartite hops
    assert np.allclose(A[np.ix_(ev, ev)], eo.d * np.eye(ev.size))
    b = np.random.default_rng(2).standard_normal(eo.N)
    x_e = np.linalg.solve(S, eo.rhs(b))
    assert np.allclose(eo.reconstruct(x_e, b), np.linalg.solve(A, b), atol=1e-12)


def test_laplacian_schur_is_better_conditioned():
    """The eigenvalues of H_eo H_oe are the squares of the hop sum's, in
    [0, 64] (both ends reached on a 4^4 torus), so cond(S) = d^2 / (d^2 - 64)
    against cond(A) = (d + 8) / (d - 8): about four times smaller."""
    dims, m2 = [4, 4, 4, 4], 0.05
    eo = EO.LaplacianEO(dims, m2)
    d = eo.d
    S = _dense(eo.schur, eo.ev.size, np.float64)
    w = np.linalg.eigvalsh(0.5 * (S + S.T))
    assert np.isclose(w.max() / w.min(), d ** 2 / (d ** 2 - 64), rtol=1e-9)
    condA = (d + 8) / (d - 8)
    assert np.isclose(condA / (w.max() / w.min()), (d + 8) ** 2 / d ** 2, rtol=1e-9)   # about 4: half the CG iterations


def test_wilson_schur_solves_the_system():
    dims, kappa = [2, 2, 2, 4], 0.12
    U = inputs.gauge_links(dims, 23)
    eo = EO.WilsonEO(dims, U, kappa)
    A = D.dense_matrix(OE.Wilson(dims, U, kappa))
    n_e = eo.ev.size * 12
    S = _dense(lambda v: eo.schur(v.reshape(-1, 12)), n_e, np.complex128)
    rng = np.random.default_rng(5)
    b = rng.standard_normal((eo.N, 12)) + 1j * rng.standard_normal((eo.N, 12))
    x_e = np.linalg.solve(S, eo.rhs(b).reshape(-1))
    assert np.allclose(eo.reconstruct(x_e, b).reshape(-1), np.linalg.solve(A, b.reshape(-1)), atol=1e-11)
    # the same Schur complement from the dense blocks (site-major, 12 components per site)
    idx_e = (eo.ev[:, None] * 12 + np.arange(12)).reshape(-1)
    idx_o = (eo.od[:, None] * 12 + np.arange(12)).reshape(-1)
    S_block = A[np.ix_(idx_e, idx_e)] - A[np.ix_(idx_e, idx_o)] @ np.linalg.inv(A[np.ix_(idx_o, idx_o)]) @ A[np.ix_(idx_o, idx_e)]
    assert np.allclose(S, S_block, atol=1e-12)


def test_odd_sides_are_refused():
    with pytest.raises(ValueError):
        EO.LaplacianEO([4, 3, 4, 4], 0.1)


def test_clover_schur_is_the_block_formula_and_solves_the_system():
    """With the clover term the diagonal blocks are site matrices: the
    matrix-free S equals the dense block formula, the even solve plus
    reconstruction is A^{-1} b, and c_sw = 0 gives the Wilson complement."""
    from oracle import clover as CL
    dims, kappa, csw = [2, 2, 2, 4], 0.12, 1.8
    U = inputs.gauge_links(dims, 24, eps=0.8)
    eo = EO.WilsonCloverEO(dims, U, kappa, csw)
    A = D.dense_matrix(CL.WilsonClover(dims, U, kappa, csw))
    n_e = eo.ev.size * 12
    S = _dense(lambda v: eo.schur(v.reshape(-1, 12)), n_e, np.complex128)
    idx_e = (eo.ev[:, None] * 12 + np.arange(12)).reshape(-1)
    idx_o = (eo.od[:, None] * 12 + np.arange(12)).reshape(-1)
    S_block = A[np.ix_(idx_e, idx_e)] - A[np.ix_(idx_e, idx_o)] @ np.linalg.inv(A[np.ix_(idx_o, idx_o)]) @ A[np.ix_(idx_o, idx_e)]
    assert np.allclose(S, S_block, atol=1e-12)
    assert not np.allclose(A[np.ix_(idx_o, idx_o)], np.eye(idx_o.size))          # the blocks are not trivial
    rng = np.random.default_rng(6)
    b = rng.standard_normal((eo.N, 12)) + 1j * rng.standard_normal((eo.N, 12))
    x_e = np.linalg.solve(S, eo.rhs(b).reshape(-1))
    assert np.allclose(eo.reconstruct(x_e, b).reshape(-1), np.linalg.solve(A, b.reshape(-1)), atol=1e-11)
    eo0, eow = EO.WilsonCloverEO(dims, U, kappa, 0.0), EO.WilsonEO(dims, U, kappa)
    v = rng.standard_normal((eo.ev.size, 12)) + 1j * rng.standard_normal((eo.ev.size, 12))
    assert np.allclose(eo0.schur(v), eow.schur(v), atol=1e-14)
