"""Pins for the oracle's deflation of singular triplets (Sec. 2.4, Eq. (6))."""
import numpy as np
import pytest

import oracle.estimator as OE
from oracle import deflation as D
from oracle.colouring import greedy_colour
from oracle.variance import exact_variance


def _lap(dims, m2):
    return OE.Laplacian(dims, m2)


def test_split_holds_for_any_subspace():
    """Eq. (6) with P in front: for random U, V (U^H A V invertible) the
    deflated part plus the trace of P A^{-1} (I - Q) is Tr(P A^{-1})."""
    dims, mu = [4, 4, 2, 2], 0
    op = _lap(dims, 0.2)
    A = D.dense_matrix(op)
    Ainv = np.linalg.inv(A)
    rng = np.random.default_rng(3)
    U = rng.standard_normal((A.shape[0], 5))
    V = rng.standard_normal((A.shape[0], 5))
    M = D.small_matrix(A @ V, U)
    Q = A @ V @ M @ U.conj().T
    for p in (0, 1, 2):
        P = D.displacement_matrix(dims, mu, p)
        exact = np.trace(P @ Ainv)
        part = D.deflated_part(U, V, M, dims, mu, [p])[0]
        rest = np.trace(P @ Ainv @ (np.eye(A.shape[0]) - Q))
        assert np.isclose(part + rest, exact, rtol=1e-12, atol=1e-12)
        assert np.isclose(part, np.trace(P @ Ainv @ Q), rtol=1e-11, atol=1e-12)


def test_laplacian_lowest_modes_are_the_constant_and_plane_waves():
    """The smallest eigenvalues of (8 + m^2) - hops on a torus are
    m^2 + sum_mu 4 sin^2(pi n_mu / D_mu): m^2 (constant mode), then
    m^2 + 4 sin^2(pi / D) for the longest side (two degenerate modes)."""
    dims, m2 = [8, 4, 4, 2], 0.1
    U, s, V = D.lowest_singular_triplets(D.dense_matrix(_lap(dims, m2)), 3)
    assert np.isclose(s[0], m2, rtol=1e-12)
    assert np.allclose(np.abs(V[:, 0]), 1 / np.sqrt(np.prod(dims)), atol=1e-10)
    assert np.allclose(s[1:], m2 + 4 * np.sin(np.pi / 8) ** 2, rtol=1e-10)


def test_full_deflation_is_exact_and_leaves_nothing_to_estimate():
    """With every triplet deflated, Q = I: the deflated part is the exact trace
    and every probe's corrected contraction vanishes."""
    dims, mu, m2 = [4, 2, 2, 2], 0, 0.3
    op = _lap(dims, m2)
    A = D.dense_matrix(op)
    U, s, V = D.lowest_singular_triplets(A, A.shape[0])
    M = D.small_matrix(A @ V, U)
    col, m = greedy_colour(dims, mu, [1], 1, 0)
    for p in (0, 1):
        P = D.displacement_matrix(dims, mu, p)
        assert np.isclose(D.deflated_part(U, V, M, dims, mu, [p])[0], np.trace(P @ np.linalg.inv(A)), rtol=1e-11)
    est = D.deflated_probed_estimates(op, col, m, 5, 2, 0, mu, [0, 1], 1e-13, U, V, M)
    assert np.allclose(est, 0.0, atol=1e-9)


def test_deflated_estimate_is_unbiased_and_undeflated_when_empty():
    """No triplets: the ordinary probed estimate.  Some triplets: the mean of
    deflated part + estimates over many sets approaches the exact trace."""
    dims, mu, m2 = [4, 4, 2, 2], 0, 0.05
    op = _lap(dims, m2)
    A = D.dense_matrix(op)
    col, m = greedy_colour(dims, mu, [1], 1, 0)
    E0 = np.zeros((A.shape[0], 0))
    plain = OE.probed_estimates(op, col, m, 9, 3, 0, mu, [1], 1e-13)
    none = D.deflated_probed_estimates(op, col, m, 9, 3, 0, mu, [1], 1e-13, E0, E0, np.zeros((0, 0)))
    assert np.allclose(plain, none, rtol=1e-12, atol=1e-12)
    U, s, V = D.lowest_singular_triplets(A, 4)
    M = D.small_matrix(A @ V, U)
    est = D.deflated_probed_estimates(op, col, m, 9, 400, 0, mu, [1], 1e-12, U, V, M)
    total = D.deflated_part(U, V, M, dims, mu, [1])[0] + est[:, 0]
    exact = np.trace(D.displacement_matrix(dims, mu, 1) @ np.linalg.inv(A))
    sigma = np.sqrt(np.var(est[:, 0].real, ddof=1) / est.shape[0])
    assert abs(total.mean().real - exact) < 5 * sigma + 1e-12


def test_deflation_reduces_the_variance_near_the_massless_limit():
    """At small m^2 the lowest modes carry most of the variance: the exact
    variance of the probed estimator of P A^{-1} (I - Q) with 8 triplets is
    well below that of P A^{-1} (Eq. (2), general form)."""
    dims, mu, m2 = [4, 4, 4, 2], 0, 0.01
    op = _lap(dims, m2)
    A = D.dense_matrix(op)
    Ainv = np.linalg.inv(A)
    U, s, V = D.lowest_singular_triplets(A, 8)
    Q = A @ V @ D.small_matrix(A @ V, U) @ U.conj().T
    col, m = greedy_colour(dims, mu, [1], 1, 0)
    P = D.displacement_matrix(dims, mu, 1)
    v0 = exact_variance(P @ Ainv, col, 0)
    v1 = exact_variance(P @ Ainv @ (np.eye(A.shape[0]) - Q), col, 0)
    assert v1 < 0.2 * v0


def test_wilson_triplets_and_split():
    """Wilson-Dirac (non-Hermitian, 12 dof per site): the triplets satisfy
    A V = U diag(s), so M = (U^H A V)^{-1} = diag(1 / s), and the split of
    Tr(P A^{-1}) holds for every displacement."""
    from paper_2106_01275_gb300 import inputs
    dims, mu, kappa = [2, 2, 2, 2], 2, 0.12
    Uf = inputs.gauge_links(dims, 7)
    op = OE.Wilson(dims, Uf, kappa)
    A = D.dense_matrix(op)
    U, s, V = D.lowest_singular_triplets(A, 10)
    assert np.allclose(A @ V, U * s[None, :], atol=1e-10)
    M = D.small_matrix(A @ V, U)
    assert np.allclose(M, np.diag(1.0 / s), atol=1e-9)
    Ainv = np.linalg.inv(A)
    Q = A @ V @ M @ U.conj().T
    for p in (0, 1):
        P = D.displacement_matrix(dims, mu, p, dof=12)
        part = D.deflated_part(U, V, M, dims, mu, [p], dof=12)[0]
        assert np.isclose(part + np.trace(P @ Ainv @ (np.eye(A.shape[0]) - Q)), np.trace(P @ Ainv), rtol=1e-10)


def test_lanczos_matches_the_dense_spectrum_of_the_laplacian():
    """Matrix-free Lanczos (full reorthogonalisation) finds the same lowest
    eigenvalues as the dense decomposition, and its vectors are eigenvectors."""
    dims, m2 = [6, 6, 6, 6], 0.05
    op = _lap(dims, m2)
    n = int(np.prod(dims))
    A = D.dense_matrix(op)
    want = np.linalg.eigvalsh(A)[:6]
    th, V = D.lanczos_lowest(lambda x: op.apply(x), n, 6, 15, block=12)     # 180 of 1296 dimensions
    assert np.allclose(th, want, rtol=1e-7, atol=1e-9)
    assert np.allclose(A @ V, V * th[None, :], atol=1e-5)


def test_gamma5_triplets_match_the_dense_svd_of_wilson():
    """gamma5-hermiticity: the lowest singular values of the Wilson operator
    from Lanczos on A^H A = (g5 A)^2 equal those of the dense SVD, and the
    triplets satisfy A V = U diag(s)."""
    from oracle import operators as OO
    from paper_2106_01275_gb300 import inputs
    dims, kappa = [2, 2, 2, 2], 0.12
    Uf = inputs.gauge_links(dims, 7)
    op = OE.Wilson(dims, Uf, kappa)
    N = int(np.prod(dims))
    A = D.dense_matrix(op)
    g5 = lambda x: OO.gamma5_apply(np.asarray(x).reshape(N, 4, 3)).reshape(-1)
    ap = lambda x: np.asarray(op.apply(np.asarray(x).reshape(N, 12))).reshape(-1)
    U, s, V = D.wilson_triplets_from_gamma5(ap, g5, 12 * N, 4, 24)     # the whole space: tests the construction
    _, s_ref, _ = D.lowest_singular_triplets(A, 4)
    assert np.allclose(s, s_ref, rtol=1e-8)
    assert np.allclose(A @ V, U * s[None, :], atol=1e-8)


def test_corrections_equal_the_plain_estimate_under_full_deflation():
    """With every triplet deflated the corrected contraction of each probe is
    zero, so the corrections equal the plain probed estimates."""
    dims, mu, m2 = [4, 2, 2, 2], 0, 0.3
    op = _lap(dims, m2)
    A = D.dense_matrix(op)
    U, s, V = D.lowest_singular_triplets(A, A.shape[0])
    M = D.small_matrix(A @ V, U)
    col, m = greedy_colour(dims, mu, [1], 1, 0)
    corr = D.deflation_corrections(col, m, 5, 2, 0, dims, mu, [0, 1], U, V, M)
    plain = OE.probed_estimates(op, col, m, 5, 2, 0, mu, [0, 1], 1e-13)
    assert np.allclose(corr, plain, rtol=1e-9, atol=1e-10)
