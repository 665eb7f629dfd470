"""Host-only Rayleigh-Ritz eigensolver of the singular-triplet solver
(pt_hermitian_eig): eigenvalues against closed forms and numpy's eigvalsh,
eigenvectors by residual and orthonormality, degenerate clusters, the
degenerate sizes and the error paths.  No GPU needed."""
import numpy as np
import pytest


def _check_pairs(T, w, X, tol):
    m = T.shape[0]
    scale = max(1.0, np.abs(w).max())
    assert np.all(np.diff(w) >= -1e-12 * scale)
    n = X.shape[1]
    assert np.abs(T @ X - X * w[None, :n]).max() <= tol * scale
    assert np.abs(X.conj().T @ X - np.eye(n)).max() <= tol * max(1, m) ** 0.5


def test_path_graph_laplacian_closed_form(ptlib):
    """tridiagonal (-1, 2, -1): eigenvalues 2 - 2 cos(pi j / (m + 1))"""
    for m in (1, 2, 3, 17, 100):
        T = 2 * np.eye(m) - np.eye(m, k=1) - np.eye(m, k=-1)
        w, X = ptlib.hermitian_eig(T, m)
        want = 2 - 2 * np.cos(np.pi * np.arange(1, m + 1) / (m + 1))
        assert np.allclose(w, want, rtol=0, atol=1e-13)
        _check_pairs(T, w, X, 1e-12)


def test_random_hermitian_against_eigvalsh(ptlib):
    rng = np.random.default_rng(7)
    for m in (4, 33, 160):
        Y = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
        T = Y + Y.conj().T
        w, X = ptlib.hermitian_eig(T, 10 if m > 10 else m)
        assert np.allclose(w, np.linalg.eigvalsh(T), rtol=0, atol=1e-11 * np.abs(w).max())
        _check_pairs(T, w, X, 1e-11)


def test_degenerate_clusters_give_orthonormal_bases(ptlib):
    """eigenvalues of multiplicity 5 and 3 (the shape of a lattice Laplacian's
    spectrum): the lowest vectors still span eigenspaces orthonormally"""
    rng = np.random.default_rng(8)
    m = 40
    Q, _ = np.linalg.qr(rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m)))
    lam = np.sort(rng.uniform(1, 5, m))
    lam[:5] = 0.25
    lam[5:8] = 1.0
    T = (Q * lam) @ Q.conj().T
    w, X = ptlib.hermitian_eig(T, 8)
    assert np.allclose(w, lam, atol=1e-12)
    _check_pairs(T, w, X, 1e-11)
    P5 = Q[:, :5] @ Q[:, :5].conj().T                         # projector on the 5-fold space
    assert np.allclose(P5 @ X[:, :5], X[:, :5], atol=1e-11)


def test_special_matrices(ptlib):
    w, X = ptlib.hermitian_eig(np.zeros((6, 6)), 6)            # zero matrix
    assert np.all(w == 0) and np.allclose(X.conj().T @ X, np.eye(6))
    D = np.diag([3.0, -1.0, 2.0, -1.0])                       # already diagonal, a repeated value
    w, X = ptlib.hermitian_eig(D, 4)
    assert np.array_equal(w, [-1.0, -1.0, 2.0, 3.0])
    _check_pairs(D, w, X, 1e-14)
    # complex tridiagonal (no reflector needed; only the phases D act)
    m = 9
    b = np.exp(1j * np.arange(m - 1)) * (1 + np.arange(m - 1))
    T = np.diag(np.arange(m, dtype=float)) + np.diag(b, -1) + np.diag(b.conj(), 1)
    w, X = ptlib.hermitian_eig(T, m)
    assert np.allclose(w, np.linalg.eigvalsh(T), atol=1e-12)
    _check_pairs(T, w, X, 1e-12)
    # only the Hermitian part counts
    rng = np.random.default_rng(9)
    Y = rng.standard_normal((12, 12)) + 1j * rng.standard_normal((12, 12))
    w, _ = ptlib.hermitian_eig(Y, 0)
    assert np.allclose(w, np.linalg.eigvalsh(0.5 * (Y + Y.conj().T)), atol=1e-12)


def test_errors(ptlib):
    with pytest.raises(ptlib.PtraceError):
        ptlib.hermitian_eig(np.full((3, 3), np.nan), 1)
    with pytest.raises(ptlib.PtraceError):
        ptlib.hermitian_eig(np.eye(3), 4)
    T = np.zeros((1, 1), dtype=np.complex128)
    assert ptlib.lib().pt_hermitian_eig(0, ptlib._np_ptr(T), 0, ptlib._np_ptr(np.zeros(1)), None) == ptlib.PT_ERR_ARG
