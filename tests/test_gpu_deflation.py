"""GPU parity for the deflation terms of given triplets (Sec. 2.4, Eq. (6)):
the per-probe corrections and the deflated part against the oracle."""
import numpy as np
import pytest

import oracle.estimator as OE
from oracle import deflation as D
from oracle.colouring import greedy_colour
from paper_2106_01275_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_01275_gb300 import build
    build.build()
    from paper_2106_01275_gb300 import ptrace
    return ptrace


@pytest.fixture(scope="module")
def ctx(pt):
    return pt.Context(0)


def _dev(X, N, dof):
    """columns of X (N dof x n_ev) -> torch complex128 [n_ev, N, dof] on the device"""
    import torch
    return torch.as_tensor(np.ascontiguousarray(X.T.reshape(X.shape[1], N, dof).astype(np.complex128))).cuda()


def test_laplacian_deflation_terms(pt, ctx):
    """Any subspace works (Eq. (6) is an identity): seeded random U, V."""
    import torch
    dims, mu, m2 = [4, 4, 4, 4], 1, 0.1
    op_o = OE.Laplacian(dims, m2)
    A = D.dense_matrix(op_o)
    rng = np.random.default_rng(12)
    U = rng.standard_normal((A.shape[0], 6))
    V = rng.standard_normal((A.shape[0], 6))
    M = D.small_matrix(A @ V, U)
    col, m = greedy_colour(dims, mu, [1], 1, 0)
    op = pt.laplacian(ctx, dims, m2)
    ps = [0, 1, 2]
    colt = torch.as_tensor(col).cuda()
    corr, exact = pt.deflation_terms(op, colt, m, mu, ps, "z2", 44, 0, 2, _dev(U, 256, 1), _dev(V, 256, 1), M)
    assert np.allclose(corr, D.deflation_corrections(col, m, 44, 2, 0, dims, mu, ps, U, V, M), rtol=1e-10, atol=1e-10)
    assert np.allclose(exact, D.deflated_part(U, V, M, dims, mu, ps), rtol=1e-10, atol=1e-12)
    # with the solves: the deflated estimate of the engine against the oracle's
    est, _, _, _ = pt.trace(op, colt, m, mu, ps, "z2", 44, 0, 2, True, "mixed_fp32", 1e-10, 5000)
    want = D.deflated_probed_estimates(op_o, col, m, 44, 2, 0, mu, ps, 1e-12, U, V, M)
    assert np.allclose(est - corr, want, rtol=1e-8, atol=1e-8)


def test_wilson_deflation_terms_with_triplets(pt, ctx):
    """Wilson-Dirac, Z4 noise, 12-fold dilution, the lowest singular triplets
    (M = diag(1 / sigma))."""
    import torch
    dims, mu, kappa = [2, 2, 4, 2], 2, 0.12
    Uf = inputs.gauge_links(dims, 19)
    op_o = OE.Wilson(dims, Uf, kappa)
    A = D.dense_matrix(op_o)
    U, s, V = D.lowest_singular_triplets(A, 8)
    M = D.small_matrix(A @ V, U)
    col, m = greedy_colour(dims, mu, [1], 1, 1)
    op = pt.wilson(ctx, dims, torch.as_tensor(Uf).cuda(), kappa, True)
    ps = [0, 1]
    N = int(np.prod(dims))
    colt = torch.as_tensor(col).cuda()
    corr, exact = pt.deflation_terms(op, colt, m, mu, ps, "z4", 8, 0, 1, _dev(U, N, 12), _dev(V, N, 12), M)
    assert np.allclose(corr, D.deflation_corrections(col, m, 8, 1, 1, dims, mu, ps, U, V, M, dof=12), rtol=1e-10,
                       atol=1e-10)
    assert np.allclose(exact, D.deflated_part(U, V, M, dims, mu, ps, dof=12), rtol=1e-10, atol=1e-12)


def _start(rng, block, N, dof, complex_):
    import torch
    X = rng.standard_normal((block, N, dof))
    if complex_:
        X = X + 1j * rng.standard_normal((block, N, dof))
    return torch.as_tensor(X.astype(np.complex128)).cuda()


def test_singular_triplets_laplacian_closed_form(pt, ctx):
    """Block Lanczos on the 6^4 shifted Laplacian: the ten lowest eigenvalues
    against m^2 + sum_mu 4 sin^2(pi n_mu / L) (a 1 + 8 + 1 degenerate pattern),
    the vectors by residual and orthonormality; U = V for an SPD operator."""
    import itertools
    dims, m2, L = [6, 6, 6, 6], 0.05, 6
    N = int(np.prod(dims))
    op = pt.laplacian(ctx, dims, m2)
    start = _start(np.random.default_rng(5), 12, N, 1, False)
    U, s, V = pt.singular_triplets(op, 10, 12, 15, start)
    want = sorted(m2 + sum(4 * np.sin(np.pi * k / L) ** 2 for k in ks)
                  for ks in itertools.product(range(L), repeat=4))[:10]
    assert np.allclose(s, want, rtol=1e-10, atol=0)
    Vh = V.cpu().numpy().reshape(10, N).T
    assert np.abs(Vh.imag).max() == 0.0                       # a real start keeps the basis real
    AV = np.stack([np.asarray(OE.Laplacian(dims, m2).apply(Vh[:, j].real)).reshape(-1) for j in range(10)], axis=1)
    assert np.abs(AV - Vh * s[None, :]).max() < 1e-8
    assert np.abs(Vh.conj().T @ Vh - np.eye(10)).max() < 1e-12
    assert np.array_equal(U.cpu().numpy(), V.cpu().numpy())


def test_singular_triplets_wilson_against_dense_svd(pt, ctx):
    """Wilson-Dirac on 2x2x4x2 with the Krylov space grown to the whole space
    (8 x 48 = 384 vectors): singular values against the dense SVD, A V = U
    diag(s) and orthonormal U, V; the triplets then deflate (Eq. (6)) exactly
    as the dense ones do."""
    import torch
    dims, mu, kappa = [2, 2, 4, 2], 2, 0.12
    N = int(np.prod(dims))
    Uf = inputs.gauge_links(dims, 19)
    op_o = OE.Wilson(dims, Uf, kappa)
    A = D.dense_matrix(op_o)
    op = pt.wilson(ctx, dims, torch.as_tensor(Uf).cuda(), kappa, True)
    start = _start(np.random.default_rng(6), 8, N, 12, True)
    Ug, s, Vg = pt.singular_triplets(op, 6, 8, 48, start)
    _, s_ref, _ = D.lowest_singular_triplets(A, 6)
    assert np.allclose(s, s_ref, rtol=1e-9, atol=0)
    Uh = Ug.cpu().numpy().reshape(6, 12 * N).T
    Vh = Vg.cpu().numpy().reshape(6, 12 * N).T
    assert np.abs(A @ Vh - Uh * s[None, :]).max() < 1e-9
    assert np.abs(Uh.conj().T @ Uh - np.eye(6)).max() < 1e-10
    assert np.abs(Vh.conj().T @ Vh - np.eye(6)).max() < 1e-12
    M = D.small_matrix(A @ Vh, Uh)
    assert np.allclose(M, np.diag(1 / s), atol=1e-8)
    col, m = greedy_colour(dims, mu, [1], 1, 1)
    corr, exact = pt.deflation_terms(op, torch.as_tensor(col).cuda(), m, mu, [0, 1], "z4", 3, 0, 1, Ug, Vg, M)
    assert np.allclose(exact, D.deflated_part(Uh, Vh, M, dims, mu, [0, 1], dof=12), rtol=1e-10, atol=1e-12)
    assert np.allclose(corr, D.deflation_corrections(col, m, 3, 1, 1, dims, mu, [0, 1], Uh, Vh, M, dof=12),
                       rtol=1e-10, atol=1e-10)


def test_singular_triplets_argument_errors(pt, ctx):
    op = pt.laplacian(ctx, [4, 4, 4, 4], 0.1)
    start = _start(np.random.default_rng(1), 65, 256, 1, False)
    for n_ev, block, n_iter in [(0, 4, 4), (17, 4, 4), (2, 65, 2), (2, 64, 17), (2, 0, 4)]:
        with pytest.raises(pt.PtraceError):
            pt.singular_triplets(op, n_ev, block, n_iter, start)
    with pytest.raises(ValueError):                            # fewer start vectors than the block
        pt.singular_triplets(op, 2, 8, 4, start[:4])
