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
