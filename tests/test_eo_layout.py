"""Even-odd half-field layout of the library (pt_eo_layout, host only; the
same index functions run in the even-odd kernels) against the oracle's
even / odd split and its neighbour tables.  No GPU needed."""
import numpy as np
import pytest

from oracle import evenodd as EO
from oracle import operators as ops


@pytest.mark.parametrize("dims", [[2, 2, 2, 2], [4, 2, 6, 2], [6, 4, 2, 8], [2, 4, 4, 6], [8, 8, 8, 16]])
def test_layout_matches_the_oracle_split(ptlib, dims):
    ev, od = EO.split(dims)
    fwd, bwd = ops.neighbour_tables(dims)
    for parity, mine, other in ((0, ev, od), (1, od, ev)):
        site, nbr = ptlib.eo_layout(dims, parity)
        assert np.array_equal(site, mine)                               # storage order within the parity
        assert np.array_equal(site >> 1, np.arange(site.size))          # entry h holds site 2h or 2h + 1
        for mu in range(4):
            assert np.array_equal(other[nbr[:, 2 * mu]], fwd[mu][mine])  # x + mu, in the other parity
            assert np.array_equal(other[nbr[:, 2 * mu + 1]], bwd[mu][mine])


def test_odd_sides_refused(ptlib):
    with pytest.raises(ptlib.PtraceError):
        ptlib.eo_layout([4, 3, 4, 4], 0)
    with pytest.raises(ptlib.PtraceError):
        ptlib.eo_layout([4, 4, 4, 4], 2)


def test_laplacian_steps_on_the_host_match_the_oracle(ptlib):
    """The library's even-odd site arithmetic and sequence of steps (run on
    the host): S, b'_e and the reconstruction against the oracle, and the
    composed even solve reproduces A^{-1} b."""
    from oracle import deflation as D
    import oracle.estimator as OE
    dims, m2 = [4, 2, 6, 2], 0.3
    N = int(np.prod(dims))
    eo = EO.LaplacianEO(dims, m2)
    rng = np.random.default_rng(1)
    xe = rng.standard_normal((2, N // 2))
    b = rng.standard_normal((2, N))
    ye = ptlib.eo_host(0, dims, 0, xe, m2=m2)
    be = ptlib.eo_host(0, dims, 1, b, m2=m2)
    x = ptlib.eo_host(0, dims, 2, xe, b, m2=m2)
    for r in range(2):
        assert np.allclose(ye[r], eo.schur(xe[r]), rtol=0, atol=1e-13)
        assert np.allclose(be[r], eo.rhs(b[r]), rtol=0, atol=1e-13)
        assert np.allclose(x[r], eo.reconstruct(xe[r], b[r]), rtol=0, atol=1e-13)
    S = ptlib.eo_host(0, dims, 0, np.eye(N // 2), m2=m2).T              # column j = S e_j
    x_e = np.linalg.solve(S, be[0])
    xs = ptlib.eo_host(0, dims, 2, x_e[None], b[:1], m2=m2)[0]
    assert np.allclose(xs, np.linalg.solve(D.dense_matrix(OE.Laplacian(dims, m2)), b[0]), atol=1e-12)


@pytest.mark.parametrize("dims,ap", [([2, 2, 4, 2], True), ([4, 2, 2, 6], False)])
def test_wilson_steps_on_the_host_match_the_oracle(ptlib, dims, ap):
    from oracle import deflation as D
    import oracle.estimator as OE
    from paper_2106_01275_gb300 import inputs
    kappa, N = 0.13, int(np.prod(dims))
    U = inputs.gauge_links(dims, 31, eps=0.7)
    eo = EO.WilsonEO(dims, U, kappa, ap)
    rng = np.random.default_rng(2)
    xe = rng.standard_normal((2, N // 2, 4, 3)) + 1j * rng.standard_normal((2, N // 2, 4, 3))
    b = rng.standard_normal((2, N, 4, 3)) + 1j * rng.standard_normal((2, N, 4, 3))
    kw = dict(kappa=kappa, U=U, antiperiodic_t=ap)
    ye = ptlib.eo_host(1, dims, 0, xe, **kw)
    be = ptlib.eo_host(1, dims, 1, b, **kw)
    x = ptlib.eo_host(1, dims, 2, xe, b, **kw)
    for r in range(2):
        assert np.allclose(ye[r].reshape(-1, 12), eo.schur(xe[r].reshape(-1, 12)), rtol=0, atol=1e-13)
        assert np.allclose(be[r].reshape(-1, 12), eo.rhs(b[r]), rtol=0, atol=1e-13)
        assert np.allclose(x[r].reshape(-1, 12), eo.reconstruct(xe[r].reshape(-1, 12), b[r]), rtol=0, atol=1e-13)
    n_e = 6 * N
    S = ptlib.eo_host(1, dims, 0, np.eye(n_e).reshape(n_e, N // 2, 4, 3), **kw).reshape(n_e, n_e).T
    x_e = np.linalg.solve(S, be[0].reshape(-1)).reshape(1, N // 2, 4, 3)
    xs = ptlib.eo_host(1, dims, 2, x_e, b[:1], **kw)[0]
    A = D.dense_matrix(OE.Wilson(dims, U, kappa, ap))
    assert np.allclose(xs.reshape(-1), np.linalg.solve(A, b[0].reshape(-1)), atol=1e-11)


def test_clover_steps_on_the_host_match_the_oracle(ptlib):
    """With the clover site blocks (A_ee = 1 + C_ee, A_oo^{-1} per site) the
    steps match the oracle's clover Schur complement and compose to A_c^{-1} b."""
    from oracle import clover as CL
    from oracle import deflation as D
    from paper_2106_01275_gb300 import inputs
    dims, kappa, csw = [2, 2, 2, 4], 0.12, 1.8
    N = int(np.prod(dims))
    U = inputs.gauge_links(dims, 24, eps=0.8)
    C = ptlib.clover_blocks_host(dims, U, kappa, csw)
    ev, od = EO.split(dims)
    Aee = np.eye(12)[None] + C[ev]
    Aoo_inv = ptlib.site_blocks_invert_host(C[od], 1.0)
    eo = EO.WilsonCloverEO(dims, U, kappa, csw)
    rng = np.random.default_rng(6)
    xe = rng.standard_normal((2, N // 2, 4, 3)) + 1j * rng.standard_normal((2, N // 2, 4, 3))
    b = rng.standard_normal((2, N, 4, 3)) + 1j * rng.standard_normal((2, N, 4, 3))
    kw = dict(kappa=kappa, U=U, blocks=(Aee, Aoo_inv))
    ye = ptlib.eo_host(1, dims, 0, xe, **kw)
    be = ptlib.eo_host(1, dims, 1, b, **kw)
    x = ptlib.eo_host(1, dims, 2, xe, b, **kw)
    for r in range(2):
        assert np.allclose(ye[r].reshape(-1, 12), eo.schur(xe[r].reshape(-1, 12)), rtol=0, atol=1e-12)
        assert np.allclose(be[r].reshape(-1, 12), eo.rhs(b[r]), rtol=0, atol=1e-12)
        assert np.allclose(x[r].reshape(-1, 12), eo.reconstruct(xe[r].reshape(-1, 12), b[r]), rtol=0, atol=1e-12)
    n_e = 6 * N
    S = ptlib.eo_host(1, dims, 0, np.eye(n_e).reshape(n_e, N // 2, 4, 3), **kw).reshape(n_e, n_e).T
    x_e = np.linalg.solve(S, be[0].reshape(-1)).reshape(1, N // 2, 4, 3)
    xs = ptlib.eo_host(1, dims, 2, x_e, b[:1], **kw)[0]
    A = D.dense_matrix(CL.WilsonClover(dims, U, kappa, csw))
    assert np.allclose(xs.reshape(-1), np.linalg.solve(A, b[0].reshape(-1)), atol=1e-11)
    with pytest.raises(ptlib.PtraceError):                       # no site blocks for the Laplacian
        ptlib.eo_host(0, dims, 0, np.zeros((1, N // 2)), m2=0.1, blocks=(Aee, Aoo_inv))


def test_even_solve_on_the_host(ptlib):
    """The building-block solver (host executor): A^{-1} b for the Laplacian,
    Wilson and clover operators against dense solves; the even Laplacian
    system needs about half the CG iterations of the full one (cond(S) is
    about four times smaller) and Wilson fewer BiCGStab iterations; maxit
    exhaustion is reported; b = 0 gives x = 0 with no iteration."""
    from oracle import clover as CL
    from oracle import deflation as D
    import oracle.estimator as OE
    from paper_2106_01275_gb300 import inputs
    rng = np.random.default_rng(9)
    dims, m2 = [8, 8, 4, 4], 0.05
    N = int(np.prod(dims))
    b = rng.standard_normal((2, N))
    x, its, rel = ptlib.eo_solve_host(0, dims, b, tol=1e-12, m2=m2)
    opL = OE.Laplacian(dims, m2)
    for r in range(2):
        xf, its_full, _ = opL.solve(b[r], 1e-12)
        assert np.allclose(x[r], np.asarray(xf).reshape(-1), rtol=0, atol=1e-9 * np.abs(xf).max())
        assert rel[r] <= 1e-12 and its[r] <= 0.7 * its_full, (its[r], its_full)
    dims = [2, 2, 4, 2]
    N = int(np.prod(dims))
    U = inputs.gauge_links(dims, 41, eps=0.7)
    bw = rng.standard_normal((1, N, 4, 3)) + 1j * rng.standard_normal((1, N, 4, 3))
    xw, itw, relw = ptlib.eo_solve_host(1, dims, bw, tol=1e-12, kappa=0.12, U=U)
    A = D.dense_matrix(OE.Wilson(dims, U, 0.12))
    assert np.allclose(xw[0].reshape(-1), np.linalg.solve(A, bw[0].reshape(-1)), atol=1e-10)
    _, its_full, _ = OE.Wilson(dims, U, 0.12).solve(bw[0], 1e-12)
    assert relw[0] <= 1e-12 and itw[0] < its_full, (itw[0], its_full)
    C = ptlib.clover_blocks_host(dims, U, 0.12, 1.5)
    ev, od = EO.split(dims)
    blocks = (np.eye(12)[None] + C[ev], ptlib.site_blocks_invert_host(C[od], 1.0))
    xc, _, relc = ptlib.eo_solve_host(1, dims, bw, tol=1e-12, kappa=0.12, U=U, blocks=blocks)
    Ac = D.dense_matrix(CL.WilsonClover(dims, U, 0.12, 1.5))
    assert relc[0] <= 1e-12 and np.allclose(xc[0].reshape(-1), np.linalg.solve(Ac, bw[0].reshape(-1)), atol=1e-10)
    with pytest.raises(ptlib.PtraceError) as ei:
        ptlib.eo_solve_host(0, [4, 4, 4, 4], rng.standard_normal((1, 256)), tol=1e-14, maxit=1, m2=0.01)
    assert ei.value.code == ptlib.PT_ERR_NOCONV
    x0, it0, rel0 = ptlib.eo_solve_host(0, [4, 4, 4, 4], np.zeros((1, 256)), m2=0.1)
    assert np.all(x0 == 0) and it0[0] == 0 and rel0[0] == 0.0
