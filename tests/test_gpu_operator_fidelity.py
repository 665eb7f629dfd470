"""GPU parity for the operator-fidelity pieces (Sec. 4.2 names a clover
Wilson-Dirac operator solved by multigrid): the clover site blocks and their
inverses, the even-odd building blocks and solver for the Laplacian, Wilson
and clover operators, the batched even-odd Laplacian trace (Eqs. (1), (5)),
multigrid-preconditioned CG (Laplacian) and adaptive multigrid FGMRES (Wilson,
with and without clover).  Every device entry point is called through the C
ABI and compared with the oracle: element by element for the site blocks and
the even-odd steps (FP64 arithmetic on both sides: 1e-12 to 1e-13), against
dense or oracle solves for the solvers, and against the oracle's probed
estimates (1e-8, the estimator's tolerance) for the trace.  Lattices are
small, with ragged sides where the operator allows them (even-odd needs even
sides, multigrid sides divisible by the block)."""
import numpy as np
import pytest

import oracle.estimator as OE
from oracle import clover as CL
from oracle import deflation as D
from oracle import evenodd as EO
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


def _dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def _wilson(pt, ctx, dims, U, kappa, ap=True):
    return pt.wilson(ctx, dims, _dev(U.astype(np.complex128)), kappa, ap)


def _cplx(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# ---------------------------------------------------------------- clover blocks
@pytest.mark.parametrize("dims,seed", [([2, 3, 2, 4], 1), ([4, 4, 4, 4], 2), ([3, 1, 5, 2], 3), ([6, 4, 2, 8], 4)])
def test_clover_blocks_match_the_oracle(pt, ctx, dims, seed):
    U = inputs.gauge_links(dims, seed, eps=0.8)
    kappa, csw = 0.125, 1.7
    op = _wilson(pt, ctx, dims, U, kappa)
    got = pt.clover_blocks(op, csw).cpu().numpy()
    want = CL.clover_blocks(U, dims, kappa, csw)
    assert np.abs(want).max() > 1e-2
    assert np.abs(got - want).max() < 1e-13 * np.abs(want).max()


def test_clover_blocks_uniform_flux_and_free_field(pt, ctx):
    dims = [4, 6, 2, 2]
    U, phi = CL.uniform_abelian_links(dims, 1, (0, 1))
    got = pt.clover_blocks(_wilson(pt, ctx, dims, U, 0.13), 2.0).cpu().numpy()
    want = -0.13 * 2.0 * np.sin(phi) * np.kron(CL.sigma(0, 1), np.eye(3))
    assert np.allclose(got, want[None], atol=1e-14)
    free = pt.clover_blocks(_wilson(pt, ctx, dims, inputs.unit_links(dims), 0.13), 2.0).cpu().numpy()
    assert np.abs(free).max() == 0.0


def test_site_blocks_invert_and_apply(pt, ctx):
    import torch
    dims = [2, 2, 2, 4]
    U = inputs.gauge_links(dims, 4, eps=0.9)
    C = CL.clover_blocks(U, dims, 0.13, 1.9)
    inv = pt.site_blocks_invert(ctx, _dev(C), 1.0).cpu().numpy()
    assert np.abs(inv - np.linalg.inv(np.eye(12)[None] + C)).max() < 1e-13
    rng = np.random.default_rng(5)
    B = _cplx(rng, (37, 12, 12))                       # a ragged count; pivoting needed
    B[:, 0, 0] = 0.0
    binv = pt.site_blocks_invert(ctx, _dev(B), 0.0).cpu().numpy()
    assert np.allclose(binv @ B, np.eye(12)[None], atol=1e-12)
    x = _cplx(rng, (3, 37, 4, 3))
    y0 = _cplx(rng, (3, 37, 4, 3))
    y = pt.site_blocks_apply(ctx, _dev(B), _dev(x), _dev(y0.copy()), beta=0.5).cpu().numpy()
    want = 0.5 * y0.reshape(3, 37, 12) + np.einsum('nij,rnj->rni', B, x.reshape(3, 37, 12))
    assert np.abs(y.reshape(3, 37, 12) - want).max() < 1e-13 * np.abs(want).max()
    B[11] = 0.0
    with pytest.raises(pt.PtraceError) as ei:
        pt.site_blocks_invert(ctx, _dev(B), 0.0)
    assert ei.value.code == pt.PT_ERR_NUMERIC
    torch.cuda.synchronize()


# ---------------------------------------------------------------- even-odd steps
def test_laplacian_eo_steps_match_the_oracle(pt, ctx):
    dims, m2 = [4, 2, 6, 2], 0.3
    N = int(np.prod(dims))
    eo = EO.LaplacianEO(dims, m2)
    rng = np.random.default_rng(1)
    xe, b = rng.standard_normal((3, N // 2)), rng.standard_normal((3, N))
    op = pt.laplacian(ctx, dims, m2)
    ye = pt.eo_schur(op, _dev(xe)).cpu().numpy()
    be = pt.eo_prepare(op, _dev(b)).cpu().numpy()
    x = pt.eo_reconstruct(op, _dev(xe), _dev(b)).cpu().numpy()
    for r in range(3):
        assert np.allclose(ye[r], eo.schur(xe[r]), rtol=0, atol=1e-13)
        assert np.allclose(be[r], eo.rhs(b[r]), rtol=0, atol=1e-13)
        assert np.allclose(x[r], eo.reconstruct(xe[r], b[r]), rtol=0, atol=1e-13)


@pytest.mark.parametrize("dims,ap", [([2, 2, 4, 2], True), ([4, 2, 2, 6], False), ([4, 4, 2, 4], True)])
def test_wilson_eo_steps_match_the_oracle(pt, ctx, dims, ap):
    kappa, N = 0.13, int(np.prod(dims))
    U = inputs.gauge_links(dims, 31, eps=0.7)
    eo = EO.WilsonEO(dims, U, kappa, ap)
    rng = np.random.default_rng(2)
    xe, b = _cplx(rng, (2, N // 2, 4, 3)), _cplx(rng, (2, N, 4, 3))
    op = _wilson(pt, ctx, dims, U, kappa, ap)
    ye = pt.eo_schur(op, _dev(xe)).cpu().numpy()
    be = pt.eo_prepare(op, _dev(b)).cpu().numpy()
    x = pt.eo_reconstruct(op, _dev(xe), _dev(b)).cpu().numpy()
    for r in range(2):
        assert np.allclose(ye[r].reshape(-1, 12), eo.schur(xe[r].reshape(-1, 12)), rtol=0, atol=1e-13)
        assert np.allclose(be[r].reshape(-1, 12), eo.rhs(b[r]), rtol=0, atol=1e-13)
        assert np.allclose(x[r].reshape(-1, 12), eo.reconstruct(xe[r].reshape(-1, 12), b[r]), rtol=0, atol=1e-13)


def test_clover_eo_blocks_and_steps_match_the_oracle(pt, ctx):
    dims, kappa, csw = [2, 2, 2, 4], 0.12, 1.8
    N = int(np.prod(dims))
    U = inputs.gauge_links(dims, 24, eps=0.8)
    op = _wilson(pt, ctx, dims, U, kappa)
    Aee, Aoo = pt.eo_clover_blocks(op, csw)
    eo = EO.WilsonCloverEO(dims, U, kappa, csw)
    assert np.abs(Aee.cpu().numpy() - eo.Aee).max() < 1e-13
    assert np.abs(Aoo.cpu().numpy() - eo.Aoo_inv).max() < 1e-12
    rng = np.random.default_rng(6)
    xe, b = _cplx(rng, (2, N // 2, 4, 3)), _cplx(rng, (2, N, 4, 3))
    blocks = (Aee, Aoo)
    ye = pt.eo_schur(op, _dev(xe), blocks).cpu().numpy()
    be = pt.eo_prepare(op, _dev(b), blocks).cpu().numpy()
    x = pt.eo_reconstruct(op, _dev(xe), _dev(b), blocks).cpu().numpy()
    for r in range(2):
        assert np.allclose(ye[r].reshape(-1, 12), eo.schur(xe[r].reshape(-1, 12)), rtol=0, atol=1e-12)
        assert np.allclose(be[r].reshape(-1, 12), eo.rhs(b[r]), rtol=0, atol=1e-12)
        assert np.allclose(x[r].reshape(-1, 12), eo.reconstruct(xe[r].reshape(-1, 12), b[r]), rtol=0, atol=1e-12)


# ---------------------------------------------------------------- even-odd solver
def test_eo_solve_laplacian(pt, ctx):
    dims, m2 = [8, 8, 4, 4], 0.05
    N = int(np.prod(dims))
    b = np.random.default_rng(9).standard_normal((2, N))
    op = pt.laplacian(ctx, dims, m2)
    x, its, rel = pt.eo_solve(op, _dev(b), tol=1e-12)
    x = x.cpu().numpy()
    opL = OE.Laplacian(dims, m2)
    for r in range(2):
        xf, its_full, _ = opL.solve(b[r], 1e-12)
        assert rel[r] <= 1e-12
        assert np.allclose(x[r], np.asarray(xf).reshape(-1), rtol=0, atol=1e-9 * np.abs(xf).max())
        assert its[r] <= 0.7 * its_full, (its[r], its_full)
    with pytest.raises(pt.PtraceError) as ei:
        pt.eo_solve(op, _dev(b[:1]), tol=1e-14, maxit=1)
    assert ei.value.code == pt.PT_ERR_NOCONV
    x0, it0, rel0 = pt.eo_solve(op, _dev(np.zeros((1, N))))
    assert np.all(x0.cpu().numpy() == 0) and it0[0] == 0 and rel0[0] == 0.0


def test_eo_solve_wilson_and_clover(pt, ctx):
    dims, kappa, csw = [2, 2, 4, 2], 0.12, 1.5
    N = int(np.prod(dims))
    U = inputs.gauge_links(dims, 41, eps=0.7)
    bw = _cplx(np.random.default_rng(9), (2, N, 4, 3))
    op = _wilson(pt, ctx, dims, U, kappa)
    A = D.dense_matrix(OE.Wilson(dims, U, kappa))
    xw, itw, relw = pt.eo_solve(op, _dev(bw), tol=1e-12)
    xw = xw.cpu().numpy()
    for r in range(2):
        _, its_full, _ = OE.Wilson(dims, U, kappa).solve(bw[r], 1e-12)
        assert relw[r] <= 1e-12 and itw[r] < its_full, (itw[r], its_full)
        assert np.allclose(xw[r].reshape(-1), np.linalg.solve(A, bw[r].reshape(-1)), atol=1e-10)
    blocks = pt.eo_clover_blocks(op, csw)
    xc, _, relc = pt.eo_solve(op, _dev(bw), tol=1e-12, blocks=blocks)
    Ac = D.dense_matrix(CL.WilsonClover(dims, U, kappa, csw))
    for r in range(2):
        assert relc[r] <= 1e-12
        assert np.allclose(xc.cpu().numpy()[r].reshape(-1), np.linalg.solve(Ac, bw[r].reshape(-1)), atol=1e-10)


# ---------------------------------------------------------------- even-odd trace
@pytest.mark.parametrize("dims,m2,mu,ps,cps,k,noise,set0,n_sets", [
    ([4, 4, 4, 4], 0.1, 0, [0, 1, 2], [0, 1, 2], 1, "z2", 0, 2),
    ([6, 4, 2, 8], 0.05, 3, [1, 3], [1, 3], 2, "z2", 3, 2),
    ([8, 8, 4, 4], 0.01, 1, [0, 4], [0, 4], 1, "z2", 0, 1),
    ([2, 2, 2, 2], 0.2, 2, [0, 1, -1], [1], 1, "z2", 1, 2),            # both neighbours along a side of 2 coincide
    ([4, 2, 4, 6], 0.2, 3, [-2, 6, 13], [1], 1, "z2", 1, 2),           # negative and wrapping displacements
    ([4, 4, 2, 2], 0.2, 0, list(range(-16, 16)), [1], 1, "z2", 1, 2),  # the full 32 outputs per solve
])
def test_trace_eo_matches_the_oracle(pt, ctx, dims, m2, mu, ps, cps, k, noise, set0, n_sets):
    col, m = greedy_colour(dims, mu, cps, k, 0)
    op = pt.laplacian(ctx, dims, m2)
    est, st = pt.trace_eo(op, _dev(col.astype(np.int32)), m, mu, ps, noise, 1000, set0, n_sets, tol=1e-11)
    want = OE.probed_estimates(OE.Laplacian(dims, m2), col, m, 1000, n_sets, {"z2": 0, "z4": 1}[noise], mu, ps,
                               1e-13, set0=set0)
    assert np.allclose(est, want, rtol=1e-8, atol=1e-9 * np.abs(want).max())
    assert st["n_rhs"] == n_sets * m and st["n_noconv"] == 0 and st["max_relres"] <= 1e-11
    assert st["kernel_launches"] > 0


def test_trace_eo_batches_and_errors(pt, ctx):
    """Tasks split over several batches (a slot cap below the task count)
    give the same estimates; odd sides and exhausted iterations are reported."""
    dims, m2, mu = [4, 4, 4, 4], 0.1, 2
    col, m = greedy_colour(dims, mu, [1], 2, 0)
    op = pt.laplacian(ctx, dims, m2)
    colt = _dev(col.astype(np.int32))
    full, _ = pt.trace_eo(op, colt, m, mu, [0, 1], "z2", 5, 0, 3, tol=1e-11)
    c2 = pt.Context(0)
    c2.set_max_slots(7)
    op2 = pt.laplacian(c2, dims, m2)
    part, st = pt.trace_eo(op2, colt, m, mu, [0, 1], "z2", 5, 0, 3, tol=1e-11)
    assert st["n_slots"] == 7
    assert np.allclose(part, full, rtol=1e-12, atol=1e-12 * np.abs(full).max())
    with pytest.raises(pt.PtraceError) as ei:
        pt.trace_eo(pt.laplacian(ctx, dims, 0.01), colt, m, mu, [1], "z2", 5, 0, 1, tol=1e-14, maxit=2)
    assert ei.value.code == pt.PT_ERR_NOCONV
    with pytest.raises(pt.PtraceError):                          # complex noise, real operator
        pt.trace_eo(op, colt, m, mu, [1], "z4", 5, 0, 1)
    with pytest.raises(pt.PtraceError):
        odd = pt.laplacian(ctx, [3, 4, 4, 4], m2)
        pt.trace_eo(odd, _dev(np.zeros(192, np.int32)), 1, 0, [1])


# ---------------------------------------------------------------- multigrid
def test_mg_solve_laplacian(pt, ctx):
    dims, m2 = [8, 8, 8, 8], 0.001
    b = np.random.default_rng(5).standard_normal((2, 4096))
    op = pt.laplacian(ctx, dims, m2)
    x, its, rel = pt.mg_solve(op, _dev(b), 2, 2, 0.8, tol=1e-10)
    x = x.cpu().numpy()
    xh, its_h, _ = pt.mg_solve_host(dims, m2, b, 2, 2, 0.8, tol=1e-10)
    for r in range(2):
        xc, its_cg, _ = OE.Laplacian(dims, m2).solve(b[r], 1e-12)
        assert rel[r] <= 1e-10
        assert np.allclose(x[r], np.asarray(xc).reshape(-1), rtol=0, atol=1e-7 * np.abs(xc).max())
        assert its[r] * 3 <= its_cg, (its[r], its_cg)
        assert abs(int(its[r]) - int(its_h[r])) <= 1                  # the host twin, up to summation order
    x4, _, rel4 = pt.mg_solve(op, _dev(b[:1]), 4, 2, 0.8, tol=1e-10)
    assert rel4[0] <= 1e-10 and np.allclose(x4.cpu().numpy()[0], x[0], atol=1e-6 * np.abs(x[0]).max())
    with pytest.raises(pt.PtraceError) as ei:
        pt.mg_solve(op, _dev(b[:1]), tol=1e-14, maxit=2)
    assert ei.value.code == pt.PT_ERR_NOCONV
    x0, it0, rel0 = pt.mg_solve(pt.laplacian(ctx, [4, 4, 4, 4], 0.1), _dev(np.zeros((1, 256))))
    assert np.all(x0.cpu().numpy() == 0) and it0[0] == 0 and rel0[0] == 0.0


def test_mg_solve_ragged(pt, ctx):
    """Sides 6 x 2 x 4 x 2 with blocks of 2 (a coarse side of 1 along dim 1)."""
    dims, m2 = [6, 2, 4, 2], 0.05
    N = int(np.prod(dims))
    b = np.random.default_rng(11).standard_normal((1, N))
    x, _, rel = pt.mg_solve(pt.laplacian(ctx, dims, m2), _dev(b), 2, 3, 0.8, tol=1e-11)
    A = D.dense_matrix(OE.Laplacian(dims, m2))
    assert rel[0] <= 1e-11 and np.allclose(x.cpu().numpy()[0], np.linalg.solve(A, b[0]), atol=1e-9)


def test_wmg_solve_wilson(pt, ctx):
    dims, kappa = [2, 2, 4, 4], 0.124
    N = int(np.prod(dims))
    U = inputs.gauge_links(dims, 5, eps=0.3)
    b = _cplx(np.random.default_rng(3), (2, N, 4, 3))
    op = _wilson(pt, ctx, dims, U, kappa)
    x, its, rel = pt.wmg_solve(op, _dev(b), 2, 4, 20, 2, 0.8, 30, 7, tol=1e-10)
    A = D.dense_matrix(OE.Wilson(dims, U, kappa))
    xh, its_h, _ = pt.wmg_solve_host(dims, U, kappa, b, 2, 4, 20, 2, 0.8, 30, 7, tol=1e-10)
    for r in range(2):
        assert rel[r] <= 1e-10
        assert np.allclose(x.cpu().numpy()[r].reshape(-1), np.linalg.solve(A, b[r].reshape(-1)), atol=1e-8)
        assert abs(int(its[r]) - int(its_h[r])) <= 2, (its, its_h)
    x0, it0, rel0 = pt.wmg_solve(op, _dev(np.zeros((1, N, 4, 3), np.complex128)))
    assert np.all(x0.cpu().numpy() == 0) and it0[0] == 0 and rel0[0] == 0.0


def test_wmg_solve_larger_and_clover(pt, ctx):
    dims, kappa, csw = [4, 4, 4, 4], 0.12, 1.7
    N = int(np.prod(dims))
    U = inputs.gauge_links(dims, 8, eps=0.4)
    b = np.random.default_rng(4).standard_normal((1, N, 4, 3)).astype(np.complex128)
    op = _wilson(pt, ctx, dims, U, kappa)
    x, _, rel = pt.wmg_solve(op, _dev(b), 2, 4, 20, 2, 0.8, 30, 1, tol=1e-10)
    xo, _, _ = OE.Wilson(dims, U, kappa).solve(b[0], 1e-12)
    assert rel[0] <= 1e-10 and np.allclose(x.cpu().numpy()[0].reshape(-1), np.asarray(xo).reshape(-1), atol=1e-8)
    xc, _, relc = pt.wmg_solve(op, _dev(b), 2, 4, 20, 2, 0.8, 30, 1, tol=1e-10, csw=csw)
    xco, _, _ = CL.WilsonClover(dims, U, kappa, csw).solve(b[0], 1e-12)
    assert relc[0] <= 1e-10
    assert np.allclose(xc.cpu().numpy()[0].reshape(-1), np.asarray(xco).reshape(-1), atol=1e-8)
