"""The library's adaptive multigrid for Wilson (pt_wmg_solve), run by its host
twin (the same site arithmetic and steps; no GPU): the prolongator is
orthonormal and commutes with g5, the nine-point coarse stencil equals the
dense Galerkin product P^H A P with the oracle's operator (coarse sides of 1
and 2, where stencil slots fold onto one block), and the preconditioned
FGMRES reproduces dense and oracle solutions in fewer iterations than
unpreconditioned GMRES."""
import numpy as np
import pytest

import oracle.estimator as OE
from oracle import deflation as D
from oracle import multigrid as MG
from paper_2106_01275_gb300 import inputs


def _dense_P(P, dims, b):
    Nc, _, nv, bs, _ = P.shape
    N = int(np.prod(dims))
    cd = [d // b for d in dims]
    M = np.zeros((12 * N, Nc * 2 * nv), dtype=np.complex128)
    for B in range(Nc):
        c = [B % cd[0], (B // cd[0]) % cd[1], (B // (cd[0] * cd[1])) % cd[2], B // (cd[0] * cd[1] * cd[2])]
        for sl in range(bs):
            k = [sl % b, (sl // b) % b, (sl // (b * b)) % b, sl // (b * b * b)]
            x = [c[mu] * b + k[mu] for mu in range(4)]
            i = x[0] + dims[0] * (x[1] + dims[1] * (x[2] + dims[2] * x[3]))
            for a in range(2):
                for v in range(nv):
                    M[12 * i + 6 * a:12 * i + 6 * a + 6, (B * 2 + a) * nv + v] = P[B, a, v, sl]
    return M


def _dense_coarse(Ac, cd):
    Nc, _, dc, _ = Ac.shape
    out = np.zeros((Nc * dc, Nc * dc), dtype=np.complex128)
    for B in range(Nc):
        c = [B % cd[0], (B // cd[0]) % cd[1], (B // (cd[0] * cd[1])) % cd[2], B // (cd[0] * cd[1] * cd[2])]
        for d in range(9):
            cc = list(c)
            if d:
                mu, s = (d - 1) // 2, (1 if (d - 1) % 2 == 0 else -1)
                cc[mu] = (cc[mu] + s) % cd[mu]
            Bn = cc[0] + cd[0] * (cc[1] + cd[1] * (cc[2] + cd[2] * cc[3]))
            out[B * dc:(B + 1) * dc, Bn * dc:(Bn + 1) * dc] += Ac[B, d]
    return out


@pytest.mark.parametrize("dims,ap", [([2, 2, 4, 4], True), ([4, 2, 2, 4], False)])
def test_setup_against_the_dense_galerkin_product(ptlib, dims, ap):
    kappa, b, nv = 0.12, 2, 3
    N = int(np.prod(dims))
    U = inputs.gauge_links(dims, 13, eps=0.5)
    P, Ac = ptlib.wmg_setup_host(dims, U, kappa, b, nv, 10, 0.8, 5, antiperiodic_t=ap)
    Pd = _dense_P(P, dims, b)
    assert np.allclose(Pd.conj().T @ Pd, np.eye(Pd.shape[1]), atol=1e-12)
    g5 = np.tile(np.repeat([1.0, 1.0, -1.0, -1.0], 3), N)
    G5c = np.tile(np.repeat([1.0, -1.0], nv), Pd.shape[1] // (2 * nv))
    assert np.allclose(g5[:, None] * Pd, Pd * G5c[None, :])
    A = D.dense_matrix(OE.Wilson(dims, U, kappa, ap))
    want = Pd.conj().T @ A @ Pd
    got = _dense_coarse(Ac, [d // b for d in dims])
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()
    assert np.allclose(G5c[:, None] * got * G5c[None, :], got.conj().T, atol=1e-12)


def test_solve_against_dense_and_unpreconditioned(ptlib):
    dims, kappa = [2, 2, 4, 4], 0.124
    N = int(np.prod(dims))
    U = inputs.gauge_links(dims, 5, eps=0.3)
    rng = np.random.default_rng(3)
    b = rng.standard_normal((1, N, 4, 3)) + 1j * rng.standard_normal((1, N, 4, 3))
    x, its, rel = ptlib.wmg_solve_host(dims, U, kappa, b, 2, 4, 20, 2, 0.8, 30, 7, tol=1e-10)
    A = D.dense_matrix(OE.Wilson(dims, U, kappa))
    assert rel[0] <= 1e-10 and np.allclose(x[0].reshape(-1), np.linalg.solve(A, b[0].reshape(-1)), atol=1e-8)
    _, its_plain, _ = MG.gmres(lambda v: A @ v, b[0].reshape(-1), tol=1e-10, restart=30)
    assert its[0] < its_plain, (its[0], its_plain)


def test_solve_on_a_larger_lattice(ptlib):
    """4^4 (coarse 2^4: every stencil direction folds onto one neighbour),
    against the oracle's BiCGStab solution."""
    dims, kappa = [4, 4, 4, 4], 0.12
    N = int(np.prod(dims))
    U = inputs.gauge_links(dims, 8, eps=0.4)
    b = np.random.default_rng(4).standard_normal((1, N, 4, 3)).astype(np.complex128)
    x, its, rel = ptlib.wmg_solve_host(dims, U, kappa, b, 2, 4, 20, 2, 0.8, 30, 1, tol=1e-10)
    xo, its_o, _ = OE.Wilson(dims, U, kappa).solve(b[0], 1e-12)
    assert rel[0] <= 1e-10 and np.allclose(x[0].reshape(-1), np.asarray(xo).reshape(-1), atol=1e-8)


def test_errors(ptlib):
    dims = [2, 2, 4, 4]
    U = inputs.gauge_links(dims, 1)
    b = np.zeros((1, 64, 4, 3), dtype=np.complex128)
    with pytest.raises(ptlib.PtraceError):
        ptlib.wmg_solve_host([2, 2, 4, 6], inputs.gauge_links([2, 2, 4, 6], 1), 0.12, np.zeros((1, 96, 4, 3)), 4)
    with pytest.raises(ptlib.PtraceError):
        ptlib.wmg_solve_host(dims, U, 0.12, b, 2, 9)                                   # nv > 8
    x, its, rel = ptlib.wmg_solve_host(dims, U, 0.12, b)
    assert np.all(x == 0) and its[0] == 0 and rel[0] == 0.0


def test_clover_operator(ptlib):
    """c_sw != 0: the fine operator is A_W + C; the coarse stencil equals the
    dense P^H A_c P and the solve reproduces the dense clover solve."""
    from oracle import clover as CL
    dims, kappa, csw, b, nv = [2, 2, 4, 4], 0.12, 1.7, 2, 3
    N = int(np.prod(dims))
    U = inputs.gauge_links(dims, 21, eps=0.6)
    P, Ac = ptlib.wmg_setup_host(dims, U, kappa, b, nv, 10, 0.8, 2, csw=csw)
    Pd = _dense_P(P, dims, b)
    A = D.dense_matrix(CL.WilsonClover(dims, U, kappa, csw))
    want = Pd.conj().T @ A @ Pd
    got = _dense_coarse(Ac, [d // b for d in dims])
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()
    _, Ac0 = ptlib.wmg_setup_host(dims, U, kappa, b, nv, 10, 0.8, 2)
    assert np.abs(Ac - Ac0).max() > 1e-3                                     # the clover term is there
    rhs = np.random.default_rng(8).standard_normal((1, N, 4, 3)) + 0j
    x, its, rel = ptlib.wmg_solve_host(dims, U, kappa, rhs, 2, 4, 20, 2, 0.8, 30, 7, tol=1e-10, csw=csw)
    assert rel[0] <= 1e-10 and np.allclose(x[0].reshape(-1), np.linalg.solve(A, rhs[0].reshape(-1)), atol=1e-8)
