"""The library's two-level multigrid for the Laplacian (pt_mg_solve), run by
its host twin (the same site arithmetic and steps; no GPU): one cycle equals
the oracle's two-grid operator, the preconditioned CG reproduces CG's
solution in a fraction of its iterations, blocks of side 4 work, and the
errors are reported."""
import numpy as np
import pytest

import oracle.estimator as OE
from oracle import multigrid as MG
from oracle import operators as ops


def _lap(dims, m2):
    return lambda x: np.asarray(ops.laplacian_apply(np.asarray(x).reshape(-1), dims, m2)).reshape(-1)


@pytest.mark.parametrize("dims,block,nu", [([4, 4, 4, 4], 2, 2), ([8, 4, 4, 8], 4, 1), ([6, 2, 4, 2], 2, 3)])
def test_cycle_matches_the_oracle(ptlib, dims, block, nu):
    m2, N = 0.01, int(np.prod(dims))
    M = MG.TwoGrid(_lap(dims, m2), np.full(N, 8 + m2), MG.prolongator_constant(dims, block), nu=nu, omega=0.8)
    rng = np.random.default_rng(4)
    for _ in range(2):
        r = rng.standard_normal(N)
        want = M(r)
        got = ptlib.mg_cycle_host(dims, m2, r, block, nu, 0.8)
        assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()


def test_preconditioned_solve(ptlib):
    dims, m2 = [8, 8, 8, 8], 0.001
    b = np.random.default_rng(5).standard_normal((2, 4096))
    x, its, rel = ptlib.mg_solve_host(dims, m2, b, 2, 2, 0.8, tol=1e-10)
    for r in range(2):
        xc, its_cg, _ = OE.Laplacian(dims, m2).solve(b[r], 1e-12)
        assert rel[r] <= 1e-10
        assert np.allclose(x[r], np.asarray(xc).reshape(-1), rtol=0, atol=1e-7 * np.abs(xc).max())
        assert its[r] * 3 <= its_cg, (its[r], its_cg)
    x4, its4, rel4 = ptlib.mg_solve_host(dims, m2, b[:1], 4, 2, 0.8, tol=1e-10)
    assert rel4[0] <= 1e-10 and np.allclose(x4[0], x[0], atol=1e-6 * np.abs(x[0]).max())


def test_errors(ptlib):
    with pytest.raises(ptlib.PtraceError):
        ptlib.mg_solve_host([4, 4, 6, 4], 0.1, np.ones((1, 384)), block=4)            # 4 does not divide 6
    with pytest.raises(ptlib.PtraceError):
        ptlib.mg_cycle_host([4, 4, 4, 4], 0.1, np.ones(256), nu=2, omega=1.5)
    rng = np.random.default_rng(6)
    with pytest.raises(ptlib.PtraceError) as ei:
        ptlib.mg_solve_host([8, 8, 8, 8], 0.001, rng.standard_normal((1, 4096)), tol=1e-14, maxit=2)
    assert ei.value.code == ptlib.PT_ERR_NOCONV
    x0, it0, rel0 = ptlib.mg_solve_host([4, 4, 4, 4], 0.1, np.zeros((1, 256)))
    assert np.all(x0 == 0) and it0[0] == 0 and rel0[0] == 0.0
