"""GPU parity for the clover Wilson operator in the batched engine
(pt_op_set_clover): the engine solves A_c = A_W + C (the clover term of
Sec. 4.2's operator class) on the even Schur complement
S = A_ee - kappa^2 D_eo A_oo^{-1} D_oe.  Traces (Eqs. (1), (5)) against the
oracle's clover operator at 1e-8 in every inner precision, solves checked
through the oracle's operator, pt_apply with the clover term, and the
refusals (odd sides, the gradient)."""
import numpy as np
import pytest

import oracle.clover as CL
import oracle.estimator as OE
import oracle.operators as OO
from oracle.colouring import greedy_colour

pytestmark = pytest.mark.gpu

PRECS = ("fp64", "mixed_fp32", "mixed_bf16")


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


def _t(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def _links(dims, seed):
    from paper_2106_01275_gb300 import inputs
    return inputs.gauge_links(dims, seed)


def test_clover_apply_matches_oracle(pt, ctx):
    """pt_apply of a clover operator is A_W x + C x (the term in FP64)."""
    dims, kappa, csw = [4, 2, 4, 6], 0.12, 1.3
    U = _links(dims, 7)
    op = pt.wilson(ctx, dims, _t(U), kappa, True)
    pt.set_clover(op, csw)
    N = int(np.prod(dims))
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, N, 4, 3)) + 1j * rng.standard_normal((2, N, 4, 3))
    y = pt.apply(op, _t(x), "fp64").cpu().numpy()
    for j in range(2):
        want = CL.clover_apply(x[j], U, kappa, csw, dims, True)
        assert np.abs(y[j] - want).max() <= 1e-12 * np.abs(want).max()
    y32 = pt.apply(op, _t(x), "mixed_fp32").cpu().numpy()
    want = CL.clover_apply(x[0], U, kappa, csw, dims, True)
    assert np.abs(y32[0] - want).max() <= 1e-5 * np.abs(want).max()
    pt.set_clover(op, 0.0)                                   # back to the Wilson operator
    y0 = pt.apply(op, _t(x), "fp64").cpu().numpy()
    want0 = OO.wilson_apply(x[1], U, kappa, dims, True)
    assert np.abs(y0[1] - want0).max() <= 1e-12 * np.abs(want0).max()


@pytest.mark.parametrize("dims,antip,csw", [([4, 4, 4, 8], True, 1.0), ([2, 4, 6, 4], False, 1.7),
                                            ([6, 2, 2, 4], True, 0.6)])
def test_clover_trace_matches_oracle(pt, ctx, dims, antip, csw):
    """Diluted Z4 traces of the clover operator, every inner precision,
    against the oracle (BiCGStab on A_W + C to 1e-12)."""
    kappa, mu = 0.12, 2
    U = _links(dims, 1234)
    col, m = greedy_colour(dims, mu, [1], 1, 0)
    op = pt.wilson(ctx, dims, _t(U), kappa, antip)
    pt.set_clover(op, csw)
    want = OE.probed_estimates(CL.WilsonClover(dims, U, kappa, csw, antip), col, m, 1000, 2, 1, mu, [0, 1, 2],
                               1e-12)
    plain = OE.probed_estimates(OE.Wilson(dims, U, kappa, antip), col, m, 1000, 2, 1, mu, [0, 1, 2], 1e-12)
    assert np.abs(want - plain).max() > 1e-3 * np.abs(plain).max()     # the term matters at this size
    for prec in PRECS:
        est, _, _, st = pt.trace(op, _t(col), m, mu, [0, 1, 2], "z4", 1000, 0, 2, True, prec, 1e-10, 5000)
        assert np.allclose(est, want, rtol=1e-8, atol=1e-7), prec
        assert st["max_relres"] <= 1e-10 and st["n_noconv"] == 0


def test_clover_undiluted_solve_and_item_shapes(pt, ctx):
    """Undiluted probes with 20 displacements (the 32-output contraction),
    pt_solve's rebuilt odd half x_o = A_oo^{-1} (b_o + kappa D_oe x_e)
    checked through the oracle's operator, and two CTA shapes."""
    import torch
    dims, kappa, csw, mu = [4, 2, 4, 4], 0.11, 1.2, 2
    U = _links(dims, 3)
    col, m = greedy_colour(dims, mu, [1], 1, 1)
    op = pt.wilson(ctx, dims, _t(U), kappa, True)
    pt.set_clover(op, csw)
    ps = list(range(-10, 10))
    want = OE.probed_estimates(CL.WilsonClover(dims, U, kappa, csw), col, m, 5, 2, 1, mu, ps, 1e-12,
                               dilute=False)
    for cta in (64, 256):
        pt.set_tuning(op, "mixed_fp32", cta_threads=cta)
        est, _, _, _ = pt.trace(op, _t(col), m, mu, ps, "z4", 5, 0, 2, False, "mixed_fp32", 1e-10, 5000)
        assert np.allclose(est, want, rtol=1e-8, atol=1e-7), cta
    pt.set_tuning(op, "mixed_fp32", reset=True)
    N = int(np.prod(dims))
    B = np.random.default_rng(4).standard_normal((3, N, 4, 3, 2))
    for prec in PRECS:
        X, _, relres, _ = pt.solve(op, _t(B), prec, 1e-10, 5000)
        Xc = X.cpu().numpy()
        for j in range(3):
            b = B[j][..., 0] + 1j * B[j][..., 1]
            x = Xc[j][..., 0] + 1j * Xc[j][..., 1]
            r = b - CL.clover_apply(x, U, kappa, csw, dims, True)
            assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(b), prec
            assert relres[j] <= 1e-10
    Z, it0, _, _ = pt.solve(op, _t(np.zeros((1, N, 4, 3, 2))), "mixed_fp32", 1e-10, 100)
    assert torch.count_nonzero(Z).item() == 0 and it0[0] == 0


def test_clover_autotune_keeps_even_odd(pt, ctx):
    """The autotuner leaves the clover operator on the even-odd engine with
    one right-hand side per item; the tuned run matches the oracle."""
    dims, kappa, csw, mu = [4, 4, 4, 4], 0.12, 1.0, 1
    U = _links(dims, 11)
    col, m = greedy_colour(dims, mu, [1], 1, 0)
    op = pt.wilson(ctx, dims, _t(U), kappa, True)
    pt.set_clover(op, csw)
    t = pt.autotune(op, _t(col), m, mu, "z4", 9, "mixed_fp32", 1e-10, 5000, 24)
    assert t["evenodd"] == 1 and t["rhs_block"] == 1
    est, _, _, st = pt.trace(op, _t(col), m, mu, [0, 1], "z4", 9, 0, 1, True, "mixed_fp32", 1e-10, 5000)
    want = OE.probed_estimates(CL.WilsonClover(dims, U, kappa, csw), col, m, 9, 1, 1, mu, [0, 1], 1e-12)
    assert np.allclose(est, want, rtol=1e-8, atol=1e-7)
    pt.set_tuning(op, "mixed_fp32", reset=True)


def test_clover_refusals(pt, ctx):
    """An odd side cannot carry the clover term (the engine runs it on the
    even Schur complement only), nor can the Laplacian; the gradient refuses
    a clover operator; the context keeps working."""
    dims = [3, 2, 2, 2]
    op = pt.wilson(ctx, dims, _t(_links(dims, 5)), 0.12, True)
    with pytest.raises(pt.PtraceError) as ei:
        pt.set_clover(op, 1.0)
    assert ei.value.code == pt.PT_ERR_ARG
    lap = pt.laplacian(ctx, [4, 4, 4, 4], 0.1)
    with pytest.raises(pt.PtraceError):
        pt.set_clover(lap, 1.0)
    dims, mu = [4, 4, 4, 4], 2
    U = _links(dims, 6)
    opc = pt.wilson(ctx, dims, _t(U), 0.12, True)
    pt.set_clover(opc, 1.0)
    col, m = greedy_colour(dims, mu, [1], 1, 0)
    with pytest.raises(pt.PtraceError) as ei:
        pt.grad(opc, _t(col), m, mu, 1, "z4", 3, 0, 1, True, "mixed_fp32", 1e-10, 2000)
    assert ei.value.code == pt.PT_ERR_ARG
    est, _, _, st = pt.trace(opc, _t(col), m, mu, [0, 1], "z4", 3, 0, 1, True, "mixed_fp32", 1e-10, 5000)
    want = OE.probed_estimates(CL.WilsonClover(dims, U, 0.12, 1.0), col, m, 3, 1, 1, mu, [0, 1], 1e-12)
    assert np.allclose(est, want, rtol=1e-8, atol=1e-7)
