"""The solver engine's failure reports, reached without faulting the GPU:
a NaN placed on the host in a right-hand side or in the gauge links must come
back as PT_ERR_NUMERIC, and a host-set cap on graph launches as
PT_ERR_TIMEOUT; the context keeps working afterwards."""
import numpy as np
import pytest

import oracle.operators as OO
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


def _t(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("evenodd", [1, 0])
@pytest.mark.parametrize("prec", ["fp64", "mixed_fp32", "mixed_bf16"])
def test_nan_in_rhs_is_numeric_error(pt, ctx, prec, evenodd):
    dims, m2 = [8, 4, 4, 6], 0.1
    N = int(np.prod(dims))
    op = pt.laplacian(ctx, dims, m2)
    pt.set_tuning(op, prec, evenodd=evenodd)
    B = np.random.default_rng(1).standard_normal((3, N))
    B[1, 17] = np.nan                                  # one entry of the middle right-hand side
    with pytest.raises(pt.PtraceError) as ei:
        pt.solve(op, _t(B), prec, 1e-10, 5000)
    assert ei.value.code == pt.PT_ERR_NUMERIC
    B[1, 17] = 0.0                                     # the same context solves the repaired sources
    X, _, relres, _ = pt.solve(op, _t(B), prec, 1e-10, 5000)
    pt.set_tuning(op, prec, reset=True)
    Xn = X.cpu().numpy()
    for j in range(3):
        r = B[j] - OO.laplacian_apply(Xn[j], dims, m2)
        assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(B[j]) and relres[j] <= 1e-10


def test_nan_in_links_is_numeric_error(pt, ctx):
    import torch
    dims, kappa, mu = [4, 4, 4, 4], 0.12, 2
    U = inputs.gauge_links(dims, 3)
    U[37, 1, 0, 2] = complex(np.nan, 0.0)
    op = pt.wilson(ctx, dims, _t(U), kappa, True)
    col = _t(np.zeros(int(np.prod(dims)), np.int32))
    with pytest.raises(pt.PtraceError) as ei:
        pt.trace(op, col, 1, mu, [1], "z4", 5, 0, 1, True, "mixed_fp32", 1e-10, 2000)
    assert ei.value.code == pt.PT_ERR_NUMERIC
    good = pt.wilson(ctx, dims, _t(inputs.gauge_links(dims, 3)), kappa, True)
    est, _, _, st = pt.trace(good, col, 1, mu, [1], "z4", 5, 0, 1, True, "mixed_fp32", 1e-10, 2000)
    assert np.all(np.isfinite(est)) and st["max_relres"] <= 1e-10
    torch.cuda.synchronize()


def test_launch_limit_is_timeout(pt):
    """A cap of one graph launch stops a solve that needs several (the engine
    returns between launches); lifting the cap lets the same solve finish."""
    c = pt.Context(0)
    dims, m2 = [8, 8, 8, 8], 0.01
    N = int(np.prod(dims))
    op = pt.laplacian(c, dims, m2)
    pt.set_tuning(op, "mixed_fp32", graph_iters=4)
    B = _t(np.random.default_rng(2).standard_normal((2, N)))
    c.set_launch_limit(1)
    with pytest.raises(pt.PtraceError) as ei:
        pt.solve(op, B, "mixed_fp32", 1e-10, 5000)
    assert ei.value.code == pt.PT_ERR_TIMEOUT
    c.set_launch_limit(0)
    X, _, relres, st = pt.solve(op, B, "mixed_fp32", 1e-10, 5000)
    assert max(relres) <= 1e-10 and st["graph_launches"] > 1
    with pytest.raises(pt.PtraceError):
        c.set_launch_limit(-1)


def test_context_closed_before_its_operator(pt):
    """A context may be finalised before an operator made with it (a garbage
    collector frees the members of a reference cycle in no particular order):
    closing the context closes its operators first, and destroying an
    operator never reads its context."""
    import gc
    dims = [4, 4, 4, 4]
    U = _t(inputs.gauge_links(dims, 9))
    c = pt.Context(0)
    op = pt.wilson(c, dims, U, 0.12, True)
    c.close()
    assert not op._h
    op.close()
    c2 = pt.Context(0)
    holder = {"ctx": c2, "op": pt.wilson(c2, dims, U, 0.12, True), "lap": pt.laplacian(c2, dims, 0.1)}
    holder["self"] = holder                               # a cycle: only the collector frees it
    del c2, holder
    gc.collect()
    c3 = pt.Context(0)                                    # the library still works
    op3 = pt.wilson(c3, dims, U, 0.12, True)
    col = _t(np.zeros(256, np.int32))
    est, _, _, st = pt.trace(op3, col, 1, 2, [1], "z4", 5, 0, 1, True, "mixed_fp32", 1e-10, 2000)
    assert np.all(np.isfinite(est)) and st["max_relres"] <= 1e-10
