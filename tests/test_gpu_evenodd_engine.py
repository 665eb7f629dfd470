"""GPU parity for the batched engine on the even Schur complement of the
Laplacian (tuning knob evenodd = 1, the default when every side is even):
traces (Eqs. (1), (5)) against the oracle at 1e-8 and against the same
engine on the full system, in FP64, FP32 and BF16 inner storage, on lattices
that take the four-entry kernels (D_0 a multiple of 8) and the one-entry
ones; solves checked through the oracle's operator; nested and 32-output
contractions; the iteration count against the full system."""
import numpy as np
import pytest

import oracle.estimator as OE
import oracle.operators as OO
from oracle.colouring import greedy_colour, nested_colour

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


PRECS = ("fp64", "mixed_fp32", "mixed_bf16")


@pytest.mark.parametrize("dims", [
    [8, 8, 8, 8],          # four entries per thread
    [16, 2, 2, 2],         # four entries per thread; sides of 2 (both neighbours one site)
    [8, 4, 6, 2],          # four entries per thread, ragged volume
    [6, 4, 2, 8],          # one entry per thread (D_0 / 2 odd)
    [4, 4, 4, 6],          # one entry per thread (D_0 not a multiple of 8)
    [2, 2, 2, 2],
])
def test_trace_matches_oracle_and_full_system(pt, ctx, dims):
    mu, m2 = 3, 0.1
    ps = [0, 1, 2]
    col, m = greedy_colour(dims, mu, [1], 1, 0)
    op = pt.laplacian(ctx, dims, m2)
    want = OE.probed_estimates(OE.Laplacian(dims, m2), col, m, 21, 2, 0, mu, ps, 1e-13)
    for prec in PRECS:
        assert pt.get_tuning(op, prec)["evenodd"] == 1
        est, _, _, st = pt.trace(op, _t(col), m, mu, ps, "z2", 21, 0, 2, True, prec, 1e-10, 5000)
        assert np.allclose(est, want, rtol=1e-8, atol=1e-9 * np.abs(want).max()), prec
        assert st["max_relres"] <= 1e-10 and st["n_noconv"] == 0
        pt.set_tuning(op, prec, evenodd=0)
        full, _, _, st_f = pt.trace(op, _t(col), m, mu, ps, "z2", 21, 0, 2, True, prec, 1e-10, 5000)
        pt.set_tuning(op, prec, reset=True)
        assert np.allclose(est, full, rtol=1e-8, atol=1e-9 * np.abs(want).max()), prec


def test_iterations_halve_on_16to4(pt, ctx):
    """16^4, m^2 = 0.01, the (4, 1) colouring along dim 3, one Z2 set: the
    even-odd engine reaches the same estimates (oracle, 1e-8) in about half
    the inner CG iterations of the full system."""
    dims, m2, mu = [16, 16, 16, 16], 0.01, 3
    col, m = greedy_colour(dims, mu, [4], 1, 0)
    op = pt.laplacian(ctx, dims, m2)
    want = OE.probed_estimates(OE.Laplacian(dims, m2), col, m, 1000, 1, 0, mu, [0, 4], 1e-12)
    est, _, _, st = pt.trace(op, _t(col), m, mu, [0, 4], "z2", 1000, 0, 1, True, "mixed_fp32", 1e-10, 20000)
    assert np.allclose(est, want, rtol=1e-8, atol=1e-8)
    pt.set_tuning(op, "mixed_fp32", evenodd=0)
    _, _, _, st_f = pt.trace(op, _t(col), m, mu, [0, 4], "z2", 1000, 0, 1, True, "mixed_fp32", 1e-10, 20000)
    pt.set_tuning(op, "mixed_fp32", reset=True)
    assert st["inner_iters"] <= 0.65 * st_f["inner_iters"], (st["inner_iters"], st_f["inner_iters"])


@pytest.mark.parametrize("dims", [[8, 4, 4, 8], [6, 2, 4, 4]])
def test_solve_through_the_oracle_operator(pt, ctx, dims):
    """pt_solve with the even-odd engine: the full solution (odd half rebuilt)
    has a true FP64 residual below the tolerance, and equals the full-system
    engine's solution."""
    import torch
    N, m2 = int(np.prod(dims)), 0.05
    op = pt.laplacian(ctx, dims, m2)
    B = np.random.default_rng(3).standard_normal((3, N))
    for prec in PRECS:
        X, iters, relres, _ = pt.solve(op, _t(B), prec, 1e-10, 5000)
        Xn = X.cpu().numpy()
        for j in range(3):
            r = B[j] - OO.laplacian_apply(Xn[j], dims, m2)
            assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(B[j]), prec
            assert relres[j] <= 1e-10
        pt.set_tuning(op, prec, evenodd=0)
        Xf, _, _, _ = pt.solve(op, _t(B), prec, 1e-10, 5000)
        pt.set_tuning(op, prec, reset=True)
        assert torch.allclose(X, Xf, rtol=1e-8, atol=1e-9 * Xf.abs().max().item()), prec
    Z, it0, _, _ = pt.solve(op, _t(np.zeros((1, N))), "mixed_fp32", 1e-10, 100)
    assert torch.count_nonzero(Z).item() == 0 and it0[0] == 0


def test_many_displacements_and_nested_levels(pt, ctx):
    """20 displacements (the 32-output contraction) and a nested colouring
    (every level's estimate from the finest level's solves), even-odd against
    the oracle."""
    import torch
    dims, m2, mu = [8, 8, 4, 4], 0.2, 0
    col, m = greedy_colour(dims, mu, [1], 1, 0)
    ps = list(range(-10, 10))
    op = pt.laplacian(ctx, dims, m2)
    est, _, _, _ = pt.trace(op, _t(col), m, mu, ps, "z2", 5, 0, 2, True, "mixed_fp32", 1e-11, 5000)
    want = OE.probed_estimates(OE.Laplacian(dims, m2), col, m, 5, 2, 0, mu, ps, 1e-13)
    assert np.allclose(est, want, rtol=1e-8, atol=1e-9 * np.abs(want).max())
    c1, m1 = greedy_colour(dims, mu, [1], 1, 0)
    c2, m2n = nested_colour(dims, mu, [1], 2, c1, 0)
    cols = torch.as_tensor(np.stack([c1, c2]).astype(np.int32)).cuda().contiguous()
    est_n, _ = pt.trace_nested(op, cols, [m1, m2n], mu, [0, 1], "z2", 9, 0, 2, True, "mixed_fp32", 1e-11, 5000)
    lap = OE.Laplacian(dims, m2)
    for lev, (c, mm) in enumerate([(c1, m1), (c2, m2n)]):
        w = OE.probed_estimates(lap, c, mm, 9, 2, 0, mu, [0, 1], 1e-13)
        assert np.allclose(est_n[lev], w, rtol=1e-8, atol=1e-9 * np.abs(w).max()), lev


def test_autotuner_chooses_between_full_and_evenodd(pt, ctx):
    dims, m2, p = [8, 8, 8, 8], 0.05, 1
    col, m = greedy_colour(dims, 0, [p], 2, 0)
    op = pt.laplacian(ctx, dims, m2)
    best = pt.autotune(op, _t(col), m, 0, "z2", 3, "mixed_fp32", 1e-10, 5000, 16)
    assert best["evenodd"] in (0, 1) and pt.get_tuning(op, "mixed_fp32")["evenodd"] == best["evenodd"]
    est, _, _, _ = pt.trace(op, _t(col), m, 0, [p], "z2", 3, 0, 2, True, "mixed_fp32", 1e-10, 5000)
    want = OE.probed_estimates(OE.Laplacian(dims, m2), col, m, 3, 2, 0, 0, [p], 1e-12)
    assert np.allclose(est, want, rtol=1e-8, atol=1e-9)
    pt.set_tuning(op, "mixed_fp32", reset=True)
    odd = pt.laplacian(ctx, [5, 4, 4, 4], m2)
    assert pt.get_tuning(odd, "mixed_fp32")["evenodd"] == 0          # an odd side: full system


# ------------------------------------------------------------------ Wilson
@pytest.mark.parametrize("dims,antip", [([4, 4, 4, 8], True), ([2, 4, 6, 4], False), ([6, 2, 2, 4], True)])
def test_wilson_trace_matches_oracle_and_full_system(pt, ctx, dims, antip):
    """Wilson-Dirac even-odd BiCGStab (S = 1 - kappa^2 D_eo D_oe) against the
    oracle and against the same engine on the full system, Z4 noise with
    12-fold dilution, in every precision."""
    from paper_2106_01275_gb300 import inputs
    kappa, mu = 0.12, 2
    U = inputs.gauge_links(dims, 1234)
    col, m = greedy_colour(dims, mu, [1], 1, 0)
    op = pt.wilson(ctx, dims, _t(U), kappa, antip)
    want = OE.probed_estimates(OE.Wilson(dims, U, kappa, antip), col, m, 1000, 2, 1, mu, [0, 1, 2], 1e-12)
    for prec in PRECS:
        assert pt.get_tuning(op, prec)["evenodd"] == 1
        est, _, _, st = pt.trace(op, _t(col), m, mu, [0, 1, 2], "z4", 1000, 0, 2, True, prec, 1e-10, 5000)
        assert np.allclose(est, want, rtol=1e-8, atol=1e-7), prec
        assert st["max_relres"] <= 1e-10 and st["n_noconv"] == 0
        pt.set_tuning(op, prec, evenodd=0)
        full, _, _, st_f = pt.trace(op, _t(col), m, mu, [0, 1, 2], "z4", 1000, 0, 2, True, prec, 1e-10, 5000)
        pt.set_tuning(op, prec, reset=True)
        assert np.allclose(est, full, rtol=1e-8, atol=1e-7), prec
        assert st["inner_iters"] < st_f["inner_iters"], (prec, st["inner_iters"], st_f["inner_iters"])


def test_wilson_undiluted_many_displacements_and_solve(pt, ctx):
    """Undiluted Z4 probes, 20 displacements (the 32-output contraction), and
    pt_solve's copy-out of the rebuilt odd half checked through the oracle's
    operator."""
    import torch
    from paper_2106_01275_gb300 import inputs
    dims, kappa, mu = [4, 2, 4, 4], 0.11, 2
    U = inputs.gauge_links(dims, 3)
    col, m = greedy_colour(dims, mu, [1], 1, 1)
    op = pt.wilson(ctx, dims, _t(U), kappa, True)
    ps = list(range(-10, 10))
    est, _, _, _ = pt.trace(op, _t(col), m, mu, ps, "z4", 5, 0, 2, False, "mixed_fp32", 1e-10, 5000)
    want = OE.probed_estimates(OE.Wilson(dims, U, kappa), col, m, 5, 2, 1, mu, ps, 1e-12, dilute=False)
    assert np.allclose(est, want, rtol=1e-8, atol=1e-7)
    N = int(np.prod(dims))
    B = np.random.default_rng(4).standard_normal((3, N, 4, 3, 2))
    for prec in PRECS:
        X, _, relres, _ = pt.solve(op, _t(B), prec, 1e-10, 5000)
        Xc = X.cpu().numpy()
        for j in range(3):
            b = B[j][..., 0] + 1j * B[j][..., 1]
            x = Xc[j][..., 0] + 1j * Xc[j][..., 1]
            r = b - OO.wilson_apply(x, U, kappa, dims, True)
            assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(b), prec
            assert relres[j] <= 1e-10
    Z, it0, _, _ = pt.solve(op, _t(np.zeros((1, N, 4, 3, 2))), "mixed_fp32", 1e-10, 100)
    assert torch.count_nonzero(Z).item() == 0 and it0[0] == 0


# ------------------------------------------------------------------ work-item shape
@pytest.mark.parametrize("cta,spt", [(64, 4), (128, 16), (256, 4), (64, 16)])
def test_item_shapes_laplacian(pt, ctx, cta, spt):
    """Every work-item shape the autotuner may pick (CTA threads x sites per
    thread) covers every site exactly once: traces against the oracle on a
    four-entry lattice and a one-entry one, even-odd and full system."""
    for dims in ([8, 8, 4, 6], [6, 4, 2, 4]):
        mu, m2 = 2, 0.2
        col, m = greedy_colour(dims, mu, [1], 1, 0)
        op = pt.laplacian(ctx, dims, m2)
        want = OE.probed_estimates(OE.Laplacian(dims, m2), col, m, 4, 2, 0, mu, [0, 1], 1e-13)
        for eo in (1, 0):
            pt.set_tuning(op, "mixed_fp32", evenodd=eo, cta_threads=cta, sites_per_thread=spt)
            t = pt.get_tuning(op, "mixed_fp32")
            assert (t["cta_threads"], t["sites_per_thread"]) == (cta, spt)
            est, _, _, st = pt.trace(op, _t(col), m, mu, [0, 1], "z2", 4, 0, 2, True, "mixed_fp32", 1e-10, 5000)
            assert np.allclose(est, want, rtol=1e-8, atol=1e-9 * np.abs(want).max()), (dims, eo)
        pt.set_tuning(op, "mixed_fp32", reset=True)


@pytest.mark.parametrize("cta", [64, 128])
def test_item_shapes_wilson(pt, ctx, cta):
    from paper_2106_01275_gb300 import inputs
    dims, kappa, mu = [4, 4, 2, 6], 0.12, 2
    U = inputs.gauge_links(dims, 55)
    col, m = greedy_colour(dims, mu, [1], 1, 0)
    op = pt.wilson(ctx, dims, _t(U), kappa, True)
    want = OE.probed_estimates(OE.Wilson(dims, U, kappa), col, m, 8, 1, 1, mu, [0, 1], 1e-12)
    for eo in (1, 0):
        pt.set_tuning(op, "mixed_fp32", evenodd=eo, cta_threads=cta)
        est, _, _, _ = pt.trace(op, _t(col), m, mu, [0, 1], "z4", 8, 0, 1, True, "mixed_fp32", 1e-10, 5000)
        assert np.allclose(est, want, rtol=1e-8, atol=1e-7), eo
    pt.set_tuning(op, "mixed_fp32", reset=True)
    with pytest.raises(pt.PtraceError):
        pt.set_tuning(op, "mixed_fp32", cta_threads=512)


@pytest.mark.parametrize("dims", [[4, 4, 2, 6], [6, 2, 4, 8], [8, 8, 8, 8]])
def test_wilson_link_sharing_groups(pt, ctx, dims):
    """rhs_block = 8 in even-odd mode: eight slots per work item, one warp
    each, the links of every 32 sites staged once in shared memory.  Traces
    against the oracle in every precision on lattices whose half volume is
    not a multiple of the 256-entry block, with work lists that are not a
    multiple of eight; solves of three sources (one group with five idle
    warps) against the ungrouped engine."""
    import torch
    from paper_2106_01275_gb300 import inputs
    kappa, mu = 0.12, 2
    U = inputs.gauge_links(dims, 99)
    col, m = greedy_colour(dims, mu, [1], 1, 0)
    op = pt.wilson(ctx, dims, _t(U), kappa, True)
    want = OE.probed_estimates(OE.Wilson(dims, U, kappa), col, m, 7, 1, 1, mu, [0, 1], 1e-12)
    for prec in PRECS:
        pt.set_tuning(op, prec, evenodd=1, rhs_block=8, cta_threads=256)
        assert pt.get_tuning(op, prec)["rhs_block"] == 8
        est, _, _, st = pt.trace(op, _t(col), m, mu, [0, 1], "z4", 7, 0, 1, True, prec, 1e-10, 5000)
        assert np.allclose(est, want, rtol=1e-8, atol=1e-7), prec
        assert st["max_relres"] <= 1e-10
    N = int(np.prod(dims))
    B = torch.as_tensor(np.random.default_rng(5).standard_normal((3, N, 4, 3, 2))).cuda().contiguous()
    X8, _, r8, _ = pt.solve(op, B, "mixed_fp32", 1e-10, 5000)
    pt.set_tuning(op, "mixed_fp32", rhs_block=1)
    X1, _, r1, _ = pt.solve(op, B, "mixed_fp32", 1e-10, 5000)
    for prec in PRECS:
        pt.set_tuning(op, prec, reset=True)
    assert max(r8) <= 1e-10 and max(r1) <= 1e-10
    assert torch.allclose(X8, X1, rtol=1e-8, atol=1e-9 * X1.abs().max().item())
