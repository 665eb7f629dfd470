"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Integer work (colourings, probes) must be bit-exact.  Floating point:
  FP64 apply: relative 1e-13;  FP32 apply: 2e-6;  BF16 apply: 2e-2
  (the inputs are rounded to the storage type first, so the bound is the
  rounding of the output plus a few ulps of accumulation);
  trace estimates for identical seeded probes: relative 1e-8 with the GPU
  solve at residual 1e-10 (the stated target) and the oracle at 1e-12.
"""
import numpy as np
import pytest

import oracle.estimator as OE
import oracle.gradient as OG
from oracle import lattice as OL
from oracle import operators as OO
from oracle.colouring import conflicts as o_conflicts
from oracle.colouring import greedy_colour
from oracle.probes import probe as o_probe
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


def _t(a, dtype=None):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype).cuda()


# ------------------------------------------------------------------ colouring (Algorithm 1)
COLOUR_CASES = [
    ([4, 4, 4, 4], 0, [1], 1, 0), ([4, 4, 4, 4], 0, [1], 2, 1), ([8, 8, 16, 8], 2, [1], 3, 0),
    ([8, 8, 16, 8], 2, [1], 3, 1), ([5, 6, 7, 3], 2, [2], 2, 0), ([5, 6, 7, 3], 1, [1, 3], 1, 1),
    ([16, 16, 16, 16], 3, [2], 2, 0), ([4, 4, 32, 4], 2, [8], 1, 1), ([32], 0, [0], 3, 0),
    ([24, 24, 24, 12], 2, [2], 1, 0),      # > 110k sites: colours kept in global memory
]


@pytest.mark.parametrize("dims,mu,p,k,order", COLOUR_CASES)
def test_colouring_bit_exact(pt, ctx, dims, mu, p, k, order):
    d4 = list(dims) + [1] * (4 - len(dims))
    want, m_want = greedy_colour(dims, mu, p, k, order)
    col, m = pt.colour(ctx, d4, mu, p, k, order)
    got = col.cpu().numpy()
    assert m == m_want
    assert np.array_equal(got, want)
    assert pt.conflicts(ctx, d4, mu, p, k, col) == 0


def test_conflict_count_detects_invalid_colouring(pt, ctx):
    dims = [4, 4, 8, 4]
    col = np.zeros(512, dtype=np.int32)                      # one colour: invalid for k >= 1
    n = pt.conflicts(ctx, dims, 2, [1], 1, _t(col))
    assert n == o_conflicts(col, dims, 2, [1], 1) and n > 0


# ------------------------------------------------------------------ probes (Eqs. (4), (5))
@pytest.mark.parametrize("noise,dof,comp", [("z2", 1, 0), ("z4", 12, 5), ("z2", 12, 0), ("z4", 12, -1)])
def test_probes_bit_exact(pt, ctx, noise, dof, comp):
    dims = [6, 5, 7, 4]
    colv, m = greedy_colour(dims, 2, [2], 2, 0)
    col = _t(colv)
    kind = 0 if noise == "z2" else 1
    for c in (0, m - 1):
        v = pt.make_probe(ctx, col, c, noise, 1234567, 3, dof, comp).cpu().numpy().reshape(-1, dof)
        want = o_probe(colv, c, 1234567, 3, kind, dof, None if comp < 0 else comp)
        assert np.array_equal(v, want)


# ------------------------------------------------------------------ operators
def _rand_field(N, dof, seed):
    r = np.random.default_rng(seed)
    if dof == 1:
        return r.standard_normal((2, N))
    return r.standard_normal((2, N, 4, 3)) + 1j * r.standard_normal((2, N, 4, 3))


@pytest.mark.parametrize("dims", [[4, 4, 4, 4], [3, 5, 2, 7], [16, 16, 16, 16]])
@pytest.mark.parametrize("prec,rtol", [("fp64", 1e-13), ("mixed_fp32", 2e-6), ("mixed_bf16", 2e-2)])
def test_laplacian_apply(pt, ctx, dims, prec, rtol):
    import torch
    N = int(np.prod(dims))
    op = pt.laplacian(ctx, dims, 0.37)
    x = _rand_field(N, 1, 1)
    if prec == "mixed_fp32":
        x = x.astype(np.float32).astype(np.float64)
    if prec == "mixed_bf16":
        x = torch.tensor(x).to(torch.bfloat16).to(torch.float64).numpy()
    y = pt.apply(op, _t(x), prec).cpu().numpy()
    for j in range(2):
        want = OO.laplacian_apply(x[j], dims, 0.37)
        assert np.max(np.abs(y[j] - want)) <= rtol * np.max(np.abs(want))


@pytest.mark.parametrize("dims,antip", [([4, 4, 4, 4], True), ([3, 4, 5, 6], True), ([2, 3, 4, 5], False),
                                        ([8, 8, 8, 16], True)])
@pytest.mark.parametrize("prec,rtol", [("fp64", 1e-13), ("mixed_fp32", 3e-6), ("mixed_bf16", 3e-2)])
def test_wilson_apply(pt, ctx, dims, antip, prec, rtol):
    import torch
    N = int(np.prod(dims))
    U = inputs.gauge_links(dims, 77)
    psi = _rand_field(N, 12, 2)
    if prec == "mixed_fp32":
        U = U.astype(np.complex64).astype(np.complex128)
        psi = psi.astype(np.complex64).astype(np.complex128)
    if prec == "mixed_bf16":
        rb = lambda a: (torch.view_as_real(torch.tensor(a)).to(torch.bfloat16).to(torch.float64))
        U = torch.view_as_complex(rb(U).contiguous()).numpy()
        psi = torch.view_as_complex(rb(psi).contiguous()).numpy()
    op = pt.wilson(ctx, dims, _t(U), 0.124, antip)
    y = pt.apply(op, _t(psi), prec).cpu().numpy()
    for j in range(2):
        want = OO.wilson_apply(psi[j], U, 0.124, dims, antip)
        assert np.max(np.abs(y[j] - want)) <= rtol * np.max(np.abs(want))


def test_wilson_apply_full_size_24c48(pt, ctx):
    """Full-size lattice of the batched Wilson workload (24^3 x 48), FP32 and FP64."""
    dims = [24, 24, 24, 48]
    N = int(np.prod(dims))
    U = inputs.gauge_links(dims, 1234)
    r = np.random.default_rng(5)
    psi = (r.standard_normal((1, N, 4, 3)) + 1j * r.standard_normal((1, N, 4, 3)))
    op = pt.wilson(ctx, dims, _t(U), 0.124, True)
    want = OO.wilson_apply(psi[0], U, 0.124, dims, True)
    y = pt.apply(op, _t(psi), "fp64").cpu().numpy()[0]
    assert np.max(np.abs(y - want)) <= 1e-13 * np.max(np.abs(want))
    # FP32: inputs rounded on the device; bound by FP32 rounding of inputs and output
    y32 = pt.apply(op, _t(psi), "mixed_fp32").cpu().numpy()[0]
    assert np.max(np.abs(y32 - want)) <= 2e-5 * np.max(np.abs(want))


def test_wilson_solve_full_size_24c48(pt, ctx):
    """Full-size lattice of the batched Wilson workload (24^3 x 48, kappa 0.124):
    the true residual of the GPU solutions, evaluated with the oracle's FP64
    operator, is below the tolerance (a property that holds at any size)."""
    dims, kappa = [24, 24, 24, 48], 0.124
    N = int(np.prod(dims))
    U = inputs.gauge_links(dims, 1234)
    op = pt.wilson(ctx, dims, _t(U), kappa, True)
    r = np.random.default_rng(8)
    B = r.standard_normal((2, N, 4, 3)) + 1j * r.standard_normal((2, N, 4, 3))
    X, iters, relres, st = pt.solve(op, _t(B), "mixed_fp32", 1e-10, 5000)
    X = X.cpu().numpy()
    for j in range(2):
        res = B[j] - OO.wilson_apply(X[j], U, kappa, dims, True)
        assert np.linalg.norm(res) <= 1.01e-10 * np.linalg.norm(B[j])


# ------------------------------------------------------------------ solves
@pytest.mark.parametrize("prec", ["fp64", "mixed_fp32", "mixed_bf16"])
def test_laplacian_solve(pt, ctx, prec):
    dims = [4, 4, 4, 6]
    N = int(np.prod(dims))
    op = pt.laplacian(ctx, dims, 0.05)
    B = _rand_field(N, 1, 3)
    X, iters, relres, st = pt.solve(op, _t(B), prec, tol=1e-10, maxit=5000)
    X = X.cpu().numpy()
    for j in range(2):
        r = B[j] - OO.laplacian_apply(X[j], dims, 0.05)
        assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(B[j])
        assert relres[j] <= 1e-10 and iters[j] > 0


@pytest.mark.parametrize("prec", ["fp64", "mixed_fp32", "mixed_bf16"])
def test_wilson_solve(pt, ctx, prec):
    dims = [4, 4, 4, 8]
    N = int(np.prod(dims))
    U = inputs.gauge_links(dims, 1234)
    op = pt.wilson(ctx, dims, _t(U), 0.12, True)
    B = _rand_field(N, 12, 4)
    X, iters, relres, st = pt.solve(op, _t(B), prec, tol=1e-10, maxit=5000)
    X = X.cpu().numpy()
    for j in range(2):
        r = B[j] - OO.wilson_apply(X[j], U, 0.12, dims, True)
        assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(B[j])


# ------------------------------------------------------------------ traces (Eqs. (1), (5))
@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("prec", ["fp64", "mixed_fp32"])
def test_trace_4to4_laplacian(pt, ctx, k, prec):
    """4^4 shifted Laplacian, m^2 = 0.1, p = 1 along dim 0, distance-k colouring,
    Z2 probes from seed 0: per-set estimates equal the oracle's."""
    dims, m2, p = [4, 4, 4, 4], 0.1, 1
    colv, m = greedy_colour(dims, 0, [p], k, 0)
    op = pt.laplacian(ctx, dims, m2)
    est, mean, var, st = pt.trace(op, _t(colv), m, 0, [0, 1, 2], "z2", 0, 0, 4, True, prec, 1e-12, 5000)
    want = OE.probed_estimates(OE.Laplacian(dims, m2), colv, m, 0, 4, 0, 0, [0, 1, 2], 1e-13)
    assert np.allclose(est, want, rtol=1e-8, atol=1e-9)
    assert np.allclose(mean, want.mean(0), rtol=1e-8, atol=1e-9)
    assert np.allclose(var, OE.sample_variance(want), rtol=1e-6, atol=1e-9)


@pytest.mark.parametrize("dims", [[5, 4, 3, 6], [6, 2, 4, 3]])
def test_trace_ragged_laplacian(pt, ctx, dims):
    """Extents that are not multiples of 4 take the one-site kernels (the 16^4
    lattice takes the four-site kernels); both must match the oracle."""
    m2, p = 0.2, 2
    colv, m = greedy_colour(dims, 2, [p], 1, 1)
    op = pt.laplacian(ctx, dims, m2)
    for prec in ("fp64", "mixed_fp32", "mixed_bf16"):
        est, _, _, st = pt.trace(op, _t(colv), m, 2, [0, p], "z2", 9, 0, 3, True, prec, 1e-11, 5000)
        want = OE.probed_estimates(OE.Laplacian(dims, m2), colv, m, 9, 3, 0, 2, [0, p], 1e-13)
        assert np.allclose(est, want, rtol=1e-8, atol=1e-9), prec


def test_hutchinson_64_vectors_4to4(pt, ctx):
    dims, m2 = [4, 4, 4, 4], 0.1
    op = pt.laplacian(ctx, dims, m2)
    col = np.zeros(256, np.int32)
    est, mean, var, st = pt.trace(op, _t(col), 1, 0, [1], "z2", 0, 0, 64, True, "fp64", 1e-12, 5000)
    want = OE.hutchinson_estimates(OE.Laplacian(dims, m2), 0, 64, 0, 0, [1], 1e-13)
    assert np.allclose(est, want, rtol=1e-8, atol=1e-9)
    assert st["n_rhs"] == 64


@pytest.mark.parametrize("prec", ["fp64", "mixed_fp32", "mixed_bf16"])
def test_trace_wilson_small(pt, ctx, prec):
    """Wilson 4^3 x 8, kappa 0.12, antiperiodic t, displacements along z,
    distance-1 colouring for p = 1, Z4 noise, full spin-colour dilution."""
    dims, kappa, mu = [4, 4, 4, 8], 0.12, 2
    U = inputs.gauge_links(dims, 1234)
    colv, m = greedy_colour(dims, mu, [1], 1, 0)
    op = pt.wilson(ctx, dims, _t(U), kappa, True)
    est, mean, var, st = pt.trace(op, _t(colv), m, mu, [0, 1, 2], "z4", 1000, 0, 2, True, prec, 1e-10, 5000)
    want = OE.probed_estimates(OE.Wilson(dims, U, kappa), colv, m, 1000, 2, 1, mu, [0, 1, 2], 1e-12)
    assert np.allclose(est, want, rtol=1e-8, atol=1e-7)
    assert st["n_rhs"] == 2 * m * 12 and st["max_relres"] <= 1e-10


def test_trace_wilson_undiluted(pt, ctx):
    dims, kappa, mu = [2, 4, 4, 4], 0.11, 2
    U = inputs.gauge_links(dims, 3)
    colv, m = greedy_colour(dims, mu, [1], 1, 1)
    op = pt.wilson(ctx, dims, _t(U), kappa, True)
    est, _, _, st = pt.trace(op, _t(colv), m, mu, [1], "z4", 5, 0, 2, False, "mixed_fp32", 1e-10, 5000)
    want = OE.probed_estimates(OE.Wilson(dims, U, kappa), colv, m, 5, 2, 1, mu, [1], 1e-12, dilute=False)
    assert np.allclose(est, want, rtol=1e-8, atol=1e-7)


def test_trace_16to4_sampled(pt, ctx):
    """16^4 Laplacian, m^2 = 0.01 (the plain-baseline lattice): one noise set of
    a (p, k) = (4, 1) colouring along dim 3; every solve is checked one by one
    through its contribution to the estimate."""
    dims, m2, mu, p, k = [16, 16, 16, 16], 0.01, 3, 4, 1
    colv, m = greedy_colour(dims, mu, [p], k, 0)
    op = pt.laplacian(ctx, dims, m2)
    col = _t(colv)
    for prec in ("fp64", "mixed_fp32"):
        est, _, _, st = pt.trace(op, col, m, mu, [p], "z2", 1000, 0, 1, True, prec, 1e-10, 20000)
        want = OE.probed_estimates(OE.Laplacian(dims, m2), colv, m, 1000, 1, 0, mu, [p], 1e-12)
        assert np.allclose(est, want, rtol=1e-8, atol=1e-8), prec


# ------------------------------------------------------------------ gradient
def test_grad_m2_laplacian(pt, ctx):
    dims, m2, p = [4, 4, 4, 4], 0.1, 1
    colv, m = greedy_colour(dims, 0, [p], 2, 0)
    op = pt.laplacian(ctx, dims, m2)
    est, dm2, _, _, st = pt.grad(op, _t(colv), m, 0, p, "z2", 0, 0, 2, True, "fp64", 1e-12, 5000)
    want = OG.grad_m2(OE.Laplacian(dims, m2), colv, m, 0, 2, 0, 0, p, 1e-13)
    assert abs(dm2 - want) <= 1e-8 * abs(want)
    est_o = OE.probed_estimates(OE.Laplacian(dims, m2), colv, m, 0, 2, 0, 0, [p], 1e-13)[:, 0]
    assert np.allclose(est, est_o, rtol=1e-8)


@pytest.mark.parametrize("prec", ["fp64", "mixed_fp32"])
def test_grad_wilson_links(pt, ctx, prec):
    dims, kappa, p, mu = [2, 2, 4, 4], 0.12, 1, 2
    U = inputs.gauge_links(dims, 8)
    colv, m = greedy_colour(dims, mu, [p], 1, 0)
    op = pt.wilson(ctx, dims, _t(U), kappa, True)
    est, dk, G, Gb, st = pt.grad(op, _t(colv), m, mu, p, "z4", 3, 0, 1, True, prec, 1e-11, 5000, links=True)
    dk_o, G_o, Gb_o = OG.grad_links(OE.Wilson(dims, U, kappa), colv, m, 3, 1, 1, mu, p, 1e-12, dilute=True)
    assert abs(dk - dk_o) <= 1e-7 * abs(dk_o)
    sc = max(np.max(np.abs(G_o)), np.max(np.abs(Gb_o)))
    assert np.max(np.abs(G.cpu().numpy() - G_o)) <= 1e-7 * sc
    assert np.max(np.abs(Gb.cpu().numpy() - Gb_o)) <= 1e-7 * sc


def test_grad_kappa_finite_difference_gpu(pt, ctx):
    """dT/dkappa from the adjoint against a central difference of GPU traces
    (step 1e-5, FP64 solves)."""
    dims, kappa, p, mu = [4, 4, 4, 4], 0.12, 1, 2
    U = inputs.gauge_links(dims, 4321)
    colv, m = greedy_colour(dims, mu, [p], 1, 0)
    col = _t(colv)
    Ud = _t(U)
    op = pt.wilson(ctx, dims, Ud, kappa, True)
    _, dk, _, _, _ = pt.grad(op, col, m, mu, p, "z4", 7, 0, 1, True, "fp64", 1e-12, 5000)
    h = 1e-5
    tp = pt.trace(pt.wilson(ctx, dims, Ud, kappa + h, True), col, m, mu, [p], "z4", 7, 0, 1, True, "fp64", 1e-13, 5000)[0]
    tm = pt.trace(pt.wilson(ctx, dims, Ud, kappa - h, True), col, m, mu, [p], "z4", 7, 0, 1, True, "fp64", 1e-13, 5000)[0]
    fd = (tp[0, 0] - tm[0, 0]) / (2 * h)
    assert abs(dk - fd) <= 1e-5 * abs(fd)


def test_grad_fd_8to4_kappa_and_links(pt, ctx):
    """The finite-difference check of the adjoint at its stated size: 8^4,
    kappa = 0.12, central differences with step 1e-5 of FP64 GPU traces, for
    dT/dkappa and for the real and imaginary parts of sampled link entries."""
    import torch
    dims, kappa, p, mu = [8, 8, 8, 8], 0.12, 1, 2
    U = inputs.gauge_links(dims, 4321)
    colv, m = greedy_colour(dims, mu, [p], 1, 0)
    col = _t(colv)
    Ud = _t(U)
    op = pt.wilson(ctx, dims, Ud, kappa, True)
    _, dk, G, Gb, _ = pt.grad(op, col, m, mu, p, "z4", 17, 0, 1, False, "fp64", 1e-12, 5000, links=True)
    G, Gb = G.cpu().numpy(), Gb.cpu().numpy()
    h = 1e-5

    def T(kap, Udev):
        o = pt.wilson(ctx, dims, Udev, kap, True)
        est = pt.trace(o, col, m, mu, [p], "z4", 17, 0, 1, False, "fp64", 1e-13, 5000)[0]
        o.close()
        return est[0, 0]

    fd = (T(kappa + h, Ud) - T(kappa - h, Ud)) / (2 * h)
    assert abs(dk - fd) <= 1e-5 * abs(fd)
    r = np.random.default_rng(1)
    for _ in range(3):
        n, nu, a, b = int(r.integers(4096)), int(r.integers(4)), int(r.integers(3)), int(r.integers(3))
        for part, dz in (("re", h), ("im", 1j * h)):
            Up, Um = Ud.clone(), Ud.clone()
            Up[n, nu, a, b] += dz
            Um[n, nu, a, b] -= dz
            fdl = (T(kappa, Up) - T(kappa, Um)) / (2 * h)
            an = (G + Gb)[n, nu, a, b] if part == "re" else 1j * (G - Gb)[n, nu, a, b]
            assert abs(an - fdl) <= 1e-5 * max(abs(fdl), 1e-2 * np.max(np.abs(G))), (n, nu, a, b, part)


def test_wilson_8c16_mixed_vs_fp64_and_sampled_oracle(pt, ctx):
    """The 8^3 x 16 Wilson configuration (kappa 0.12, antiperiodic t, (p, 2)
    colourings for displacements along z, Z4 noise, 12x dilution): mixed FP32
    and BF16-storage estimates equal the FP64 ones to 1e-8 for every
    displacement p = 1..8 contracted from one solve per probe, and a sample of
    the probes solved one by one matches the oracle's BiCGStab solutions."""
    dims, kappa, mu = [8, 8, 8, 16], 0.12, 2
    U = inputs.gauge_links(dims, 1234)
    op = pt.wilson(ctx, dims, _t(U), kappa, True)
    plist = list(range(1, 9))
    for p in (1, 4):
        colv, m = greedy_colour(dims, mu, [p], 2, 1)
        col = _t(colv)
        e64 = pt.trace(op, col, m, mu, plist, "z4", 1000, 0, 1, True, "fp64", 1e-10, 5000)[0]
        for prec in ("mixed_fp32", "mixed_bf16"):
            e = pt.trace(op, col, m, mu, plist, "z4", 1000, 0, 1, True, prec, 1e-10, 5000)[0]
            assert np.allclose(e, e64, rtol=1e-8, atol=1e-6), (p, prec)
    # sampled solves against the oracle
    from oracle.estimator import Wilson
    ow = Wilson(dims, U, kappa)
    colv, m = greedy_colour(dims, mu, [4], 2, 1)
    for c, a in ((0, 0), (m - 1, 7)):
        v = o_probe(colv, c, 1000, 0, 1, 12, a)
        x_o, _, _ = ow.solve(v, 1e-12)
        X, _, rel, _ = pt.solve(op, _t(v.reshape(1, -1, 4, 3)), "mixed_fp32", 1e-10, 5000)
        x = X.cpu().numpy().reshape(-1, 12)
        assert np.linalg.norm(x - x_o) <= 1e-8 * np.linalg.norm(x_o)


# ------------------------------------------------------------------ autotuner
def test_autotune_then_parity(pt, ctx):
    """The autotuner picks parameters from its candidate sets, stores them for
    the operator, and traces with the tuned engine still match the oracle."""
    dims, m2, p = [8, 8, 8, 8], 0.05, 1
    colv, m = greedy_colour(dims, 0, [p], 2, 0)
    op = pt.laplacian(ctx, dims, m2)
    best = pt.autotune(op, _t(colv), m, 0, "z2", 3, "mixed_fp32", 1e-10, 5000, 16)
    assert best["delta"] in (1e-2, 1e-3, 1e-4, 1e-5, 1e-6) and best["graph_iters"] in (4, 8, 16)
    assert best["group"] == 1 and best["seconds_per_rhs"] > 0
    assert pt.get_tuning(op, "mixed_fp32")["delta"] == best["delta"]
    est, _, _, _ = pt.trace(op, _t(colv), m, 0, [p], "z2", 3, 0, 2, True, "mixed_fp32", 1e-10, 5000)
    want = OE.probed_estimates(OE.Laplacian(dims, m2), colv, m, 3, 2, 0, 0, [p], 1e-12)
    assert np.allclose(est, want, rtol=1e-8, atol=1e-9)
    # Wilson: the slot group is tuned too; explicit settings are honoured
    dims, kappa, mu = [4, 4, 4, 8], 0.12, 2
    U = inputs.gauge_links(dims, 1234)
    colw, mw = greedy_colour(dims, mu, [1], 1, 0)
    opw = pt.wilson(ctx, dims, _t(U), kappa, True)
    bw = pt.autotune(opw, _t(colw), mw, mu, "z4", 5, "mixed_fp32", 1e-10, 5000, 12)
    assert bw["group"] in (1, 2, 4, 8, 16)
    assert bw["rhs_block"] in (1, 2) and bw["overlap"] == 0
    pt.set_tuning(opw, "mixed_fp32", delta=1e-3, group=2, graph_iters=4, rhs_block=1, overlap=0, evenodd=1,
                  cta_threads=256)
    assert pt.get_tuning(opw, "mixed_fp32") == {"delta": 1e-3, "group": 2, "graph_iters": 4, "rhs_block": 1,
                                                "overlap": 0, "evenodd": 1, "cta_threads": 256,
                                                "sites_per_thread": 1, "seconds_per_rhs": 0.0}
    est, _, _, _ = pt.trace(opw, _t(colw), mw, mu, [1], "z4", 5, 0, 1, True, "mixed_fp32", 1e-10, 5000)
    want = OE.probed_estimates(OE.Wilson(dims, U, kappa), colw, mw, 5, 1, 1, mu, [1], 1e-12)
    assert np.allclose(est, want, rtol=1e-8, atol=1e-7)
    pt.set_tuning(opw, "mixed_fp32", reset=True)
    pt.set_tuning(op, "mixed_fp32", reset=True)


@pytest.mark.parametrize("prec,group", [("mixed_fp32", 8), ("mixed_fp32", 1), ("mixed_bf16", 4)])
def test_wilson_two_rhs_items_parity(pt, ctx, prec, group):
    """rhs_block = 2 (two right-hand sides per item, one link load for both):
    traces match the oracle, and solves of an odd number of sources (a pair
    with one member) match the one-per-item engine."""
    import torch
    dims, kappa, mu = [4, 6, 4, 8], 0.12, 2
    U = inputs.gauge_links(dims, 77)
    col, m = greedy_colour(dims, mu, [2], 1, 1)
    op = pt.wilson(ctx, dims, _t(U), kappa, True)
    pt.set_tuning(op, prec, group=group, rhs_block=2)
    assert pt.get_tuning(op, prec)["rhs_block"] == 2
    est, _, _, st = pt.trace(op, _t(col), m, mu, [0, 2], "z4", 9, 0, 2, True, prec, 1e-10, 5000)
    want = OE.probed_estimates(OE.Wilson(dims, U, kappa), col, m, 9, 2, 1, mu, [0, 2], 1e-12)
    assert np.allclose(est, want, rtol=1e-8, atol=1e-7)
    assert st["max_relres"] <= 1e-10
    N = int(np.prod(dims))
    rng = np.random.default_rng(4)
    B = torch.as_tensor(rng.standard_normal((3, N, 4, 3, 2))).cuda().contiguous()
    X2, _, r2, _ = pt.solve(op, B, prec, 1e-10, 5000)
    pt.set_tuning(op, prec, rhs_block=1)
    X1, _, r1, _ = pt.solve(op, B, prec, 1e-10, 5000)
    assert max(r1) <= 1e-10 and max(r2) <= 1e-10
    assert torch.allclose(X2, X1, rtol=1e-8, atol=1e-9 * X1.abs().max().item())
    pt.set_tuning(op, prec, reset=True)


def test_overlapped_iterations_parity(pt, ctx):
    """overlap = 1 (contraction and FP64 outer steps as graph branches beside
    the inner kernels): traces still match the oracle, Laplacian and Wilson,
    with several colourings so that the three groups are busy at once."""
    import torch
    dims, m2, mu = [8, 8, 8, 8], 0.05, 3
    cols, ms = [], []
    for p, k in [(0, 1), (1, 2), (2, 2)]:
        c, m = greedy_colour(dims, mu, [p], k, 0)
        cols.append(c)
        ms.append(m)
    op = pt.laplacian(ctx, dims, m2)
    pt.set_tuning(op, "mixed_fp32", overlap=1, graph_iters=4)
    est, st = pt.trace_multi(op, torch.as_tensor(np.stack(cols)).cuda().contiguous(), ms, mu, [0, 1, 2], "z2", 8,
                             0, 2, True, "mixed_fp32", 1e-10, 5000)
    lap = OE.Laplacian(dims, m2)
    for i in range(3):
        want = OE.probed_estimates(lap, cols[i], ms[i], 8, 2, 0, mu, [0, 1, 2], 1e-12)
        assert np.allclose(est[i], want, rtol=1e-8, atol=1e-8)
    pt.set_tuning(op, "mixed_fp32", reset=True)
    dims, kappa, mu = [4, 4, 8, 4], 0.12, 2
    U = inputs.gauge_links(dims, 31)
    c0, m0 = greedy_colour(dims, mu, [1], 1, 1)
    opw = pt.wilson(ctx, dims, _t(U), kappa, True)
    for prec in ("mixed_fp32", "fp64"):
        pt.set_tuning(opw, prec, overlap=1, graph_iters=4)
        est, _, _, st = pt.trace(opw, _t(c0), m0, mu, [0, 1], "z4", 6, 0, 1, True, prec, 1e-10, 5000)
        want = OE.probed_estimates(OE.Wilson(dims, U, kappa), c0, m0, 6, 1, 1, mu, [0, 1], 1e-12)
        assert np.allclose(est, want, rtol=1e-8, atol=1e-7)
        pt.set_tuning(opw, prec, reset=True)


@pytest.mark.parametrize("dims", [[4, 3, 8, 4], [8, 3, 5, 3], [32, 2, 2, 4], [8, 5, 4, 4], [128, 1, 2, 1]])
def test_laplacian_four_site_paths(pt, ctx, dims):
    """The four-site Laplacian kernels (D_0 a multiple of 4) on short rows,
    long rows, sides of 1 to 3 and volumes that are not a multiple of the
    block: traces in FP64, FP32 and BF16 storage against the oracle."""
    mu = 2
    col, m = greedy_colour(dims, mu, [1], 1, 0)
    op = pt.laplacian(ctx, dims, 0.3)
    want = OE.probed_estimates(OE.Laplacian(dims, 0.3), col, m, 17, 2, 0, mu, [0, 1], 1e-12)
    for prec in ("fp64", "mixed_fp32", "mixed_bf16"):
        est, _, _, st = pt.trace(op, _t(col), m, mu, [0, 1], "z2", 17, 0, 2, True, prec, 1e-10, 5000)
        assert np.allclose(est, want, rtol=1e-8, atol=1e-9), prec
        assert st["max_relres"] <= 1e-10


# ------------------------------------------------------------------ edge cases
def test_edge_cases(pt, ctx):
    import torch
    dims = [3, 1, 5, 2]                                     # ragged, a size-1 dimension
    N = 30
    op = pt.laplacian(ctx, dims, 0.5)
    # zero right-hand sides solve to zero
    B = torch.zeros((1, N), dtype=torch.float64, device="cuda")
    X, iters, relres, st = pt.solve(op, B, "mixed_fp32", 1e-10, 100)
    assert torch.count_nonzero(X).item() == 0
    # nrhs = 0
    X, _, _, st = pt.solve(op, torch.zeros((0, N), dtype=torch.float64, device="cuda"), "fp64", 1e-10, 100)
    assert X.shape == (0, N)
    # maxit too small -> PT_ERR_NOCONV, reported
    B = _t(_rand_field(N, 1, 9)[:1])
    with pytest.raises(pt.PtraceError) as ei:
        pt.solve(op, B, "fp64", 1e-14, 2)
    assert ei.value.code == pt.PT_ERR_NOCONV
    # invalid arguments
    with pytest.raises(pt.PtraceError):
        pt.solve(op, B, "fp64", 0.0, 10)
    col = _t(np.zeros(N, np.int32))
    with pytest.raises(pt.PtraceError):
        pt.trace(op, col, 1, 0, [1], "z4", 0, 0, 1)         # Z4 on a real field
    # single site lattice
    op1 = pt.laplacian(ctx, [1, 1, 1, 1], 0.5)
    est, _, _, _ = pt.trace(op1, _t(np.zeros(1, np.int32)), 1, 0, [0], "z2", 0, 0, 2, True, "fp64", 1e-12, 100)
    assert np.allclose(est, 1.0 / 0.5)
