"""Property tests over random lattice shapes for the index arithmetic that the
new device kernels share with their host twins: the even-odd half-field
layout against the oracle's split and neighbour tables, and the multigrid
blocks through one two-grid cycle against the oracle's.  CPU only."""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

from oracle import evenodd as EO  # noqa: E402
from oracle import multigrid as MG  # noqa: E402
from oracle import operators as ops  # noqa: E402

even = st.sampled_from([2, 4, 6, 8])


@settings(max_examples=40, deadline=None)
@given(dims=st.lists(even, min_size=4, max_size=4), parity=st.integers(0, 1))
def test_half_field_layout(ptlib, dims, parity):
    ev, od = EO.split(dims)
    mine, other = (ev, od) if parity == 0 else (od, ev)
    site, nbr = ptlib.eo_layout(dims, parity)
    assert np.array_equal(site, mine)
    fwd, bwd = ops.neighbour_tables(dims)
    for mu in range(4):
        assert np.array_equal(other[nbr[:, 2 * mu]], fwd[mu][mine])
        assert np.array_equal(other[nbr[:, 2 * mu + 1]], bwd[mu][mine])


@settings(max_examples=25, deadline=None)
@given(coarse=st.lists(st.integers(1, 3), min_size=4, max_size=4), block=st.sampled_from([1, 2]),
       seed=st.integers(0, 1000))
def test_multigrid_blocks(ptlib, coarse, block, seed):
    dims = [c * block for c in coarse]
    N, m2 = int(np.prod(dims)), 0.05
    apply_a = lambda x: np.asarray(ops.laplacian_apply(np.asarray(x).reshape(-1), dims, m2)).reshape(-1)
    M = MG.TwoGrid(apply_a, np.full(N, 8 + m2), MG.prolongator_constant(dims, block), nu=1, omega=0.8)
    r = np.random.default_rng(seed).standard_normal(N)
    want = M(r)
    got = ptlib.mg_cycle_host(dims, m2, r, block, 1, 0.8)
    assert np.abs(got - want).max() <= 1e-9 * max(1.0, np.abs(want).max())


@settings(max_examples=12, deadline=None)
@given(dims=st.lists(st.sampled_from([2, 4]), min_size=4, max_size=4), mu=st.integers(0, 3),
       ps=st.lists(st.integers(-5, 5), min_size=1, max_size=4), k=st.integers(1, 2), seed=st.integers(0, 10 ** 6))
def test_even_odd_trace(ptlib, dims, mu, ps, k, seed):
    noise = 0                                    # Z2: the Laplacian is real
    import oracle.estimator as OE
    from oracle.colouring import greedy_colour
    col, m = greedy_colour(dims, mu, [abs(p) for p in ps], k, 0)
    est, _ = ptlib.trace_eo_host(dims, 0.3, col, m, mu, ps, noise, seed, 0, 1, tol=1e-11)
    want = OE.probed_estimates(OE.Laplacian(dims, 0.3), col, m, seed, 1, noise, mu, ps, 1e-13)
    assert np.allclose(est, want, rtol=1e-8, atol=1e-9 * max(1.0, np.abs(want).max()))


@settings(max_examples=6, deadline=None)
@given(dims=st.sampled_from([[2, 2, 2, 4], [2, 2, 4, 2], [4, 2, 2, 2], [2, 4, 2, 2]]), nv=st.integers(1, 4),
       seed=st.integers(0, 1000), ap=st.booleans())
def test_wilson_coarse_stencil(ptlib, dims, nv, seed, ap):
    import oracle.estimator as OE
    from oracle import deflation as D
    from paper_2106_01275_gb300 import inputs
    from test_wmg_host import _dense_P, _dense_coarse
    U = inputs.gauge_links(dims, seed, eps=0.5)
    P, Ac = ptlib.wmg_setup_host(dims, U, 0.12, 2, nv, 5, 0.8, seed, antiperiodic_t=ap)
    Pd = _dense_P(P, dims, 2)
    A = D.dense_matrix(OE.Wilson(dims, U, 0.12, ap))
    want = Pd.conj().T @ A @ Pd
    assert np.abs(_dense_coarse(Ac, [d // 2 for d in dims]) - want).max() < 1e-12 * np.abs(want).max()
