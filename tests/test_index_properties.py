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
