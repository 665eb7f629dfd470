"""GPU parity for the tile policy, tiled colouring and the clearance
statistic (Sec. 3.5; Thm 3.6; Sec. 4.3, Tables 2, 4 and 5) against the
oracle: integer results, compared bit for bit."""
import numpy as np
import pytest

from conftest import read_golden
from oracle.clearance import clearance as o_clearance
from oracle.colouring import first_fit_violations, greedy_colour, tile_replicate
from oracle.tiles import tile_dims as o_tile_dims

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


# offsets that wrap the torus several times and merge (sides below the stencil's reach)
WRAP_CASES = [([4, 4, 4, 4], 2, [3], 4, 1), ([3, 3, 3, 3], 0, [2], 3, 0), ([2, 3, 5, 7], 3, [4], 2, 1),
              ([1, 1, 6, 1], 2, [1], 2, 0), ([2, 2, 2, 2], 1, [0], 1, 0)]


@pytest.mark.parametrize("dims,mu,p,k,order", WRAP_CASES)
def test_colouring_with_wrapping_offsets(pt, ctx, dims, mu, p, k, order):
    want, m_want = greedy_colour(dims, mu, p, k, order)
    col, m = pt.colour(ctx, dims, mu, p, k, order)
    assert m == m_want
    assert np.array_equal(col.cpu().numpy(), want)


# lattices whose colours do not fit in shared memory: the extended-array walk
# (signed halos; sides shorter than the stencil's reach; several displacements)
EXT_CASES = [([30, 20, 18, 12], 1, [3], 2, 1), ([4, 4, 64, 128], 3, [2], 3, 0), ([24, 24, 24, 12], 2, [1, 4], 1, 1),
             ([16, 16, 32, 16], 2, [5], 3, 0), ([16, 16, 32, 16], 2, [7], 7, 1)]


@pytest.mark.parametrize("dims,mu,p,k,order", EXT_CASES)
def test_colouring_large_lattices(pt, ctx, dims, mu, p, k, order):
    want, m_want = greedy_colour(dims, mu, p, k, order)
    col, m = pt.colour(ctx, dims, mu, p, k, order)
    assert m == m_want
    assert np.array_equal(col.cpu().numpy(), want)


@pytest.mark.parametrize("dims,mu,p,k,order", [([16, 16, 16, 32], 2, [2], 2, 1), ([24, 24, 24, 48], 2, [4], 2, 0),
                                               ([12, 12, 24, 12], 2, [1, 2], 1, 1)])
def test_colour_tiled_matches_oracle(pt, ctx, dims, mu, p, k, order):
    tile = o_tile_dims(dims, mu, p, k)
    tcol, m_want = greedy_colour(tile, mu, p, k, order)
    want = tile_replicate(tcol, tile, dims)
    col, m, got_tile = pt.colour_tiled(ctx, dims, mu, p, k, order)
    assert got_tile == tile and m == m_want
    assert np.array_equal(col.cpu().numpy(), want)
    assert pt.conflicts(ctx, dims, mu, p, k, col) == 0          # the repeated tile is valid on the lattice


def test_tile_replicate_ragged(pt, ctx):
    rng = np.random.default_rng(3)
    tile, dims = [3, 2, 5, 4], [6, 4, 10, 8]
    tcol = rng.integers(0, 50, size=int(np.prod(tile))).astype(np.int32)
    got = pt.tile_replicate(ctx, tile, _t(tcol), dims).cpu().numpy()
    assert np.array_equal(got, tile_replicate(tcol, tile, dims))
    with pytest.raises(pt.PtraceError):
        pt.tile_replicate(ctx, [4, 2, 5, 4], _t(tcol), dims)        # 4 does not divide 6


CLEAR_CASES = [([5, 4, 3, 6], 3, [0, 1, 2], [1, 2, 3], "random"), ([4, 7, 3, 3], 1, [0, 3], [0, 1, 2, 4], "random"),
               ([8, 8, 16, 8], 2, list(range(6)), list(range(1, 7)), (2, 3)),
               ([16, 16, 32, 16], 2, [0, 2, 4, 8], [1, 2, 5, 9], (4, 2)),
               ([9, 10, 11, 12], 0, [0, 1, 5], [1, 3, 6], "random")]


@pytest.mark.parametrize("dims,mu,ps,ks,kind", CLEAR_CASES)
def test_clearance_bit_exact(pt, ctx, dims, mu, ps, ks, kind):
    if kind == "random":
        col = np.random.default_rng(11).integers(0, 4, size=int(np.prod(dims))).astype(np.int32)
    else:
        col, _ = greedy_colour(dims, mu, [kind[0]], kind[1], 1)
    m_want, s_want = o_clearance(col, dims, mu, ps, ks)
    m, s = pt.clearance(ctx, dims, mu, _t(col), ps, ks)
    assert np.array_equal(s, s_want)
    assert np.array_equal(m, m_want)


def _half_up(x):
    return np.floor(x * 100.0 + 0.5) / 100.0


def test_table5_on_the_32cube_x_64_lattice(pt, ctx):
    """Sec. 4.3 at the paper's size: the (8, 10) red-black colouring of the
    32^4 tile (Table 2), repeated over the 32^3 x 64 lattice (2,097,152
    nodes), reproduces every entry of Table 5.  The colouring itself is
    checked on a sample of tile sites against the greedy definition."""
    dims = [32, 32, 32, 64]
    col, m, tile = pt.colour_tiled(ctx, dims, 2, [8], 10, "redblack")
    assert tile == [32, 32, 32, 32]
    tcol = col.view(2, -1)[0].cpu().numpy()                        # the tile: first half of the lattice in t
    sites = np.random.default_rng(5).choice(tcol.size, 1500, replace=False)
    assert first_fit_violations(tcol, tile, 2, [8], 10, 1, sites) == []
    assert pt.conflicts(ctx, dims, 2, [8], 10, col) == 0
    want = {int(r[0]): [float(v) for v in r[1:]] for r in read_golden("table5_clearance.txt")}
    ps, ks = list(range(9)), list(range(1, 13))
    matches, size = pt.clearance(ctx, dims, 2, col, ps, ks)
    N = int(np.prod(dims))
    pct = _half_up(100.0 * matches / (N * size))
    for j, k in enumerate(ks):
        assert np.allclose(pct[:, j], want[k], atol=1e-9), (k, pct[:, j], want[k])


NESTED_CASES = [([16, 16, 16, 16], 3, [2], 0), ([16, 16, 16, 16], 3, [4], 1), ([6, 5, 8, 4], 2, [1], 1),
                ([24, 24, 24, 12], 2, [1], 0)]          # the last: colours beyond shared memory


@pytest.mark.parametrize("dims,mu,p,order", NESTED_CASES)
def test_nested_colouring_bit_exact(pt, ctx, dims, mu, p, order):
    """Colourings grown k = 1 -> 2 -> 3 (-> 4 on 16^4, the lap16 lattice):
    every level bit-exact against the oracle, valid, and nested."""
    from oracle.colouring import nested_colour
    kmax = 4 if dims == [16, 16, 16, 16] else 3
    prev, m_prev = pt.colour(ctx, dims, mu, p, 1, order)
    want_prev, _ = greedy_colour(dims, mu, p, 1, order)
    assert np.array_equal(prev.cpu().numpy(), want_prev)
    for k in range(2, kmax + 1):
        want, m_want = nested_colour(dims, mu, p, k, want_prev, order)
        col, m = pt.colour_nested(ctx, dims, mu, p, k, prev, m_prev, order)
        assert m == m_want
        assert np.array_equal(col.cpu().numpy(), want)
        assert pt.conflicts(ctx, dims, mu, p, k, col) == 0
        prev, m_prev, want_prev = col, m, want


def test_nested_rejects_parent_out_of_range(pt, ctx):
    import torch
    dims = [4, 4, 8, 4]
    parent = torch.full((512,), 3, dtype=torch.int32, device="cuda")
    with pytest.raises(pt.PtraceError):
        pt.colour_nested(ctx, dims, 2, [1], 2, parent, 2)       # parent colour 3 >= n_parent 2
    col, m = pt.colour_nested(ctx, dims, 2, [1], 2, parent, 4)   # and the context is still usable
    want, mw = greedy_colour(dims, 2, [1], 2, 0)
    assert m == mw and np.array_equal(col.cpu().numpy(), want)


def test_nested_trace_matches_independent_levels(pt, ctx):
    """Solving only the finest of nested colourings k = 1, 2, 3 gives, at every
    level, the estimate the oracle gets by solving that level's own probes."""
    import torch
    import oracle.estimator as OE
    from oracle.colouring import nested_colour
    dims, m2, mu, ps = [8, 8, 8, 8], 0.05, 3, [0, 1, 2]
    c1, m1 = greedy_colour(dims, mu, [2], 1, 0)
    c2, m2_ = nested_colour(dims, mu, [2], 2, c1, 0)
    c3, m3 = nested_colour(dims, mu, [2], 3, c2, 0)
    cols = torch.as_tensor(np.stack([c1, c2, c3])).cuda().contiguous()
    op = pt.laplacian(ctx, dims, m2)
    est, st = pt.trace_nested(op, cols, [m1, m2_, m3], mu, ps, "z2", 21, 0, 2, True, "mixed_fp32", 1e-10, 5000)
    assert st["n_rhs"] == 2 * m3
    lap = OE.Laplacian(dims, m2)
    for l, (c, m) in enumerate([(c1, m1), (c2, m2_), (c3, m3)]):
        want = OE.probed_estimates(lap, c, m, 21, 2, 0, mu, ps, 1e-12)
        assert np.allclose(est[l], want, rtol=1e-8, atol=1e-8), l
    # colourings that are not nested are refused
    bad = torch.as_tensor(np.stack([c2, c1])).cuda().contiguous()
    with pytest.raises(pt.PtraceError):
        pt.trace_nested(op, bad, [m2_, m1], mu, ps, "z2", 21, 0, 1, True, "mixed_fp32", 1e-10, 5000)


def test_nested_trace_wilson_diluted(pt, ctx):
    import torch
    import oracle.estimator as OE
    from oracle.colouring import nested_colour
    from paper_2106_01275_gb300 import inputs
    dims, kappa, mu = [4, 4, 8, 4], 0.12, 2
    U = inputs.gauge_links(dims, 5)
    c1, m1 = greedy_colour(dims, mu, [1], 1, 1)
    c2, m2 = nested_colour(dims, mu, [1], 2, c1, 1)
    cols = torch.as_tensor(np.stack([c1, c2])).cuda().contiguous()
    op = pt.wilson(ctx, dims, torch.as_tensor(U).cuda(), kappa, True)
    est, st = pt.trace_nested(op, cols, [m1, m2], mu, [0, 1], "z4", 3, 0, 1, True, "mixed_fp32", 1e-10, 5000)
    assert st["n_rhs"] == 12 * m2
    W = OE.Wilson(dims, U, kappa)
    for l, (c, m) in enumerate([(c1, m1), (c2, m2)]):
        want = OE.probed_estimates(W, c, m, 3, 1, 1, mu, [0, 1], 1e-12)
        assert np.allclose(est[l], want, rtol=1e-8, atol=1e-7), l


def test_colour_store_matches_tiled_colouring(pt, ctx, tmp_path):
    """The tile store (Sec. 3.5): a miss colours the tile on the GPU and stores
    it, a hit reads it back; both equal pt_colour_tiled bit for bit."""
    from paper_2106_01275_gb300 import colour_db
    db = colour_db.ColourDB(tmp_path)
    dims, mu, ps, k = [8, 8, 16, 8], 2, [3], 2
    want, m_want, tile = pt.colour_tiled(ctx, dims, mu, ps, k, "natural")
    col, m, tile1, hit = db.colour(ctx, dims, mu, ps, k, "natural")
    assert not hit and tile1 == tile and m == m_want
    assert np.array_equal(col.cpu().numpy(), want.cpu().numpy())
    col2, m2, _, hit2 = db.colour(ctx, dims, mu, [-3], k, "natural")
    assert hit2 and m2 == m and np.array_equal(col2.cpu().numpy(), want.cpu().numpy())
    stored, m3 = db.get(tile, mu, ps, k, "natural")
    o_col, o_m = greedy_colour(tile, mu, ps, k, 0)
    assert m3 == o_m and np.array_equal(stored, o_col)
