"""Pins for the oracle's clearance statistic (Sec. 3.3, Thm 3.6; Sec. 4.3, Table 5)."""
import itertools
import multiprocessing as mp

import numpy as np
import pytest

from conftest import read_golden
from oracle import lattice as L
from oracle.clearance import clearance, clearance_percent, offset_matches, shell
from oracle.colouring import greedy_colour, tile_replicate


def _brute(col, dims, mu, p, k):
    """The statistic node by node: for each x, the set of nodes y != x whose
    distance to the nearer of x + p e_mu, x - p e_mu is k, and how many share
    x's colour.  Returns (sum over x of the count, the set size, which must be
    the same for every x)."""
    d = len(dims)
    xs = L.coords(dims)
    R = [p + k if nu == mu else k for nu in range(d)]
    box = [np.array(o) - np.array(R) for o in itertools.product(*[range(2 * r + 1) for r in R])]
    e = np.zeros(d, dtype=int)
    e[mu] = p
    total, sizes = 0, set()
    for i in range(xs.shape[0]):
        ys = set()
        for o in box:
            if min(np.abs(o - e).sum(), np.abs(o + e).sum()) == k:
                y = int(L.index_of(xs[i] + o, dims))
                if y != i:
                    ys.add(y)
        sizes.add(len(ys))
        total += sum(int(col[y] == col[i]) for y in ys)
    assert len(sizes) == 1
    return total, sizes.pop()


@pytest.mark.parametrize("dims,mu,p,k", [([5, 4, 3, 6], 3, 1, 1), ([5, 4, 3, 6], 3, 2, 2),
                                         ([4, 7, 3, 3], 1, 0, 2), ([6, 3, 4, 4], 0, 3, 1),
                                         ([3, 3, 3, 3], 2, 1, 3)])
def test_matches_node_by_node_definition(dims, mu, p, k):
    """Random colourings of ragged tori (shells that wrap onto themselves
    included): the offset-by-offset sum equals the node-by-node count."""
    rng = np.random.default_rng(7)
    col = rng.integers(0, 3, size=int(np.prod(dims))).astype(np.int32)
    m, s = clearance(col, dims, mu, [p], [k])
    bt, bs = _brute(col, dims, mu, p, k)
    assert (int(m[0, 0]), int(s[0, 0])) == (bt, bs)


def test_shell_sizes_of_p0_are_l1_spheres():
    """For p = 0 on a torus wider than 2k the shell is the 4D L1 sphere of
    radius k: sum_i 2^i C(4, i) C(k - 1, i - 1) nodes."""
    from math import comb
    for k in range(1, 8):
        want = sum(2 ** i * comb(4, i) * comb(k - 1, i - 1) for i in range(1, 5))
        assert len(shell([16, 16, 16, 16], 2, 0, k)) == want


def test_shells_partition_the_union_of_balls():
    """The shells k = 1..K around the pair are disjoint and together make the
    displaced neighbourhood N(x, p, K) minus x (Eq. (8))."""
    from oracle.stencil import displaced_stencil
    dims = [20, 20, 20, 20]
    for p, K in [(0, 3), (2, 2), (3, 4)]:
        seen = set()
        for k in range(0, K + 1):
            s = set(shell(dims, 2, p, k))
            assert not (s & seen)
            seen |= s
        st = {tuple(int(v) % D for v, D in zip(o, dims)) for o in displaced_stencil(4, 2, [p], K)}
        st.discard((0, 0, 0, 0))
        assert seen == st


def test_trivial_colourings():
    """One colour everywhere: every node is uncleared (100 %); all colours
    distinct: every node is cleared (0 %)."""
    dims = [6, 6, 6, 6]
    N = int(np.prod(dims))
    same = clearance_percent(np.zeros(N, np.int32), dims, 2, [0, 1, 2], [1, 2, 3])
    assert np.all(same == 100.0)
    diff = clearance_percent(np.arange(N, dtype=np.int32), dims, 2, [0, 1, 2], [1, 2, 3])
    assert np.all(diff == 0.0)


@pytest.mark.parametrize("p0,k0,tile", [(2, 3, [8, 8, 16, 8]), (1, 2, [8, 8, 8, 8]), (4, 2, [8, 8, 16, 8])])
def test_theorem_3_6_clearance(p0, k0, tile):
    """Thm 3.6: a (p0, k0)-colouring clears, for displacement p, every
    distance k <= k0 - |p - p0| (no node there shares x's colour)."""
    col, _ = greedy_colour(tile, 2, [p0], k0, 1)
    ps = list(range(0, p0 + k0 + 1))
    ks = list(range(1, k0 + 1))
    m, s = clearance(col, tile, 2, ps, ks)
    for i, p in enumerate(ps):
        for j, k in enumerate(ks):
            if k <= k0 - abs(p - p0):
                assert m[i, j] == 0, (p, k)
    # and the theorem is tight somewhere: the colouring is not a distance-(k0 + 1) colouring
    assert clearance(col, tile, 2, [p0], [k0 + 1])[0][0, 0] > 0


def test_tile_average_equals_lattice_average():
    """A colouring repeated from a tile gives the same statistic on the
    lattice as on the tile when no shell wraps differently (the tile holds
    the neighbourhood, Sec. 3.5): the identity used for Table 5."""
    tile, lat = [8, 8, 16, 8], [8, 8, 16, 16]
    col, _ = greedy_colour(tile, 2, [2], 2, 1)
    big = tile_replicate(col, tile, lat)
    a = clearance_percent(col, tile, 2, [0, 1, 2, 3], [1, 2, 3])
    b = clearance_percent(big, lat, 2, [0, 1, 2, 3], [1, 2, 3])
    assert np.array_equal(a, b)


def _chunk(args):
    col, dims, offs = args
    return offset_matches(col, dims, offs)


def _half_up(x):
    return np.floor(x * 100.0 + 0.5) / 100.0


@pytest.mark.slow
def test_table5_from_the_red_black_8_10_colouring():
    """Table 5: the red-black greedy (8, 10)-colouring of the 32^4 tile
    (Table 2), repeated over the 32^3 x 64 lattice, leaves exactly the
    printed percentages uncleared for p = 0..8, k = 1..12 (108 entries, two
    decimals, half up).  The tile and the lattice give the same averages
    (no shell here reaches 32 along z or t)."""
    want = {int(r[0]): [float(v) for v in r[1:]] for r in read_golden("table5_clearance.txt")}
    dims = [32, 32, 32, 32]
    col, m = greedy_colour(dims, 2, [8], 10, 1)
    ps, ks = list(range(9)), list(range(1, 13))
    shells = {(p, k): shell(dims, 2, p, k) for p in ps for k in ks}
    distinct = sorted(set(o for s in shells.values() for o in s))
    chunks = [distinct[i::16] for i in range(16)]
    with mp.get_context("spawn").Pool(min(8, mp.cpu_count())) as pool:
        parts = pool.map(_chunk, [(col, dims, c) for c in chunks])
    counts = {}
    for c, r in zip(chunks, parts):
        counts.update(zip(c, r.tolist()))
    N = int(np.prod(dims))
    for k in ks:
        got = [_half_up(100.0 * sum(counts[o] for o in shells[(p, k)]) / (N * len(shells[(p, k)]))) for p in ps]
        assert np.allclose(got, want[k], atol=1e-9), (k, got, want[k])
    # the same colouring through the plain entry point, on a few entries
    sub = clearance_percent(col, dims, 2, [0, 1], [3, 4])
    assert np.allclose(_half_up(sub), [[want[3][0], want[4][0]], [want[3][1], want[4][1]]])
