"""Pins for the oracle's stencil and greedy colouring (Secs. 2.1, 3, 3.1, 3.3, 3.5, 4.1)."""
import itertools

import numpy as np
import pytest

from conftest import read_golden
from oracle import lattice as L
from oracle.bounds import lower_bound
from oracle.colouring import conflicts, greedy_colour, tile_replicate
from oracle.stencil import displaced_stencil, l1_ball


def _table4_rows(kmax):
    for r in read_golden("table4_colours.txt"):
        p, k, tz, tx, ty, tt, colours, lb = map(int, r)
        if k <= kmax:
            # the paper lists tiles as (z, x, y, t); the lattice here is (x, y, z, t)
            yield p, k, [tx, ty, tz, tt], colours, lb


@pytest.mark.parametrize("p,k,dims,colours,lb", list(_table4_rows(3)))
def test_table4_colour_counts_k_le_3(p, k, dims, colours, lb):
    """Table 4 first numbers: min over natural and red-black greedy orders."""
    m = [greedy_colour(dims, 2, [p], k, order)[1] for order in (0, 1)]
    assert min(m) == colours


@pytest.mark.slow
def test_table4_colour_counts_k4():
    for p, k, dims, colours, lb in _table4_rows(4):
        if k == 4:
            m = [greedy_colour(dims, 2, [p], k, order)[1] for order in (0, 1)]
            assert min(m) == colours, (p, k)


def test_fig1_1d_distance3_four_colours():
    """Sec. 2.1, Fig. 1: a 32-node periodic 1D Laplacian, distance-3 colouring -> 4 colours."""
    col, m = greedy_colour([32], 0, [0], 3, 0)
    assert m == 4
    assert conflicts(col, [32], 0, [0], 3) == 0


def test_stencil_is_graph_of_symmetrised_PAk():
    """Sec. 3, Fig. 2: 1D periodic lattice of 32 points, p = 10, k = 4.  The
    neighbourhood N(x,p,k) (minus x) is the nonzero pattern of row x of
    P A^k + (P A^k)^T, with A the 1D Laplacian (dense matrix powers)."""
    n, p, k = 32, 10, 4
    A = 2.0 * np.eye(n) - np.roll(np.eye(n), 1, axis=1) - np.roll(np.eye(n), -1, axis=1)
    A = A + 0.01 * np.eye(n)
    Ak = np.linalg.matrix_power(A, k)
    perm = L.shift_map([n], 0, p)
    PAk = Ak[perm, :]
    pattern = (np.abs(PAk) + np.abs(PAk.T)) > 1e-12
    st = displaced_stencil(1, 0, [p], k)
    for x in range(n):
        mine = {(x + int(o[0])) % n for o in st} - {x}
        theirs = set(np.nonzero(pattern[x])[0].tolist()) - {x}
        assert mine == theirs


def test_stencil_sizes_4d():
    """|N(x,0,k)| = |B_k| - 1 with |B_k| = 1, 9, 41, 129, 321 in 4D."""
    for k, b in zip(range(0, 5), [1, 9, 41, 129, 321]):
        assert len(l1_ball(4, k)) == b
        assert displaced_stencil(4, 2, [0], k).shape[0] == b - 1


@pytest.mark.parametrize("p,k", [(p, k) for k in range(1, 5) for p in range(k, 8)])
def test_theorem_3_1(p, k):
    """Thm 3.1: if p >= k, no y != x with y_1 = x_1 is in N(x,p,k)."""
    st = displaced_stencil(3, 0, [p], k)
    assert not np.any(st[:, 0] == 0)


@pytest.mark.parametrize("p,k,lam", [(p, k, lam) for p in range(0, 5) for k in range(1, 5)
                                     for lam in range(0, k + 1)])
def test_theorem_3_6_clearance(p, k, lam):
    """Thm 3.6: N(0, p +- lam, k - lam) is contained in N(0, p, k)."""
    big = {tuple(o) for o in displaced_stencil(3, 0, [p], k)}
    for q in (p + lam, p - lam):
        small = {tuple(o) for o in displaced_stencil(3, 0, [abs(q)], k - lam)}
        assert small <= big


def test_multi_displacement_is_union():
    """Sec. 3.4: the stencil of a list of displacements is the union."""
    u = {tuple(o) for o in displaced_stencil(4, 2, [1, 3], 2)}
    a = {tuple(o) for o in displaced_stencil(4, 2, [1], 2)}
    b = {tuple(o) for o in displaced_stencil(4, 2, [3], 2)}
    assert u == a | b


@pytest.mark.parametrize("dims,mu,p,k,order", [
    ([6, 5, 7, 4], 2, 1, 1, 0), ([6, 5, 7, 4], 2, 2, 2, 1), ([8, 4, 4, 6], 0, 3, 2, 0),
    ([5, 5, 5, 5], 3, 0, 2, 1), ([7, 6, 9, 4], 2, 4, 3, 0), ([3, 4, 5, 6], 1, 1, 3, 1)])
def test_colouring_valid_brute_force(dims, mu, p, k, order):
    """Validity by brute force: no two sites at L1 torus distance <= k from the
    displaced centres x +- p share a colour; colours <= |stencil| + 1."""
    col, m = greedy_colour(dims, mu, [p], k, order)
    xs = L.coords(dims)
    D = np.asarray(dims)
    for i in range(xs.shape[0]):
        for sgn in (+1, -1):
            c = xs[i].copy()
            c[mu] += sgn * p
            diff = np.abs(xs - c) % D
            dist = np.minimum(diff, D - diff).sum(axis=1)
            near = (dist <= k)
            near[i] = False
            assert not np.any(col[near] == col[i])
    assert m <= displaced_stencil(4, mu, [p], k).shape[0] + 1
    assert set(np.unique(col).tolist()) == set(range(m))


def test_colouring_greedy_first_fit_property():
    """Every site's colour is the smallest one absent among its earlier-visited
    neighbours (the defining property of sequential greedy)."""
    dims, mu, p, k = [6, 4, 8, 4], 2, 2, 2
    for order in (0, 1):
        col, _ = greedy_colour(dims, mu, [p], k, order)
        visit = L.visit_order(dims, mu, order)
        rank = np.empty_like(visit)
        rank[visit] = np.arange(visit.shape[0])
        st = displaced_stencil(4, mu, [p], k)
        xs = L.coords(dims)
        nb = L.index_of(xs[:, None, :] + st[None], dims)
        for x in range(xs.shape[0]):
            earlier = {int(col[y]) for y in nb[x] if y != x and rank[y] < rank[x]}
            c = 0
            while c in earlier:
                c += 1
            assert col[x] == c


@pytest.mark.parametrize("p,k,dims", [(0, 1, [4, 4, 4, 4]), (2, 1, [4, 4, 8, 4]), (1, 2, [8, 8, 8, 8]),
                                      (3, 2, [8, 8, 16, 8]), (4, 3, [8, 8, 16, 8])])
def test_colour_count_at_least_lower_bound(p, k, dims):
    """Eq. (13) bounds the colour count on tiles meeting the Sec. 3.5 size rule."""
    for order in (0, 1):
        _, m = greedy_colour(dims, 2, [p], k, order)
        assert m >= lower_bound(4, p, k)


def test_tile_replication_is_valid():
    """Sec. 3.5: a colouring of a tile that fits N(x,p,k) repeats validly."""
    tile = [4, 4, 8, 4]
    col, m = greedy_colour(tile, 2, [2], 1, 0)
    big = [8, 8, 16, 8]
    colb = tile_replicate(col, tile, big)
    assert conflicts(colb, big, 2, [2], 1) == 0
    assert int(colb.max()) + 1 == m


def test_redblack_order_is_parity_split():
    dims = [4, 3, 5, 2]
    o = L.redblack_order(dims, 2)
    par = L.parity(dims)[o]
    n_even = int((L.parity(dims) == 0).sum())
    assert np.all(par[:n_even] == 0) and np.all(par[n_even:] == 1)
    assert sorted(o.tolist()) == list(range(120))


def test_first_fit_checker_accepts_greedy_and_flags_changes():
    """The sampled checker used at full size: silent on the greedy colouring
    (all sites), and flags a site whose colour is changed."""
    from oracle.colouring import first_fit_violations
    dims = [6, 4, 8, 4]
    for order in (0, 1):
        col, m = greedy_colour(dims, 2, [2], 2, order)
        assert first_fit_violations(col, dims, 2, [2], 2, order, range(col.size)) == []
        bad = col.copy()
        bad[100] = (bad[100] + 1) % m
        assert 100 in first_fit_violations(bad, dims, 2, [2], 2, order, range(col.size))


def _first_fit_nested(col_local_pairs, parent, dims, mu, p, k, order):
    """Independent check of the nested definition: per node, the local colour
    is the smallest absent among earlier-visited neighbours of the same parent
    class; pairs are numbered in first-visit order."""
    st = displaced_stencil(4, mu, [p], k)
    visit = L.visit_order(dims, mu, order)
    rank = np.empty_like(visit)
    rank[visit] = np.arange(visit.shape[0])
    xs = L.coords(dims)
    nb = L.index_of(xs[:, None, :] + st[None], dims)
    col = col_local_pairs
    # recover local colours: within a parent class, number the child classes by first visit
    seen, numbering = {}, []
    for x in visit:
        c = int(col[x])
        if c not in seen:
            seen[c] = len(seen)
            numbering.append(c)
    assert numbering == list(range(len(numbering)))               # first-visit order
    local = {}
    for x in visit:
        pa, c = int(parent[x]), int(col[x])
        earlier = {local[int(y)] for y in nb[x] if y != x and rank[y] < rank[x] and parent[y] == pa}
        lo = 0
        while lo in earlier:
            lo += 1
        local[int(x)] = lo
    # equal colour <=> equal (parent, local)
    key = {}
    for x in range(col.size):
        kk = (int(parent[x]), local[x])
        assert key.setdefault(int(col[x]), kk) == kk


@pytest.mark.parametrize("dims,mu,p,order", [([8, 8, 8, 8], 3, 2, 0), ([8, 8, 8, 8], 3, 0, 1), ([6, 4, 8, 4], 2, 1, 1)])
def test_nested_colouring_levels(dims, mu, p, order):
    """Nested colourings for k = 1..3: valid at each level, every class inside
    one parent class, local first-fit within each parent class, pairs numbered
    in first-visit order."""
    from oracle.colouring import nested_colour
    prev, _ = greedy_colour(dims, mu, [p], 1, order)
    for k in (2, 3):
        col, m = nested_colour(dims, mu, [p], k, prev, order)
        assert conflicts(col, dims, mu, [p], k) == 0
        assert set(np.unique(col).tolist()) == set(range(m))
        for c in range(m):
            assert np.unique(prev[col == c]).size == 1             # nesting
        _first_fit_nested(col, prev, dims, mu, p, k, order)
        prev = col


@pytest.mark.parametrize("order", [0, 1])
def test_nested_with_one_parent_is_algorithm_1(order):
    """A constant parent colouring leaves nothing to nest: the result is the
    plain greedy colouring (first-fit colours already appear in order)."""
    from oracle.colouring import nested_colour
    for dims, mu, p, k in [([8, 8, 8, 8], 3, 2, 2), ([5, 6, 7, 3], 2, 1, 2)]:
        want, mw = greedy_colour(dims, mu, [p], k, order)
        got, mg = nested_colour(dims, mu, [p], k, np.zeros(int(np.prod(dims)), np.int32), order)
        assert mg == mw and np.array_equal(got, want)


def test_nested_probes_sum_to_parent_probe():
    """The point of nesting: the probes of the child classes of a parent class
    sum to the parent's probe (Eq. (4) with shared noise), so solves at the
    finer level give the coarser estimate by linearity."""
    from oracle.colouring import nested_colour
    from oracle.probes import probe
    dims, mu, p = [8, 8, 8, 8], 3, 2
    par, mp_ = greedy_colour(dims, mu, [p], 1, 0)
    ch, mc = nested_colour(dims, mu, [p], 2, par, 0)
    for kind in (0, 1):                                             # Z2, Z4
        for c1 in range(mp_):
            kids = np.unique(ch[par == c1])
            s = sum(probe(ch, int(c2), 11, 0, kind) for c2 in kids)
            assert np.array_equal(s, probe(par, c1, 11, 0, kind))
