"""Greedy displaced distance-k colouring (Algorithm 1, Sec. 3.1) and checks.

The sequential greedy loop itself is the plain C routine in greedy_colour.c;
this module prepares its inputs (stencil, Eq. (8); visit order, Sec. 3.1) and
provides the validity check used by the tests.
"""
import ctypes

import numpy as np

from . import build as _build
from .lattice import index_of, coords, visit_order, volume
from .stencil import displaced_stencil

_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        _lib.oracle_greedy_colour.restype = ctypes.c_int
        _lib.oracle_greedy_colour.argtypes = [
            ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
            ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64),
            ctypes.POINTER(ctypes.c_int32)]
    return _lib


def greedy_colour(dims, mu, p_list, k, order=0, visit=None):
    """Colour the torus `dims` for displacement(s) p_list along mu, distance k.

    order: 0 natural, 1 red-black (Sec. 3.1), or pass an explicit `visit`
    permutation of the storage indices.  Returns (col[int32, N], n_colours);
    colours are 0-based.
    """
    d = len(dims)
    st = displaced_stencil(d, mu, p_list, k).astype(np.int32)
    if visit is None:
        visit = visit_order(dims, mu, order)
    visit = np.ascontiguousarray(visit, dtype=np.int64)
    N = volume(dims)
    assert visit.shape == (N,)
    col = np.empty(N, dtype=np.int32)
    dims_c = (ctypes.c_int * d)(*[int(D) for D in dims])
    st_c = np.ascontiguousarray(st.reshape(-1))
    lib = _load()
    m = lib.oracle_greedy_colour(
        d, dims_c, int(st.shape[0]),
        st_c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
        visit.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
        col.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    if m < 0:
        raise MemoryError("oracle colouring failed")
    return col, int(m)


def nested_colour(dims, mu, p_list, k, parent, order=0):
    """Nested colouring at distance k under a coarser colouring `parent` (the
    hierarchical mode: a colouring grown from k1 to k > k1).  Greedy walk of
    Algorithm 1 in which a node only sees the neighbours of N(x, p, k) that
    share its parent colour; the colour of x is the pair (parent(x), local
    first-fit colour), the pairs numbered 0, 1, ... in the order the walk
    first meets them.  Nodes with the same colour then share the parent
    colour, and two neighbours never share a colour (different parents, or
    the same parent and different local colours).  Returns (col, n_colours)."""
    d = len(dims)
    st = displaced_stencil(d, mu, p_list, k).astype(np.int32)
    visit = np.ascontiguousarray(visit_order(dims, mu, order), dtype=np.int64)
    N = volume(dims)
    parent = np.ascontiguousarray(parent, dtype=np.int32)
    assert parent.shape == (N,)
    local = np.empty(N, dtype=np.int32)
    lib = _load()
    fn = lib.oracle_greedy_colour_nested
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                   ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
    st_c = np.ascontiguousarray(st.reshape(-1))
    m_local = fn(d, (ctypes.c_int * d)(*[int(D) for D in dims]), int(st.shape[0]),
                 st_c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                 visit.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                 parent.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                 local.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    if m_local < 0:
        raise MemoryError("oracle colouring failed")
    ids = {}
    col = np.empty(N, dtype=np.int32)
    for x in visit:
        key = (int(parent[x]), int(local[x]))
        if key not in ids:
            ids[key] = len(ids)
        col[x] = ids[key]
    return col, len(ids)


def conflicts(col, dims, mu, p_list, k):
    """Number of ordered pairs (x, y), y in N(x,p,k), y != x, sharing a colour.
    A valid distance-k colouring of the displaced graph has none."""
    d = len(dims)
    st = displaced_stencil(d, mu, p_list, k)
    xs = coords(dims)
    nb = index_of(xs[:, None, :] + st[None, :, :], dims)
    self_idx = np.arange(xs.shape[0])[:, None]
    same = (col[nb] == col[:, None]) & (nb != self_idx)
    return int(same.sum())


def tile_replicate(tile_col, tile_dims, dims):
    """Repeat a colouring of a tile over a lattice whose sides it divides
    (Sec. 3.5, tiles)."""
    for T, D in zip(tile_dims, dims):
        if D % T:
            raise ValueError("tile side must divide the lattice side")
    xs = coords(dims)
    return np.asarray(tile_col)[index_of(xs % np.asarray(tile_dims), tile_dims)]


def first_fit_violations(col, dims, mu, p_list, k, order, sites):
    """Sites x (of `sites`) whose colour is not the smallest colour absent
    among the neighbours of N(x, p, k) visited before x (Algorithm 1).  When
    no site of the lattice violates it, `col` is the greedy colouring itself
    (by induction over the visit order), so a sample of sites checks a
    colouring too large to recompute."""
    d = len(dims)
    st = displaced_stencil(d, mu, p_list, k)
    visit = visit_order(dims, mu, order)
    rank = np.empty_like(visit)
    rank[visit] = np.arange(visit.shape[0])
    col = np.asarray(col)
    xs = coords(dims)
    bad = []
    for x in sites:
        nb = index_of(xs[x][None, :] + st, dims)
        nb = nb[(nb != x) & (rank[nb] < rank[x])]
        earlier = np.zeros(len(st) + 2, dtype=bool)
        earlier[col[nb]] = True
        if int(col[x]) != int(np.argmin(earlier)):
            bad.append(int(x))
    return bad
