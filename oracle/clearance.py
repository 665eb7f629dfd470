"""Clearance of a colouring at other displacements (Sec. 3.3, Thm 3.6; Sec. 4.3,
Table 5).  Test infrastructure only.

A (p0, k0)-colouring used for displacement p leaves some neighbours of the
displaced pair x+ = x + p e_mu, x- = x - p e_mu unannihilated: those y that
share x's colour.  Table 5 reports, for each (p, k), the percentage of the
nodes at distance exactly k from the pair {x+, x-} that share x's colour,
averaged over all nodes x.

Readings (the section states the statistic in one sentence):
  * "distance k from x+ or x-" is the distance to the nearer of the two,
    min(||o - p e_mu||_1, ||o + p e_mu||_1) = k for y = x + o, o in Z^d;
  * the shell is a set of nodes (y taken mod D, each node once) and x itself
    (at distance p from both) is left out.
With the red-black greedy (8, 10)-colouring of the 32^4 tile (Table 2) these
readings reproduce every entry of Table 5.

The shell's offsets, reduced mod D, do not depend on x (the torus is
translation invariant), so the average over x of count_x / |S| is
Sum_{o in S} #{x : col(x) = col(x + o)} / (N |S|): the same finite integer sum
taken offset by offset, which is how it is evaluated here.
"""
import ctypes

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        _lib.oracle_offset_matches.restype = None
        _lib.oracle_offset_matches.argtypes = [
            ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int32), ctypes.c_int,
            ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64)]
    return _lib


def _l1_ball(n, r):
    """All integer vectors of length n with L1 norm <= r."""
    if n == 0:
        yield ()
        return
    for a in range(-r, r + 1):
        for rest in _l1_ball(n - 1, r - abs(a)):
            yield (a,) + rest


def shell(dims, mu, p, k):
    """Offsets (reduced mod dims, as tuples) of the nodes y != x with
    min(||y - x+||_1, ||y - x-||_1) = k."""
    d = len(dims)
    out = set()
    for rest in _l1_ball(d - 1, k):
        t = k - sum(abs(a) for a in rest)          # distance left for dimension mu
        for om in {p + t, p - t, -p + t, -p - t}:
            if min(abs(om - p), abs(om + p)) != t:
                continue
            o = rest[:mu] + (om,) + rest[mu:]
            red = tuple(o[nu] % dims[nu] for nu in range(d))
            if any(red):
                out.add(red)
    return sorted(out)


def offset_matches(col, dims, offsets):
    """#{x : col(x) = col(x + o)} for each offset o (rows of `offsets`)."""
    d = len(dims)
    offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32).reshape(-1, d))
    col = np.ascontiguousarray(col, dtype=np.int32)
    assert col.shape == (int(np.prod(dims)),)
    out = np.zeros(offs.shape[0], dtype=np.int64)
    if offs.shape[0]:
        _load().oracle_offset_matches(
            d, (ctypes.c_int * d)(*[int(D) for D in dims]), col.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
            int(offs.shape[0]), offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
            out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    return out


def clearance(col, dims, mu, p_list, k_list):
    """Integer form of the statistic: (matches, shell_size), each an int64
    array [len(p_list), len(k_list)]; matches = Sum_x #{y in S_x : col(y) =
    col(x)}.  The percentage of Table 5 is 100 matches / (N shell_size)."""
    shells = {(p, k): shell(dims, mu, p, k) for p in p_list for k in k_list}
    distinct = sorted(set(o for s in shells.values() for o in s))
    counts = dict(zip(distinct, offset_matches(col, dims, distinct).tolist())) if distinct else {}
    matches = np.zeros((len(p_list), len(k_list)), dtype=np.int64)
    size = np.zeros((len(p_list), len(k_list)), dtype=np.int64)
    for i, p in enumerate(p_list):
        for j, k in enumerate(k_list):
            s = shells[(p, k)]
            size[i, j] = len(s)
            matches[i, j] = sum(counts[o] for o in s)
    return matches, size


def clearance_percent(col, dims, mu, p_list, k_list):
    matches, size = clearance(col, dims, mu, p_list, k_list)
    N = int(np.prod(dims))
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(size > 0, 100.0 * matches / (N * np.maximum(size, 1)), 0.0)
