"""Toroidal lattice Z^d_D, storage index and the displacement permutation.

Sec. 2 (Background): the lattice is Z_{D_1} x ... x Z_{D_d}; two nodes are
neighbours when their coordinates differ by one in one dimension, modulo D.
Sec. 3 (Probing for permutations): P places the elements of A^{-1} that belong
to the displacement p on the main diagonal; its inverse P^T maps y -> y - p.

Storage index (a choice of this implementation; the paper leaves "the
particular index ordering of the application" open, Sec. 3):
    idx(x) = x_0 + D_0 (x_1 + D_1 (x_2 + D_2 x_3)),   x_0 fastest.

Reading of the direction of P (Sec. 3; the sum over A^{-1}_{x, x+p} and the
MATLAB ``perm`` line disagree on which index carries +p): here
    (P f)(x) = f(x + p e_mu),  so  Tr(P A^{-1}) = sum_x A^{-1}(x + p, x).
P is a pure permutation (no boundary sign), as in the paper.
"""
import numpy as np


def volume(dims):
    n = 1
    for D in dims:
        n *= int(D)
    return n


def coords(dims):
    """Coordinates of every site, shape [N, d], row i = coordinates of idx i."""
    d = len(dims)
    N = volume(dims)
    idx = np.arange(N, dtype=np.int64)
    out = np.zeros((N, d), dtype=np.int64)
    rem = idx.copy()
    for mu in range(d):
        out[:, mu] = rem % dims[mu]
        rem //= dims[mu]
    return out


def index_of(xs, dims):
    """Storage index of coordinate rows xs (taken modulo dims)."""
    xs = np.asarray(xs, dtype=np.int64)
    idx = np.zeros(xs.shape[:-1], dtype=np.int64)
    stride = 1
    for mu, D in enumerate(dims):
        idx += (xs[..., mu] % D) * stride
        stride *= D
    return idx


def shift_map(dims, mu, p):
    """perm[i] = idx(x_i + p e_mu): (P f)[i] = f[perm[i]]  (Sec. 3, perm)."""
    xs = coords(dims)
    xs[:, mu] += p
    return index_of(xs, dims)


def displace(f, dims, mu, p):
    """(P f)(x) = f(x + p e_mu) for f of shape [N, ...]."""
    return np.asarray(f)[shift_map(dims, mu, p)]


def displace_T(f, dims, mu, p):
    """(P^T f)(y) = f(y - p e_mu)  (Sec. 3: the inverse permutation)."""
    return np.asarray(f)[shift_map(dims, mu, -p)]


def parity(dims):
    """Red-black parity (sum of coordinates mod 2) of every site."""
    return coords(dims).sum(axis=1) % 2


def natural_order(dims, mu=None):
    """Natural visit order: the storage order, x_0 fastest (Sec. 3.1 names a
    "natural" order without fixing the index order).

    Reading: the lattice is held in the application's (x, y, z, t) order with
    x fastest and t slowest (the usual LQCD lexicographic order), whatever the
    displaced dimension.  With the paper's Table 2 tiles mapped back from
    (z, x, y, t) to (x, y, z, t), the smaller colour count of this order and
    of red-black reproduces every k <= 4 entry of Table 4.  `mu` is accepted
    for symmetry with the other orders and does not change the result.
    """
    return np.arange(volume(dims), dtype=np.int64)


def redblack_order(dims, mu):
    """Red-black visit order: every even-parity site (sum of coordinates even)
    in natural order, then every odd-parity site in natural order (Sec. 3.1)."""
    nat = natural_order(dims, mu)
    par = parity(dims)[nat]
    return np.concatenate([nat[par == 0], nat[par == 1]])


def visit_order(dims, mu, order):
    if order == 0:
        return natural_order(dims, mu)
    if order == 1:
        return redblack_order(dims, mu)
    raise ValueError("order must be 0 (natural) or 1 (red-black)")
