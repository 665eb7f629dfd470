"""Displaced distance-k neighbourhood as a stencil of coordinate offsets.

Eq. (8), Sec. 3: N(x,p,k) = {y : ||y - x^+||_1 <= k} U {y : ||y - x^-||_1 <= k}
with x^{+-} = x +- p (Eq. (7)); x itself is excluded during colouring.
Sec. 3.1: the neighbourhood is stored once as a list of offsets ("stencil")
that are added to the coordinates of any node (Algorithm 2 builds it; its body
is not in the text, so this follows the set definition directly).
Sec. 3.4: for several displacements the stencils are unioned.
"""
import itertools

import numpy as np


def l1_ball(d, k):
    """All integer offsets o in Z^d with ||o||_1 <= k."""
    rng = range(-k, k + 1)
    return [o for o in itertools.product(rng, repeat=d) if sum(abs(c) for c in o) <= k]


def displaced_stencil(d, mu, p_list, k):
    """Sorted list of offsets o != 0 with o in N(0, p_n e_mu, k) for some n.

    Duplicates from overlapping balls are removed (Sec. 3.1 removes them by
    sorting).  Returns an int64 array of shape [n_offsets, d].
    """
    if isinstance(p_list, (int, np.integer)):
        p_list = [int(p_list)]
    out = set()
    for p in p_list:
        centre = [0] * d
        centre[mu] = int(p)
        for sgn in (+1, -1):
            for o in l1_ball(d, k):
                y = tuple(sgn * centre[i] + o[i] for i in range(d))
                if any(y):
                    out.add(y)
    return np.array(sorted(out), dtype=np.int64).reshape(-1, d)


def neighbour_sets(dims, mu, p_list, k):
    """For every site x the set of sites x + o (mod D), o in the stencil, with
    x itself removed (Sec. 3: "we exclude {x} from the neighbourhood")."""
    from .lattice import coords, index_of
    d = len(dims)
    st = displaced_stencil(d, mu, p_list, k)
    xs = coords(dims)
    nb = index_of(xs[:, None, :] + st[None, :, :], dims)  # [N, n_off]
    self_idx = np.arange(xs.shape[0])[:, None]
    return [set(row[row != self_idx[i, 0]].tolist()) for i, row in enumerate(nb)]
