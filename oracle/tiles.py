"""Tile policy of Sec. 3.5 (test infrastructure only).

A tile is a smaller torus whose colouring is repeated over the lattice.  It
must hold a whole displaced neighbourhood N(x, p, k): every side at least
2k + 1, and the side along the displacement at least 2(p + k) + 1 (for a list
of displacements, the largest p decides).  Its sides must divide the lattice's.
The paper takes the smallest power of two above the minimum, capped at the
lattice side; for lattice sides that are not powers of two (a factor of three,
which the paper mentions) this is read as the smallest divisor of the lattice
side that is at least the minimum, else the lattice side itself.  For
power-of-two sides both readings give the same tile (Table 2).
"""


def min_tile_side(i, mu, p_list, k):
    """Smallest side along dimension i that holds N(x, p, k) (Sec. 3.5)."""
    if i == mu:
        return 2 * (max(int(p) for p in p_list) + k) + 1
    return 2 * k + 1


def tile_dims(dims, mu, p_list, k):
    out = []
    for i, D in enumerate(dims):
        need = min_tile_side(i, mu, p_list, k)
        side = D
        for t in range(1, D + 1):
            if D % t == 0 and t >= need:
                side = t
                break
        out.append(side)
    return out
