"""Probing vectors.

Eq. (4), Sec. 2.1: z_j(i) = 1 if colour(i) = j, else 0.
Eq. (5), Sec. 2.2: the unbiased probes are z_0 (.) z_j with z_0 a Rademacher
vector; s independent z_0 give s Hutchinson steps on A^{-1} (.) H H^T.
Sec. 4.2: spin-colour dilution is the Kronecker product with the 12 x 12
identity, so each probe becomes 12 vectors, one per spin-colour component a.

Layout: a probe on a lattice with `dof` components per site is an array of
shape [N, dof] (dof = 1 for the scalar Laplacian, 12 = 4 spins x 3 colours for
Wilson-Dirac, component a = 3 * spin + colour).
"""
import numpy as np

from .rng import noise


def probe(col, colour, seed, s, kind, dof=1, component=0):
    """Diluted (component = a): v_{s,c,a}(x, b) = z0_s(x) [col(x) = c] delta_{a b}.

    Undiluted (component = None): every component of a site of colour c gets
    its own noise value, the one of counter dof * x + b, so that the estimate
    has no bias from the off-diagonal spin-colour entries of a site.
    """
    col = np.asarray(col)
    N = col.shape[0]
    v = np.zeros((N, dof), dtype=np.complex128 if kind == 1 else np.float64)
    mask = col == colour
    if component is None:
        z = noise(seed, s, N * dof, kind).reshape(N, dof)
        v[mask, :] = z[mask, :]
    else:
        z0 = noise(seed, s, N, kind)
        v[mask, component] = z0[mask]
    return v


def probing_indicator(col, m):
    """H: the N x m matrix whose columns are the vectors of Eq. (4)."""
    col = np.asarray(col)
    H = np.zeros((col.shape[0], m))
    H[np.arange(col.shape[0]), col] = 1.0
    return H
