"""Lattice operators A, in FP64.

The paper abstracts its LQCD operator (a clover Wilson-Dirac matrix, Sec. 4.2)
to "a non-singular matrix discretised on a regular toroidal lattice" (Sec. 2).
Two concrete operators are used here; their definitions are this
implementation's choice, not the paper's:

Shifted scalar Laplacian (periodic, d dimensions):
    (A f)(x) = (2d + m^2) f(x) - sum_mu [ f(x + mu) + f(x - mu) ]

Wilson-Dirac operator (4D, 12 = 4 spin x 3 colour components per site):
    (A psi)(x) = psi(x) - kappa * (H psi)(x)
    (H psi)(x) = sum_mu [ (1 - g_mu) U_mu(x) psi(x + mu) eta_+(x, mu)
                        + (1 + g_mu) U_mu(x - mu)^dagger psi(x - mu) eta_-(x, mu) ]
with eta = -1 on hops that cross the time boundary when time is antiperiodic
(mu = 3), else +1.  Gamma matrices in the chiral Euclidean basis
    g_k = [[0, -i s_k], [i s_k, 0]]  (k = 1, 2, 3 -> mu = 0, 1, 2),
    g_4 = [[0, I], [I, 0]]           (mu = 3),
    g_5 = g_1 g_2 g_3 g_4 = diag(1, 1, -1, -1).

Array layouts: a scalar field is [N] (or [N, 1]); a spinor field is
[N, 4, 3] (spin, colour); links are [N, 4, 3, 3] (direction mu, row a,
column b).  N is in storage order (x_0 fastest).
"""
import numpy as np

from .lattice import coords, index_of, volume

SIGMA = [np.array([[0, 1], [1, 0]], dtype=np.complex128),
         np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
         np.array([[1, 0], [0, -1]], dtype=np.complex128)]


def gammas():
    """[g_0, g_1, g_2, g_3] for mu = x, y, z, t, and g_5."""
    Z = np.zeros((2, 2), dtype=np.complex128)
    I2 = np.eye(2, dtype=np.complex128)
    g = []
    for k in range(3):
        g.append(np.block([[Z, -1j * SIGMA[k]], [1j * SIGMA[k], Z]]))
    g.append(np.block([[Z, I2], [I2, Z]]))
    g5 = g[0] @ g[1] @ g[2] @ g[3]
    return g, g5


def neighbour_tables(dims):
    """fwd[mu][i] = idx(x_i + mu), bwd[mu][i] = idx(x_i - mu)."""
    xs = coords(dims)
    fwd, bwd = [], []
    for mu in range(len(dims)):
        e = np.zeros(len(dims), dtype=np.int64)
        e[mu] = 1
        fwd.append(index_of(xs + e, dims))
        bwd.append(index_of(xs - e, dims))
    return fwd, bwd


def boundary_signs(dims, antiperiodic_t):
    """eta_+[mu][i] for the hop x -> x + mu and eta_-[mu][i] for x -> x - mu."""
    xs = coords(dims)
    N = volume(dims)
    ep = [np.ones(N) for _ in dims]
    em = [np.ones(N) for _ in dims]
    if antiperiodic_t:
        t = len(dims) - 1
        ep[t] = np.where(xs[:, t] == dims[t] - 1, -1.0, 1.0)
        em[t] = np.where(xs[:, t] == 0, -1.0, 1.0)
    return ep, em


def laplacian_apply(f, dims, m2):
    """(A f)(x) = (2d + m^2) f(x) - sum_mu [f(x+mu) + f(x-mu)] (periodic)."""
    f = np.asarray(f)
    fwd, bwd = neighbour_tables(dims)
    out = (2 * len(dims) + m2) * f
    for mu in range(len(dims)):
        out = out - f[fwd[mu]] - f[bwd[mu]]
    return out


def wilson_hop(psi, U, dims, antiperiodic_t=True):
    """(H psi)(x) as in the module docstring; psi [N,4,3], U [N,4,3,3]."""
    g, _ = gammas()
    I4 = np.eye(4, dtype=np.complex128)
    fwd, bwd = neighbour_tables(dims)
    ep, em = boundary_signs(dims, antiperiodic_t)
    out = np.zeros_like(psi, dtype=np.complex128)
    for mu in range(4):
        # forward hop: (1 - g_mu) U_mu(x) psi(x + mu)
        u_psi = np.einsum('nab,nsb->nsa', U[:, mu], psi[fwd[mu]])
        out += ep[mu][:, None, None] * np.einsum('st,nta->nsa', I4 - g[mu], u_psi)
        # backward hop: (1 + g_mu) U_mu(x - mu)^dagger psi(x - mu)
        udag_psi = np.einsum('nba,nsb->nsa', np.conj(U[bwd[mu], mu]), psi[bwd[mu]])
        out += em[mu][:, None, None] * np.einsum('st,nta->nsa', I4 + g[mu], udag_psi)
    return out


def wilson_apply(psi, U, kappa, dims, antiperiodic_t=True):
    """(A psi) = psi - kappa H psi."""
    psi = np.asarray(psi, dtype=np.complex128)
    return psi - kappa * wilson_hop(psi, U, dims, antiperiodic_t)


def wilson_apply_dagger(psi, U, kappa, dims, antiperiodic_t=True):
    """(A^dagger psi)(x) = psi(x) - kappa sum_mu [
         (1 - g_mu) U_mu(x - mu)^dagger psi(x - mu) eta_-(x, mu)
       + (1 + g_mu) U_mu(x) psi(x + mu) eta_+(x, mu) ]
    -- the conjugate transpose of each hop of A, written out."""
    g, _ = gammas()
    I4 = np.eye(4, dtype=np.complex128)
    fwd, bwd = neighbour_tables(dims)
    ep, em = boundary_signs(dims, antiperiodic_t)
    psi = np.asarray(psi, dtype=np.complex128)
    hop = np.zeros_like(psi)
    for mu in range(4):
        udag_psi = np.einsum('nba,nsb->nsa', np.conj(U[bwd[mu], mu]), psi[bwd[mu]])
        hop += em[mu][:, None, None] * np.einsum('st,nta->nsa', I4 - g[mu], udag_psi)
        u_psi = np.einsum('nab,nsb->nsa', U[:, mu], psi[fwd[mu]])
        hop += ep[mu][:, None, None] * np.einsum('st,nta->nsa', I4 + g[mu], u_psi)
    return psi - kappa * hop


def gamma5_apply(psi):
    _, g5 = gammas()
    return np.einsum('st,nta->nsa', g5, np.asarray(psi))
