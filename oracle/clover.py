"""Clover (Sheikholeslami-Wohlert) term of the Wilson-Dirac operator (test
infrastructure only; the operator-fidelity row that follows deflation).

The paper's production operator is a clover Wilson-Dirac matrix (Sec. 4.2)
whose definition it takes from the lattice literature.  The textbook form is
written out here; the sign that goes with this package's hopping term is a
convention, chosen as

    (A_c psi)(x) = (A_W psi)(x) - kappa c_sw sum_{mu < nu} sigma_{mu nu} F_{mu nu}(x) psi(x),

  sigma_{mu nu} = (i / 2) [g_mu, g_nu]                 (Hermitian 4 x 4),
  F_{mu nu}(x)  = (Q_{mu nu}(x) - Q_{mu nu}(x)^H) / (8 i)  (Hermitian 3 x 3),

and Q_{mu nu}(x) the sum of the four plaquettes in the (mu, nu) plane that
start and end at x, each run in the same sense (the "clover leaves").  The
term is site-local (one Hermitian 12 x 12 block per site), commutes with g_5
(so A_c keeps g_5-hermiticity), and vanishes where the links are trivial.
"""
import numpy as np

from . import operators as ops
from .lattice import volume


def sigma(mu, nu):
    g, _ = ops.gammas()
    return 0.5j * (g[mu] @ g[nu] - g[nu] @ g[mu])


def _dag(M):
    return np.conj(np.swapaxes(M, -1, -2))


def clover_leaves(U, dims, mu, nu):
    """Q_{mu nu}(x), [N, 3, 3]: the four plaquettes at x in the (mu, nu) plane,
    each a closed loop from x that turns the same way:
      x -> x+mu -> x+mu+nu -> x+nu -> x,
      x -> x+nu -> x+nu-mu -> x-mu -> x,
      x -> x-mu -> x-mu-nu -> x-nu -> x,
      x -> x-nu -> x-nu+mu -> x+mu -> x."""
    fwd, bwd = ops.neighbour_tables(dims)
    Um, Un = U[:, mu], U[:, nu]
    p_m, p_n, m_m, m_n = fwd[mu], fwd[nu], bwd[mu], bwd[nu]
    # 1: U_mu(x) U_nu(x+mu) U_mu(x+nu)^H U_nu(x)^H
    q = Um @ Un[p_m] @ _dag(Um[p_n]) @ _dag(Un)
    # 2: U_nu(x) U_mu(x+nu-mu)^H U_nu(x-mu)^H U_mu(x-mu)
    q = q + Un @ _dag(Um[m_m[p_n]]) @ _dag(Un[m_m]) @ Um[m_m]
    # 3: U_mu(x-mu)^H U_nu(x-mu-nu)^H U_mu(x-mu-nu) U_nu(x-nu)
    q = q + _dag(Um[m_m]) @ _dag(Un[m_n[m_m]]) @ Um[m_n[m_m]] @ Un[m_n]
    # 4: U_nu(x-nu)^H U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^H
    q = q + _dag(Un[m_n]) @ Um[m_n] @ Un[p_m[m_n]] @ _dag(Um)
    return q


def field_strength(U, dims, mu, nu):
    """F_{mu nu}(x) = (Q - Q^H) / (8 i), [N, 3, 3] Hermitian."""
    Q = clover_leaves(U, dims, mu, nu)
    return (Q - _dag(Q)) / 8j


def clover_blocks(U, dims, kappa, csw):
    """C(x) = -kappa c_sw sum_{mu<nu} sigma_{mu nu} (x) F_{mu nu}(x) as [N, 12, 12]
    (component = 3 * spin + colour)."""
    N = volume(dims)
    C = np.zeros((N, 12, 12), dtype=np.complex128)
    for mu in range(4):
        for nu in range(mu + 1, 4):
            F = field_strength(U, dims, mu, nu)
            C += np.einsum('st,nab->nsatb', sigma(mu, nu), F).reshape(N, 12, 12)
    return -kappa * csw * C


def clover_apply(psi, U, kappa, csw, dims, antiperiodic_t=True):
    """(A_c psi) = (A_W psi) + C psi, psi [N, 4, 3]."""
    psi = np.asarray(psi, dtype=np.complex128)
    N = volume(dims)
    C = clover_blocks(U, dims, kappa, csw)
    local = np.einsum('nij,nj->ni', C, psi.reshape(N, 12)).reshape(N, 4, 3)
    return ops.wilson_apply(psi, U, kappa, dims, antiperiodic_t) + local


def clover_apply_dagger(psi, U, kappa, csw, dims, antiperiodic_t=True):
    """A_c^H = A_W^H + C (each C(x) is Hermitian)."""
    psi = np.asarray(psi, dtype=np.complex128)
    N = volume(dims)
    C = clover_blocks(U, dims, kappa, csw)
    local = np.einsum('nij,nj->ni', C, psi.reshape(N, 12)).reshape(N, 4, 3)
    return ops.wilson_apply_dagger(psi, U, kappa, dims, antiperiodic_t) + local


def uniform_abelian_links(dims, phi_quanta, plane=(0, 1)):
    """Links of a uniform abelian flux through every plaquette of one plane:
    each plaquette of `plane` equals exp(i phi) times the identity, with
    phi = 2 pi n / (L_mu L_nu) (n = phi_quanta, so the flux closes on the
    torus), every other plaquette 1.  Landau-like gauge: U_nu(x) = e^{i phi x_mu},
    U_mu(x) = e^{-i phi L_mu x_nu} on the last slice x_mu = L_mu - 1, else 1."""
    from .lattice import coords
    mu, nu = plane
    xs = coords(dims)
    N = volume(dims)
    Lm, Ln = dims[mu], dims[nu]
    phi = 2 * np.pi * phi_quanta / (Lm * Ln)
    U = np.zeros((N, 4, 3, 3), dtype=np.complex128)
    U[:] = np.eye(3)
    U[:, nu] = np.exp(1j * phi * xs[:, mu])[:, None, None] * np.eye(3)
    last = xs[:, mu] == Lm - 1
    U[last, mu] = np.exp(-1j * phi * Lm * xs[last, nu])[:, None, None] * np.eye(3)
    return U, phi


class WilsonClover:
    """Clover Wilson-Dirac operator, dof = 12 (same interface as the oracle's Wilson)."""
    dof = 12

    def __init__(self, dims, U, kappa, csw, antiperiodic_t=True):
        self.dims, self.U, self.kappa, self.csw = list(dims), np.asarray(U), float(kappa), float(csw)
        self.ap = bool(antiperiodic_t)

    def _sp(self, x):
        return np.asarray(x, dtype=np.complex128).reshape(-1, 4, 3)

    def apply(self, x):
        return clover_apply(self._sp(x), self.U, self.kappa, self.csw, self.dims, self.ap).reshape(-1, 12)

    def apply_dagger(self, x):
        return clover_apply_dagger(self._sp(x), self.U, self.kappa, self.csw, self.dims, self.ap).reshape(-1, 12)

    def solve(self, b, tol=1e-10, maxit=100000):
        from .solvers import bicgstab
        f = lambda v: self.apply(v).reshape(-1)
        x, its, rel = bicgstab(f, np.asarray(b, dtype=np.complex128).reshape(-1), tol, maxit)
        return x.reshape(-1, 12), its, rel
