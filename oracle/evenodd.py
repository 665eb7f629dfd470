"""Even-odd (red-black) preconditioning of the two operators (test
infrastructure only; the solver-fidelity row that follows deflation).

On a torus with every side even, the hopping terms of both operators connect
sites of opposite parity, so with the sites ordered even first

    A = [[A_ee, A_eo], [A_oe, A_oo]],   A_ee = A_oo = d I   (d = 8 + m^2 for the
                                                             Laplacian, 1 for Wilson)

and A x = b is solved through the Schur complement on the even sites,

    S x_e = b_e - A_eo A_oo^{-1} b_o,   S = A_ee - A_eo A_oo^{-1} A_oe,
    x_o = A_oo^{-1} (b_o - A_oe x_e).

For the Laplacian A_eo = -H_eo (H the sum of the eight hops), so
S = d - H_eo H_oe / d; for Wilson A_eo = -kappa D_eo, so S = 1 - kappa^2 D_eo D_oe.
The Krylov vectors then live on half the sites, and S is better conditioned
than A.  The paper's solves use the library's own (multigrid) solver; this is
the standard first step towards it for these operators.
"""
import numpy as np

from . import operators as ops
from .lattice import parity


def check_even(dims):
    if any(D % 2 for D in dims):
        raise ValueError("even-odd preconditioning needs every lattice side even")


def split(dims):
    """(even site indices, odd site indices), each in storage order."""
    check_even(dims)
    par = parity(dims)
    return np.nonzero(par == 0)[0], np.nonzero(par == 1)[0]


def _full(v_e, v_o, ev, od, N, dof):
    f = np.zeros((N, dof), dtype=np.result_type(v_e, v_o))
    f[ev] = v_e.reshape(-1, dof)
    f[od] = v_o.reshape(-1, dof)
    return f


class LaplacianEO:
    """Schur complement of the shifted Laplacian on the even sites."""

    def __init__(self, dims, m2):
        self.dims, self.m2, self.d = list(dims), m2, 2 * len(dims) + m2
        self.ev, self.od = split(dims)
        self.N = int(np.prod(dims))

    def hop(self, f):
        """H f = sum_mu [f(x + mu) + f(x - mu)] on the whole lattice."""
        return self.d * f - ops.laplacian_apply(f, self.dims, self.m2)

    def hop_eo(self, x_o):
        """(H_eo x_o): the even sites of H applied to a field that lives on the odd sites."""
        f = np.zeros(self.N)
        f[self.od] = x_o
        return self.hop(f)[self.ev]

    def hop_oe(self, x_e):
        f = np.zeros(self.N)
        f[self.ev] = x_e
        return self.hop(f)[self.od]

    def schur(self, x_e):
        return self.d * x_e - self.hop_eo(self.hop_oe(x_e)) / self.d

    def rhs(self, b):
        b = np.asarray(b).reshape(-1)
        return b[self.ev] + self.hop_eo(b[self.od]) / self.d

    def reconstruct(self, x_e, b):
        b = np.asarray(b).reshape(-1)
        x = np.zeros(self.N)
        x[self.ev] = x_e
        x[self.od] = (b[self.od] + self.hop_oe(x_e)) / self.d
        return x


class WilsonEO:
    """Schur complement of the Wilson-Dirac operator on the even sites."""

    def __init__(self, dims, U, kappa, antiperiodic_t=True):
        self.dims, self.U, self.kappa, self.ap = list(dims), np.asarray(U), kappa, antiperiodic_t
        self.ev, self.od = split(dims)
        self.N = int(np.prod(dims))

    def _hop(self, f):
        return ops.wilson_hop(f.reshape(self.N, 4, 3), self.U, self.dims, self.ap).reshape(self.N, 12)

    def hop_eo(self, x_o):
        f = np.zeros((self.N, 12), dtype=np.complex128)
        f[self.od] = np.asarray(x_o).reshape(-1, 12)
        return self._hop(f)[self.ev]

    def hop_oe(self, x_e):
        f = np.zeros((self.N, 12), dtype=np.complex128)
        f[self.ev] = np.asarray(x_e).reshape(-1, 12)
        return self._hop(f)[self.od]

    def schur(self, x_e):
        x_e = np.asarray(x_e).reshape(-1, 12)
        return x_e - self.kappa ** 2 * self.hop_eo(self.hop_oe(x_e))

    def rhs(self, b):
        b = np.asarray(b).reshape(self.N, 12)
        return b[self.ev] + self.kappa * self.hop_eo(b[self.od])

    def reconstruct(self, x_e, b):
        b = np.asarray(b).reshape(self.N, 12)
        x = np.zeros((self.N, 12), dtype=np.complex128)
        x[self.ev] = np.asarray(x_e).reshape(-1, 12)
        x[self.od] = b[self.od] + self.kappa * self.hop_oe(x_e)
        return x


class WilsonCloverEO(WilsonEO):
    """Schur complement of the clover Wilson-Dirac operator (oracle/clover.py).
    The diagonal blocks are no longer the identity but per-site 12 x 12
    matrices, A_ee = 1 + C_ee and A_oo = 1 + C_oo, so

        S = A_ee - kappa^2 D_eo A_oo^{-1} D_oe,
        rhs = b_e + kappa D_eo A_oo^{-1} b_o,
        x_o = A_oo^{-1} (b_o + kappa D_oe x_e),

    with A_oo^{-1} the site-by-site inverse (a library inverse per site)."""

    def __init__(self, dims, U, kappa, csw, antiperiodic_t=True):
        super().__init__(dims, U, kappa, antiperiodic_t)
        from .clover import clover_blocks
        C = clover_blocks(self.U, self.dims, kappa, csw)
        I12 = np.eye(12)
        self.Aee = I12 + C[self.ev]
        self.Aoo_inv = np.linalg.inv(I12 + C[self.od])

    @staticmethod
    def _blk(B, x):
        return np.einsum('nij,nj->ni', B, np.asarray(x).reshape(-1, 12))

    def schur(self, x_e):
        x_e = np.asarray(x_e).reshape(-1, 12)
        return self._blk(self.Aee, x_e) - self.kappa ** 2 * self.hop_eo(self._blk(self.Aoo_inv, self.hop_oe(x_e)))

    def rhs(self, b):
        b = np.asarray(b).reshape(self.N, 12)
        return b[self.ev] + self.kappa * self.hop_eo(self._blk(self.Aoo_inv, b[self.od]))

    def reconstruct(self, x_e, b):
        b = np.asarray(b).reshape(self.N, 12)
        x = np.zeros((self.N, 12), dtype=np.complex128)
        x[self.ev] = np.asarray(x_e).reshape(-1, 12)
        x[self.od] = self._blk(self.Aoo_inv, b[self.od] + self.kappa * self.hop_oe(x_e))
        return x
