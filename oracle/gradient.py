"""Adjoint gradient of the probed trace estimate (not in the paper).

With the probes held fixed, T(theta) = sum_v v^H P A(theta)^{-1} v and
    dT/dtheta = - sum_v y^H (dA/dtheta) x,   x = A^{-1} v,  y = A^{-dagger} P^T v,
because d(A^{-1}) = -A^{-1} (dA) A^{-1} and v^H P A^{-1} = y^H.

Laplacian: dA/dm^2 = I, so dT/dm^2 = -sum y^H x.
Wilson:    dA/dkappa = -H, so dT/dkappa = sum y^H H x.
Links:     the entries of U_mu(x) are treated as 9 free complex numbers each
(not constrained to SU(3)).  A depends on U through the forward hop
-kappa eta_+ (1 - g_mu) U_mu(x) psi(x + mu) and on conj(U) through the backward
hop -kappa eta_- (1 + g_mu) U_mu(x)^dagger psi(x) arriving at x + mu.  Hence
    G_mu(x)_ab    = dT/dU_ab
                  = kappa eta_+(x,mu) sum_v sum_{s,s'} conj(y(x)_{s,a}) (1 - g_mu)_{s s'} x(x+mu)_{s',b}
    Gbar_mu(x)_ab = dT/d conj(U_ab)
                  = kappa eta_+(x,mu) sum_v sum_{s,s'} conj(y(x+mu)_{s,b}) (1 + g_mu)_{s s'} x(x)_{s',a}
(eta_-(x + mu, mu) = eta_+(x, mu)).  For real parameters:
    dT/dRe U_ab = G + Gbar,   dT/dIm U_ab = i (G - Gbar).
"""
import numpy as np

from . import operators as ops
from .lattice import displace_T
from .probes import probe


def _probe_pairs(op, col, m, seed, n_sets, kind, mu, p, tol, dilute=True):
    """Yield (v, x, y) for every probe: x = A^{-1} v, y = A^{-dagger} P^T v."""
    comps = range(op.dof) if dilute else [None]
    for s in range(n_sets):
        for c in range(m):
            for a in comps:
                v = probe(col, c, seed, s, kind, op.dof, a)
                if not np.any(v):
                    continue
                x, _, _ = op.solve(v, tol)
                y, _, _ = op.solve_dagger(displace_T(v, op.dims, mu, p), tol)
                yield v, x, y


def grad_m2(op, col, m, seed, n_sets, kind, mu, p, tol):
    """dT/dm^2 summed over all probes of all sets (Laplacian)."""
    g = 0.0
    for _, x, y in _probe_pairs(op, col, m, seed, n_sets, kind, mu, p, tol):
        g -= np.vdot(y, x)
    return g


def grad_kappa(op, col, m, seed, n_sets, kind, mu, p, tol, dilute=True):
    """dT/dkappa summed over all probes (Wilson)."""
    g = 0.0
    for _, x, y in _probe_pairs(op, col, m, seed, n_sets, kind, mu, p, tol, dilute):
        g += np.vdot(y, op.hop(x))
    return g


def grad_links(op, col, m, seed, n_sets, kind, mu, p, tol, dilute=True):
    """(dT/dkappa, G, Gbar) with G, Gbar of shape [N, 4, 3, 3] (Wilson)."""
    g, _ = ops.gammas()
    I4 = np.eye(4, dtype=np.complex128)
    fwd, _ = ops.neighbour_tables(op.dims)
    ep, _ = ops.boundary_signs(op.dims, op.ap)
    N = op.U.shape[0]
    G = np.zeros((N, 4, 3, 3), dtype=np.complex128)
    Gb = np.zeros((N, 4, 3, 3), dtype=np.complex128)
    dk = 0.0
    for _, x, y in _probe_pairs(op, col, m, seed, n_sets, kind, mu, p, tol, dilute):
        dk += np.vdot(y, op.hop(x))
        X = x.reshape(N, 4, 3)
        Y = y.reshape(N, 4, 3)
        for nu in range(4):
            Xf = X[fwd[nu]]
            Yf = Y[fwd[nu]]
            w = op.kappa * ep[nu][:, None, None]
            # sum_{s,s'} conj(Y(x)_{s,a}) (1 - g)_{s s'} X(x+nu)_{s',b}
            G[:, nu] += w * np.einsum('nsa,st,ntb->nab', np.conj(Y), I4 - g[nu], Xf)
            # sum_{s,s'} conj(Y(x+nu)_{s,b}) (1 + g)_{s s'} X(x)_{s',a}
            Gb[:, nu] += w * np.einsum('nsb,st,nta->nab', np.conj(Yf), I4 + g[nu], X)
    return dk, G, Gb
