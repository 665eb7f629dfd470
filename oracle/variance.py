"""Exact variance of the probed estimator on tiny lattices.

Eq. (2), Sec. 1: for real symmetric B and Z2 noise, Var(z^T B z) =
2 (||B||_F^2 - sum_i B_ii^2).  P A^{-1} is not symmetric, so the general forms
are used (they reduce to Eq. (2) when B = B^T):

  Z2 noise:  Var = 1/2 sum_{i != j, same class} |B_ij + B_ji|^2
  Z4 noise:  Var = sum_{i != j, same class} |B_ij|^2

where i, j run over sites and "same class" means same colour: only those
pairs survive the Hadamard product with H H^T (Sec. 2.2).

With spin-colour dilution (Sec. 4.2) the noise value of a site is shared by
its `dof` components (Kronecker product with the identity), so the estimate
sum_a v_a^H B v_a only sees, for each pair of sites, the trace over components
of the dof x dof block: M_xy = sum_a B[(x,a), (y,a)].  The formulas above are
applied to M (for dof = 1, M = B).
"""
import numpy as np


def block_trace(B, dof):
    """M_xy = sum_a B[(x, a), (y, a)] for a site-major (N dof) x (N dof) matrix."""
    B = np.asarray(B)
    N = B.shape[0] // dof
    return np.einsum('xaya->xy', B.reshape(N, dof, N, dof))


def exact_variance(B, col, kind, dof=1):
    """Variance of one estimate sum_{c,a} v_{c,a}^H B v_{c,a}.

    B: dense (N dof) x (N dof) matrix P A^{-1} (site-major); col: colour of
    every site (all zeros for unprobed Hutchinson); kind 0 = Z2, 1 = Z4.
    """
    M = block_trace(B, dof)
    col = np.asarray(col)
    same = (col[:, None] == col[None, :]) & ~np.eye(M.shape[0], dtype=bool)
    if kind == 0:
        S = M + M.T
        return 0.5 * float(np.sum(np.abs(S[same]) ** 2))
    return float(np.sum(np.abs(M[same]) ** 2))
