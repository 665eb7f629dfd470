"""Trace estimators and their statistics.

Eq. (1): Hutchinson, Tr(M) ~ (1/s) sum_i z_i^T M z_i.  For complex probes the
transpose is read as the conjugate transpose (z^H M z).
Eqs. (4), (5): with a colouring of m colours and s noise vectors z0^(s), one
estimate per noise vector is
    T_s = sum_{c < m} sum_{a < dof} v_{s,c,a}^H  P  A^{-1}  v_{s,c,a},
i.e. one Hutchinson step on (P A^{-1}) (.) H H^T (Sec. 2.2).  The unprobed
Hutchinson estimator is the case m = 1 (every site colour 0).
Sec. 4.2: estimates are averaged over s; v(.) is the per-vector variance,
estimated by the sample variance; speedup over Hutchinson Eq. (15), over
classical probing Eq. (16), normalised relative error Eq. (17).
"""
import numpy as np

from . import operators as ops
from .lattice import displace
from .probes import probe
from .solvers import bicgstab, cg


class Laplacian:
    """Shifted scalar Laplacian, dof = 1 per site."""
    dof = 1

    def __init__(self, dims, m2):
        self.dims, self.m2 = list(dims), float(m2)

    def apply(self, x):
        return ops.laplacian_apply(np.asarray(x).reshape(-1), self.dims, self.m2).reshape(-1, 1)

    def solve(self, b, tol=1e-12, maxit=100000):
        f = lambda v: ops.laplacian_apply(v, self.dims, self.m2)
        x, its, rel = cg(f, np.asarray(b, dtype=np.float64).reshape(-1), tol, maxit)
        return x.reshape(-1, 1), its, rel

    apply_dagger = apply               # real symmetric
    solve_dagger = solve


class Wilson:
    """Wilson-Dirac operator, dof = 12 per site (component = 3 * spin + colour)."""
    dof = 12

    def __init__(self, dims, U, kappa, antiperiodic_t=True):
        self.dims, self.U, self.kappa, self.ap = list(dims), np.asarray(U), float(kappa), bool(antiperiodic_t)

    def _sp(self, x):
        return np.asarray(x, dtype=np.complex128).reshape(-1, 4, 3)

    def apply(self, x):
        return ops.wilson_apply(self._sp(x), self.U, self.kappa, self.dims, self.ap).reshape(-1, 12)

    def apply_dagger(self, x):
        return ops.wilson_apply_dagger(self._sp(x), self.U, self.kappa, self.dims, self.ap).reshape(-1, 12)

    def hop(self, x):
        return ops.wilson_hop(self._sp(x), self.U, self.dims, self.ap).reshape(-1, 12)

    def solve(self, b, tol=1e-10, maxit=100000):
        f = lambda v: self.apply(v).reshape(-1)
        x, its, rel = bicgstab(f, np.asarray(b, dtype=np.complex128).reshape(-1), tol, maxit)
        return x.reshape(-1, 12), its, rel

    def solve_dagger(self, b, tol=1e-10, maxit=100000):
        f = lambda v: self.apply_dagger(v).reshape(-1)
        x, its, rel = bicgstab(f, np.asarray(b, dtype=np.complex128).reshape(-1), tol, maxit)
        return x.reshape(-1, 12), its, rel


def probed_estimates(op, col, m, seed, n_sets, kind, mu, p_list, tol, dilute=True, set0=0):
    """est[s, n] = sum_{c, a} v_{s,c,a}^H P_{p_n} A^{-1} v_{s,c,a}  (Eqs. (1), (5)).

    `dilute`: True -> one probe per component a (Kronecker product with the
    identity, Sec. 4.2); False -> one probe per colour with independent noise
    in every component.  The scalar Laplacian has dof = 1 either way.
    Returns a complex128 array [n_sets, n_p].
    """
    dims = op.dims
    comps = range(op.dof) if dilute else [None]
    est = np.zeros((n_sets, len(p_list)), dtype=np.complex128)
    for s in range(n_sets):
        for c in range(m):
            for a in comps:
                v = probe(col, c, seed, set0 + s, kind, op.dof, a)
                if not np.any(v):
                    continue
                x, _, _ = op.solve(v, tol)
                for n, p in enumerate(p_list):
                    est[s, n] += np.vdot(v, displace(x, dims, mu, p))
    return est


def hutchinson_estimates(op, seed, n_sets, kind, mu, p_list, tol, dilute=True):
    """Unprobed Hutchinson: the probed estimator with a single colour."""
    N = 1
    for D in op.dims:
        N *= D
    return probed_estimates(op, np.zeros(N, dtype=np.int32), 1, seed, n_sets, kind, mu, p_list, tol, dilute)


def mean(est):
    return np.mean(est, axis=0)


def sample_variance(est):
    """Per-vector variance with the s - 1 denominator; |.|^2 for complex."""
    est = np.asarray(est)
    mu = np.mean(est, axis=0)
    return np.sum(np.abs(est - mu) ** 2, axis=0) / (est.shape[0] - 1)


def sigma_mean(est):
    return np.sqrt(sample_variance(est) / np.asarray(est).shape[0])


def speedup_over_hutchinson(var_h, var_p, m):
    """Eq. (15): v(P A^{-1}) / (m v((P A^{-1}) (.) H H^T))."""
    return var_h / (m * var_p)


def speedup_over_cp(var_cp, m0, var_p, mp):
    """Eq. (16): v((P_p A^{-1}) (.) H_0 H_0^T) m_0 / (v((P_p A^{-1}) (.) H_p H_p^T) m_p)."""
    return (var_cp * m0) / (var_p * mp)


def normalised_relative_error(var, m_p, M, trace):
    """Eq. (17): sqrt(v m_p / M) / tr."""
    return np.sqrt(var * m_p / M) / trace


def time_to_sigma(time_per_set, var, sigma):
    """Time to reach a target standard deviation of the mean: the number of
    noise sets needed, ceil(v / sigma^2), times the time per set."""
    return time_per_set * np.ceil(var / sigma ** 2)
