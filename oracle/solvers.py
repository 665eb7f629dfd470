"""Textbook Krylov solvers in FP64 and a dense solve for tiny lattices.

The paper treats the solves A^{-1} z_j as a black box (Sec. 2.1: "the bulk of
the computation is spent on the iterative method"; Sec. 4.2 used multigrid).
CG (Saad, Iterative Methods for Sparse Linear Systems, Alg. 6.18) for the
symmetric positive definite Laplacian; BiCGStab (Saad, Alg. 7.7) for the
non-Hermitian Wilson-Dirac operator.  Both stop when the TRUE relative
residual ||b - A x|| / ||b|| is below `tol`: the recursive residual is used
to decide when to check, and the iteration restarts from x if the check fails.
Vectors are flattened numpy arrays (real or complex).
"""
import numpy as np


def _dot(a, b):
    return np.vdot(a, b)            # conj(a) . b


def cg(apply_A, b, tol=1e-12, maxit=100000):
    b = np.asarray(b)
    bn = np.sqrt(_dot(b, b).real)
    x = np.zeros_like(b)
    if bn == 0.0:
        return x, 0, 0.0
    its = 0
    while True:
        r = b - apply_A(x)
        if np.sqrt(_dot(r, r).real) <= tol * bn or its >= maxit:
            return x, its, float(np.sqrt(_dot(r, r).real) / bn)
        p = r.copy()
        rr = _dot(r, r).real
        while its < maxit:
            q = apply_A(p)
            alpha = rr / _dot(p, q).real
            x = x + alpha * p
            r = r - alpha * q
            rr_new = _dot(r, r).real
            its += 1
            if np.sqrt(rr_new) <= tol * bn:
                break
            p = r + (rr_new / rr) * p
            rr = rr_new


def bicgstab(apply_A, b, tol=1e-10, maxit=100000):
    b = np.asarray(b, dtype=np.complex128)
    bn = np.sqrt(_dot(b, b).real)
    x = np.zeros_like(b)
    if bn == 0.0:
        return x, 0, 0.0
    its = 0
    while True:
        r = b - apply_A(x)
        if np.sqrt(_dot(r, r).real) <= tol * bn or its >= maxit:
            return x, its, float(np.sqrt(_dot(r, r).real) / bn)
        r0 = r.copy()
        p = r.copy()
        rho = _dot(r0, r)
        while its < maxit:
            v = apply_A(p)
            alpha = rho / _dot(r0, v)
            s = r - alpha * v
            t = apply_A(s)
            tt = _dot(t, t).real
            omega = _dot(t, s) / tt if tt > 0 else 0.0
            x = x + alpha * p + omega * s
            r = s - omega * t
            its += 1
            if np.sqrt(_dot(r, r).real) <= tol * bn or omega == 0.0:
                break
            rho_new = _dot(r0, r)
            beta = (rho_new / rho) * (alpha / omega)
            p = r + beta * (p - omega * v)
            rho = rho_new


def dense_solve(A, b):
    """Dense LU solve (LAPACK via numpy) for tiny lattices."""
    return np.linalg.solve(A, b)
