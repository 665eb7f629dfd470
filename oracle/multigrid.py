"""Two-level aggregation multigrid as a preconditioner (test infrastructure
only; the solver-fidelity row after deflation: the paper's solves use an
adaptive multigrid library, Sec. 4.2, whose method it does not describe).

The textbook construction, for a lattice cut into blocks of b^4 sites:

* aggregates: the sites of one block (for Wilson, and one chirality: spins
  (0, 1) or (2, 3), so that the prolongator commutes with g5);
* prolongator P (columns orthonormal): for the Laplacian the normalised
  indicator of each block; adaptively, the restriction to each aggregate of
  a few near-null vectors (random vectors after smoothing iterations on
  A x = 0), orthonormalised aggregate by aggregate;
* coarse operator A_c = P^H A P (Galerkin), solved exactly;
* two-grid cycle M: nu damped-Jacobi sweeps, the coarse correction
  x += P A_c^{-1} P^H r, nu more sweeps; every step is linear, so M is a
  fixed linear preconditioner and right-preconditioned GMRES applies.

Written for small lattices (dense coarse operator); every function takes the
fine operator as a matrix-free apply.
"""
import numpy as np

from .lattice import coords, volume


def block_index(dims, b):
    """Aggregate (block) number of every site for blocks of b^4 sites, blocks
    in storage order of the coarse lattice."""
    if any(D % b for D in dims):
        raise ValueError("the block side must divide every lattice side")
    xs = coords(dims)
    cd = [D // b for D in dims]
    bx = xs // b
    return bx[:, 0] + cd[0] * (bx[:, 1] + cd[1] * (bx[:, 2] + cd[2] * bx[:, 3])), cd


def prolongator_constant(dims, b):
    """P [N, n_blocks]: the normalised indicator of each block."""
    agg, cd = block_index(dims, b)
    N, nb = volume(dims), int(np.prod(cd))
    P = np.zeros((N, nb))
    P[np.arange(N), agg] = 1.0 / np.sqrt(b ** 4)
    return P


def jacobi_sweeps(apply_a, diag, b, x, nu, omega):
    """nu damped-Jacobi sweeps x <- x + omega D^{-1} (b - A x)."""
    for _ in range(nu):
        x = x + omega * (b - apply_a(x)) / diag
    return x


def near_null_vectors(apply_a, diag, n, n_vec, sweeps, seed, dtype=np.float64, omega=0.8):
    """n_vec random vectors relaxed by `sweeps` damped-Jacobi sweeps on A x = 0:
    the smooth error the smoother leaves, which the coarse space must hold."""
    rng = np.random.default_rng(seed)
    V = rng.standard_normal((n, n_vec))
    if dtype == np.complex128:
        V = V + 1j * rng.standard_normal((n, n_vec))
    zero = np.zeros(n, dtype=V.dtype)
    return np.stack([jacobi_sweeps(apply_a, diag, zero, V[:, k], sweeps, omega) for k in range(n_vec)], axis=1)


def prolongator_adaptive(V, dims, b, dof):
    """P [N dof, n_agg n_vec]: per aggregate (block x chirality half for
    dof = 12, block for dof = 1) the restriction of the columns of V,
    orthonormalised by a QR of that restriction."""
    agg, cd = block_index(dims, b)
    N, nb = volume(dims), int(np.prod(cd))
    n_vec = V.shape[1]
    halves = 2 if dof == 12 else 1
    P = np.zeros((N * dof, nb * halves * n_vec), dtype=V.dtype)
    comp = np.arange(dof)
    for blk in range(nb):
        sites = np.nonzero(agg == blk)[0]
        for h in range(halves):
            cs = comp if dof == 1 else comp[(comp // 6) == h]              # spins (0, 1) or (2, 3)
            rows = (sites[:, None] * dof + cs[None, :]).reshape(-1)
            Q, _ = np.linalg.qr(V[rows, :])
            col0 = (blk * halves + h) * n_vec
            P[rows, col0:col0 + n_vec] = Q
    return P


def coarse_operator(apply_a, P):
    """A_c = P^H A P, column by column from the matrix-free apply."""
    AP = np.stack([np.asarray(apply_a(P[:, j])).reshape(-1) for j in range(P.shape[1])], axis=1)
    return P.conj().T @ AP


class TwoGrid:
    """The two-grid cycle M (a linear map r -> M r, from x = 0)."""

    def __init__(self, apply_a, diag, P, nu=2, omega=0.8):
        self.apply_a, self.diag, self.P, self.nu, self.omega = apply_a, diag, P, nu, omega
        self.Ac = coarse_operator(apply_a, P)
        self.Ac_inv = np.linalg.inv(self.Ac)

    def __call__(self, r):
        x = jacobi_sweeps(self.apply_a, self.diag, r, np.zeros_like(r), self.nu, self.omega)
        x = x + self.P @ (self.Ac_inv @ (self.P.conj().T @ (r - self.apply_a(x))))
        return jacobi_sweeps(self.apply_a, self.diag, r, x, self.nu, self.omega)


def gmres(apply_a, b, tol=1e-10, restart=30, maxit=2000, precond=None):
    """Right-preconditioned restarted GMRES (Saad, Iterative Methods for Sparse
    Linear Systems, Alg. 6.9 with right preconditioning): solves A M y = b,
    x = M y.  Returns (x, iterations, relative residual)."""
    M = precond if precond is not None else (lambda r: r)
    b = np.asarray(b)
    dt = np.result_type(b.dtype, np.float64)
    x = np.zeros(b.shape, dtype=dt)
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return x, 0, 0.0
    its = 0
    while its < maxit:
        r = b - apply_a(x)
        beta = np.linalg.norm(r)
        if beta <= tol * bn:
            break
        V = [r / beta]
        Z = []
        H = np.zeros((restart + 1, restart), dtype=dt)
        g = np.zeros(restart + 1, dtype=dt)
        g[0] = beta
        k_used = 0
        for k in range(restart):
            z = M(V[k])
            w = apply_a(z)
            Z.append(z)
            for i in range(k + 1):                      # modified Gram-Schmidt
                H[i, k] = np.vdot(V[i], w)
                w = w - H[i, k] * V[i]
            H[k + 1, k] = np.linalg.norm(w)
            its += 1
            k_used = k + 1
            y, *_ = np.linalg.lstsq(H[:k + 2, :k + 1], g[:k + 2], rcond=None)
            res = np.linalg.norm(g[:k + 2] - H[:k + 2, :k + 1] @ y)
            if res <= tol * bn or H[k + 1, k] == 0.0 or its >= maxit:
                break
            V.append(w / H[k + 1, k])
        y, *_ = np.linalg.lstsq(H[:k_used + 1, :k_used], g[:k_used + 1], rcond=None)
        x = x + sum(y[i] * Z[i] for i in range(k_used))
    r = b - apply_a(x)
    return x, its, float(np.linalg.norm(r) / bn)
