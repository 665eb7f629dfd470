"""Deflation of the lowest singular triplets (Sec. 2.4), for the displaced
trace.  Test infrastructure only.

With U, V holding approximate left and right singular vectors of the smallest
singular values of A, Q = A V (U^H A V)^{-1} U^H is an oblique projector and
Eq. (6) splits the trace; with the displacement P in front,

    Tr(P A^{-1}) = Tr(P A^{-1} Q) + Tr(P A^{-1} (I - Q)).

The first part is the trace of a small matrix: A^{-1} Q = V M U^H with
M = (U^H A V)^{-1}, so Tr(P A^{-1} Q) = Tr(M U^H P V).  The second part is
estimated with the probes; for a probe v,

    v^H P A^{-1} (I - Q) v = v^H P A^{-1} v - (v^H P V) M (U^H v),

one solve (the same as without deflation) and a correction that needs only
the probe and the triplets.  The identity holds for any U, V with U^H A V
invertible; singular vectors make the second part's variance small.

Dense routines (small lattices): the triplets come from numpy's SVD, a library
routine used as one step.
"""
import numpy as np

from .lattice import displace
from .probes import probe


def dense_matrix(op):
    """The operator as a dense (N dof) x (N dof) matrix, column by column."""
    N = int(np.prod(op.dims))
    n = N * op.dof
    dt = np.complex128 if op.dof > 1 else np.float64
    A = np.zeros((n, n), dtype=dt)
    for j in range(n):
        e = np.zeros(n, dtype=dt)
        e[j] = 1.0
        A[:, j] = np.asarray(op.apply(e.reshape(N, op.dof) if op.dof > 1 else e)).reshape(-1)
    return A


def lowest_singular_triplets(A, n_ev):
    """(U, s, V): the n_ev smallest singular values of A, ascending, and their
    left / right singular vectors as columns (A V = U diag(s))."""
    Uf, sf, Vhf = np.linalg.svd(A)
    order = np.argsort(sf)[:n_ev]
    return Uf[:, order], sf[order], Vhf.conj().T[:, order]


def displacement_matrix(dims, mu, p, dof=1):
    """P as a dense permutation matrix: (P f)(x) = f(x + p e_mu)."""
    N = int(np.prod(dims))
    n = N * dof
    P = np.zeros((n, n))
    for j in range(n):
        e = np.zeros((N, dof))
        e.reshape(-1)[j] = 1.0
        P[:, j] = displace(e, dims, mu, p).reshape(-1)
    return P


def small_matrix(A_apply_V, U):
    """M = (U^H A V)^{-1}, from A V (columns) and U."""
    return np.linalg.inv(U.conj().T @ A_apply_V)


def deflated_part(U, V, M, dims, mu, p_list, dof=1):
    """Tr(M U^H P V) for every displacement of p_list."""
    out = np.zeros(len(p_list), dtype=np.complex128)
    N = int(np.prod(dims))
    for n, p in enumerate(p_list):
        PV = np.stack([displace(V[:, i].reshape(N, dof) if dof > 1 else V[:, i], dims, mu, p).reshape(-1)
                       for i in range(V.shape[1])], axis=1)
        out[n] = np.trace(M @ (U.conj().T @ PV))
    return out


def deflated_probed_estimates(op, col, m, seed, n_sets, kind, mu, p_list, tol, U, V, M, dilute=True, set0=0):
    """est[s, n] = sum_{c, a} [v^H P_n A^{-1} v - (v^H P_n V) M (U^H v)], v = v_{s,c,a}:
    the probed estimate of Tr(P_n A^{-1} (I - Q)) (Sec. 2.4 with Eqs. (4), (5))."""
    dims = op.dims
    N = int(np.prod(dims))
    comps = range(op.dof) if dilute else [None]
    est = np.zeros((n_sets, len(p_list)), dtype=np.complex128)
    for s in range(n_sets):
        for c in range(m):
            for a in comps:
                v = probe(col, c, seed, set0 + s, kind, op.dof, a)
                if not np.any(v):
                    continue
                x, _, _ = op.solve(v, tol)
                vf = np.asarray(v).reshape(-1)
                uv = U.conj().T @ vf
                for n, p in enumerate(p_list):
                    corr = 0.0
                    if V.shape[1]:
                        PV = np.stack([displace(V[:, i].reshape(N, op.dof) if op.dof > 1 else V[:, i], dims, mu,
                                                p).reshape(-1) for i in range(V.shape[1])], axis=1)
                        corr = (vf.conj() @ PV) @ (M @ uv)
                    est[s, n] += np.vdot(v, displace(x, dims, mu, p)) - corr
    return est


def lanczos_lowest(apply_h, n, n_ev, n_iter, seed=0, dtype=np.float64, block=8):
    """Lowest n_ev eigenpairs of a Hermitian operator given by its action:
    block Lanczos (a random block of `block` vectors, every new block
    orthogonalised twice against the whole basis, n_iter blocks at most),
    then Rayleigh-Ritz on the basis.  A block as large as the multiplicity of
    the wanted eigenvalues resolves degenerate ones (a single start vector
    sees one vector per distinct eigenvalue).  Returns (values ascending,
    vectors as columns).  A matrix-free route to the triplets for lattices
    where a dense decomposition is out of reach."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, block))
    if dtype == np.complex128:
        X = X + 1j * rng.standard_normal((n, block))
    Q, _ = np.linalg.qr(X)
    basis = [Q]
    for _ in range(n_iter - 1):
        W = np.stack([np.asarray(apply_h(Q[:, i])).reshape(-1) for i in range(Q.shape[1])], axis=1)
        B = np.concatenate(basis, axis=1)
        for _ in range(2):
            W = W - B @ (B.conj().T @ W)
        Q, R = np.linalg.qr(W)
        keep = np.abs(np.diag(R)) > 1e-10 * max(1.0, np.abs(np.diag(R)).max(initial=0.0))
        Q = Q[:, keep]
        if Q.shape[1] == 0 or sum(b.shape[1] for b in basis) >= n:
            break
        basis.append(Q)
    B = np.concatenate(basis, axis=1)
    AB = np.stack([np.asarray(apply_h(B[:, i])).reshape(-1) for i in range(B.shape[1])], axis=1)
    T = B.conj().T @ AB
    th, S = np.linalg.eigh(0.5 * (T + T.conj().T))
    return th[:n_ev], B @ S[:, :n_ev]


def wilson_triplets_from_gamma5(apply_a, gamma5, n, n_ev, n_iter, seed=0):
    """Singular triplets of a gamma5-Hermitian operator (A^H = g5 A g5): the
    right singular vectors are eigenvectors of A^H A = (g5 A)^2, the lowest
    from Lanczos; sigma = ||A v|| and u = A v / sigma.  Returns (U, s, V)."""
    apply_aha = lambda x: gamma5(apply_a(gamma5(apply_a(x))))
    th, V = lanczos_lowest(apply_aha, n, n_ev, n_iter, seed, np.complex128)
    AV = np.stack([np.asarray(apply_a(V[:, i])).reshape(-1) for i in range(V.shape[1])], axis=1)
    s = np.linalg.norm(AV, axis=0)
    return AV / s[None, :], s, V


def deflation_corrections(col, m, seed, n_sets, kind, dims, mu, p_list, U, V, M, dof=1, set0=0):
    """corr[s, n] = sum_{c, a} (v^H P_n V) M (U^H v) over the diluted probes
    v = v_{s,c,a}: the part of the deflated estimate that needs no solve."""
    N = int(np.prod(dims))
    corr = np.zeros((n_sets, len(p_list)), dtype=np.complex128)
    for s in range(n_sets):
        for c in range(m):
            for a in range(dof):
                v = probe(col, c, seed, set0 + s, kind, dof, a)
                if not np.any(v):
                    continue
                vf = np.asarray(v).reshape(-1)
                uv = U.conj().T @ vf
                for n, p in enumerate(p_list):
                    PV = np.stack([displace(V[:, i].reshape(N, dof) if dof > 1 else V[:, i], dims, mu, p)
                                   .reshape(-1) for i in range(V.shape[1])], axis=1)
                    corr[s, n] += (vf.conj() @ PV) @ (M @ uv)
    return corr
