"""Pins for the oracle's RNG, operators, solvers, estimator, variance and gradient."""
import itertools

import numpy as np
import pytest

from conftest import read_golden
from oracle import estimator as E
from oracle import gradient as Gr
from oracle import lattice as L
from oracle import operators as ops
from oracle import rng
from oracle import variance as V
from oracle.colouring import greedy_colour
from oracle.probes import probe
from paper_2106_01275_gb300 import inputs


# ---------------------------------------------------------------- RNG (Sec. 1)
def test_splitmix64_reference_outputs():
    want = [int(r[0], 16) for r in read_golden("splitmix64.txt")]
    got = [rng.mix64_int(n * rng.GAMMA) for n in (1, 2, 3)]
    assert got == want
    # the numpy path agrees with the exact-integer path
    z = rng.mix64(np.array([n * rng.GAMMA % 2 ** 64 for n in (1, 2, 3)], dtype=np.uint64))
    assert [int(v) for v in z] == want


def test_noise_distribution():
    N = 200000
    z2 = rng.z2(7, 3, N)
    assert set(np.unique(z2).tolist()) == {-1.0, 1.0}
    assert abs(z2.mean()) < 5 / np.sqrt(N)
    z4 = rng.z4(7, 3, N)
    counts = np.array([np.sum(z4 == v) for v in (1, 1j, -1, -1j)])
    chi2 = np.sum((counts - N / 4) ** 2 / (N / 4))
    assert counts.sum() == N and chi2 < 16.3          # 3 dof, p ~ 0.001
    assert not np.array_equal(rng.z2(7, 3, 64), rng.z2(7, 4, 64))
    assert not np.array_equal(rng.z2(7, 3, 64), rng.z2(8, 3, 64))


def test_probe_partition_of_unity():
    """Sum over colours of the probes of one set is z0 (x) e_a (Eqs. (4), (5))."""
    dims = [4, 4, 4, 4]
    col, m = greedy_colour(dims, 0, [1], 2, 0)
    for kind, dof, a in ((0, 1, 0), (1, 12, 5)):
        tot = sum(probe(col, c, 11, 2, kind, dof, a) for c in range(m))
        z0 = rng.noise(11, 2, 256, kind)
        want = np.zeros((256, dof), dtype=tot.dtype)
        want[:, a] = z0
        assert np.array_equal(tot, want)


# ---------------------------------------------------------------- operators
def test_gamma_algebra():
    g, g5 = ops.gammas()
    I4 = np.eye(4)
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T)
        for nu in range(4):
            assert np.allclose(g[mu] @ g[nu] + g[nu] @ g[mu], 2 * (mu == nu) * I4)
    assert np.allclose(g5, np.diag([1, 1, -1, -1]))


def dense_laplacian_loops(dims, m2):
    """Dense matrix written site by site (independent of the apply)."""
    N = L.volume(dims)
    xs = L.coords(dims)
    A = np.zeros((N, N))
    for i in range(N):
        A[i, i] += 2 * len(dims) + m2
        for mu in range(len(dims)):
            for s in (+1, -1):
                y = xs[i].copy()
                y[mu] = (y[mu] + s) % dims[mu]
                A[i, int(L.index_of(y, dims))] -= 1.0
    return A


def dense_wilson_loops(dims, U, kappa):
    """Dense Wilson matrix written block by block (independent of the apply)."""
    g, _ = ops.gammas()
    N = L.volume(dims)
    xs = L.coords(dims)
    A = np.eye(12 * N, dtype=np.complex128)
    I4 = np.eye(4)
    for i in range(N):
        for mu in range(4):
            yf = xs[i].copy(); yf[mu] += 1
            yb = xs[i].copy(); yb[mu] -= 1
            sf = -1.0 if (mu == 3 and yf[3] == dims[3]) else 1.0
            sb = -1.0 if (mu == 3 and yb[3] < 0) else 1.0
            jf = int(L.index_of(yf, dims)); jb = int(L.index_of(yb, dims))
            A[12 * i:12 * i + 12, 12 * jf:12 * jf + 12] -= kappa * sf * np.kron(I4 - g[mu], U[i, mu])
            A[12 * i:12 * i + 12, 12 * jb:12 * jb + 12] -= kappa * sb * np.kron(I4 + g[mu], U[jb, mu].conj().T)
    return A


def test_laplacian_apply_matches_dense():
    dims, m2 = [3, 4, 2, 5], 0.3
    A = dense_laplacian_loops(dims, m2)
    f = np.random.default_rng(0).standard_normal(L.volume(dims))
    assert np.allclose(ops.laplacian_apply(f, dims, m2), A @ f, atol=1e-13)


def test_wilson_apply_matches_dense_and_gamma5_hermiticity():
    dims = [2, 2, 2, 4]
    U = inputs.gauge_links(dims, 5)
    A = dense_wilson_loops(dims, U, 0.13)
    r = np.random.default_rng(1)
    psi = r.standard_normal((32, 4, 3)) + 1j * r.standard_normal((32, 4, 3))
    assert np.allclose(ops.wilson_apply(psi, U, 0.13, dims).reshape(-1), A @ psi.reshape(-1), atol=1e-13)
    assert np.allclose(ops.wilson_apply_dagger(psi, U, 0.13, dims).reshape(-1),
                       A.conj().T @ psi.reshape(-1), atol=1e-13)
    # gamma5 A gamma5 = A^dagger
    lhs = ops.gamma5_apply(ops.wilson_apply(ops.gamma5_apply(psi), U, 0.13, dims))
    assert np.allclose(lhs, ops.wilson_apply_dagger(psi, U, 0.13, dims), atol=1e-13)


def test_links_are_su3():
    U = inputs.gauge_links([2, 2, 2, 2], 3)
    UU = np.einsum('...ab,...cb->...ac', U, U.conj())
    assert np.allclose(UU, np.eye(3), atol=1e-13)
    assert np.allclose(np.linalg.det(U), 1.0, atol=1e-13)


def lattice_momenta(dims, antiperiodic_t=False):
    ks = []
    for mu, D in enumerate(dims):
        n = np.arange(D)
        ks.append(2 * np.pi * (n + (0.5 if (antiperiodic_t and mu == 3) else 0.0)) / D)
    return np.stack(np.meshgrid(*ks, indexing='ij'), -1).reshape(-1, len(dims))


def free_laplacian_trace(dims, m2, mu, p, power=1):
    """Tr(P_p A^{-power}) = sum_k cos(k_mu p) / lambda(k)^power (Fourier)."""
    K = lattice_momenta(dims)
    lam = m2 + 4 * np.sum(np.sin(K / 2) ** 2, axis=1)
    return np.sum(np.cos(K[:, mu] * p) / lam ** power)


def free_wilson_trace(dims, kappa, mu, p):
    """Tr(P_p A^{-1}) for U = 1, antiperiodic t: 12 sum_k cos(k_mu p) a / (a^2 + 4 kappa^2 sum sin^2 k)."""
    K = lattice_momenta(dims, antiperiodic_t=True)
    a = 1 - 2 * kappa * np.sum(np.cos(K), axis=1)
    den = a ** 2 + 4 * kappa ** 2 * np.sum(np.sin(K) ** 2, axis=1)
    return 12 * np.sum(np.cos(K[:, mu] * p) * a / den)


def dense_inverse_of_apply(apply, n, dtype=np.float64):
    cols = [apply(np.eye(n, dtype=dtype)[i]) for i in range(n)]
    return np.linalg.inv(np.stack(cols, axis=1))


def test_free_laplacian_trace_closed_form():
    dims, m2 = [4, 4, 4, 4], 0.1
    Ai = dense_inverse_of_apply(lambda f: ops.laplacian_apply(f, dims, m2), 256)
    for p in (0, 1, 2):
        perm = L.shift_map(dims, 0, p)
        assert abs(np.trace(Ai[perm, :]) - free_laplacian_trace(dims, m2, 0, p)) < 1e-11
    assert abs(free_laplacian_trace(dims, m2, 0, 1) - 15.5360518473118) < 1e-10


def test_free_wilson_trace_closed_form():
    dims, kappa = [4, 4, 4, 4], 0.12
    U = inputs.unit_links(dims)
    A = dense_wilson_loops(dims, U, kappa)
    f = np.random.default_rng(4).standard_normal(12 * 256) + 0j
    assert np.allclose(A @ f, ops.wilson_apply(f.reshape(-1, 4, 3), U, kappa, dims).reshape(-1))
    Ai = np.linalg.inv(A)
    for p in (0, 1, 2):
        perm = L.shift_map(dims, 2, p)
        idx = (12 * perm[:, None] + np.arange(12)[None, :]).reshape(-1)
        tr = np.trace(Ai[idx, :])
        assert abs(tr - free_wilson_trace(dims, kappa, 2, p)) < 1e-9 * abs(tr)


def test_gauge_invariance_p0_only():
    """Tr(A^{-1}) is invariant under U_mu(x) -> g(x) U_mu(x) g(x+mu)^dagger; a
    displaced trace is not (the displacement carries no parallel transport)."""
    dims, kappa = [2, 2, 2, 4], 0.12
    U = inputs.gauge_links(dims, 9)
    g = inputs.random_su3(32, 10)
    fwd, _ = ops.neighbour_tables(dims)
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[:, mu] = np.einsum('nab,nbc,ndc->nad', g, U[:, mu], g[fwd[mu]].conj())
    def tr(Ul, p):
        app = lambda f: ops.wilson_apply(f.reshape(-1, 4, 3), Ul, kappa, dims).reshape(-1)
        Ai = dense_inverse_of_apply(app, 384, np.complex128)
        perm = L.shift_map(dims, 2, p)
        idx = (12 * perm[:, None] + np.arange(12)[None, :]).reshape(-1)
        return np.trace(Ai[idx, :])
    assert abs(tr(U, 0) - tr(Ug, 0)) < 1e-10 * abs(tr(U, 0))
    assert abs(tr(U, 1) - tr(Ug, 1)) > 1e-6


# ---------------------------------------------------------------- solvers
def test_cg_and_bicgstab_match_dense():
    dims = [4, 4, 4, 4]
    lap = E.Laplacian(dims, 0.1)
    b = np.random.default_rng(2).standard_normal((256, 1))
    x, its, rel = lap.solve(b, 1e-12)
    A = dense_laplacian_loops(dims, 0.1)
    assert rel < 1e-12 and np.allclose(x[:, 0], np.linalg.solve(A, b[:, 0]), rtol=0, atol=1e-10)
    dims = [2, 2, 2, 4]
    U = inputs.gauge_links(dims, 4)
    w = E.Wilson(dims, U, 0.12)
    r = np.random.default_rng(3)
    b = r.standard_normal((32, 12)) + 1j * r.standard_normal((32, 12))
    x, its, rel = w.solve(b, 1e-10)
    A = dense_wilson_loops(dims, U, 0.12)
    assert rel < 1e-10
    assert np.allclose(x.reshape(-1), np.linalg.solve(A, b.reshape(-1)), atol=1e-8)
    y, _, rel = w.solve_dagger(b, 1e-10)
    assert rel < 1e-10 and np.allclose(y.reshape(-1), np.linalg.solve(A.conj().T, b.reshape(-1)), atol=1e-8)


# ---------------------------------------------------------------- estimator and variance
def test_all_distinct_colours_give_exact_trace():
    """With every site its own colour the probed estimate is exact (Eq. (4))."""
    dims, m2 = [4, 4, 4, 4], 0.1
    lap = E.Laplacian(dims, m2)
    col = np.arange(256, dtype=np.int32)
    est = E.probed_estimates(lap, col, 256, 0, 1, 0, 0, [0, 1, 2], 1e-12)
    for n, p in enumerate((0, 1, 2)):
        assert abs(est[0, n] - free_laplacian_trace(dims, m2, 0, p)) < 1e-9


def test_estimator_matches_dense_quadratures():
    """Eq. (5): the CG-based estimate equals sum v^T (P A^{-1}) v from the dense inverse."""
    dims, m2, p = [4, 4, 4, 4], 0.1, 1
    lap = E.Laplacian(dims, m2)
    col, m = greedy_colour(dims, 0, [p], 1, 0)
    est = E.probed_estimates(lap, col, m, 0, 3, 0, 0, [p], 1e-12)
    B = np.linalg.inv(dense_laplacian_loops(dims, m2))[L.shift_map(dims, 0, p), :]
    for s in range(3):
        z0 = rng.z2(0, s, 256)
        want = sum((z0 * (col == c)) @ B @ (z0 * (col == c)) for c in range(m))
        assert abs(est[s, 0] - want) < 1e-9


def brute_force_variance(B, cls, kind, N):
    """Variance of sum_classes v^H B v over ALL 2^N (Z2) noise vectors."""
    signs = np.array(list(itertools.product([1.0, -1.0], repeat=N)))  # [2^N, N]
    T = np.zeros(signs.shape[0], dtype=np.complex128)
    for c in np.unique(cls):
        Z = signs * (cls == c)[None, :]
        T += np.einsum('si,ij,sj->s', Z, B, Z)
    return float(np.mean(np.abs(T - T.mean()) ** 2))


def test_exact_variance_vs_enumeration_1d_ring():
    n, p = 16, 3
    A = (2.05 * np.eye(n) - np.roll(np.eye(n), 1, 1) - np.roll(np.eye(n), -1, 1))
    B = np.linalg.inv(A)[L.shift_map([n], 0, p), :]
    for k in (0, 1, 2):
        col, m = greedy_colour([n], 0, [p], k, 0) if k else (np.zeros(n, np.int32), 1)
        assert abs(V.exact_variance(B, col, 0) - brute_force_variance(B, col, 0, n)) < 1e-12
    # Eq. (2) for a symmetric matrix (p = 0, no probing)
    B0 = np.linalg.inv(A)
    assert abs(V.exact_variance(B0, np.zeros(n, int), 0)
               - 2 * (np.sum(B0 ** 2) - np.sum(np.diag(B0) ** 2))) < 1e-12


def test_exact_variance_vs_enumeration_2to4_lattice():
    dims = [2, 2, 2, 2]
    A = dense_laplacian_loops(dims, 0.2)
    B = np.linalg.inv(A)[L.shift_map(dims, 0, 1), :]
    col, m = greedy_colour(dims, 0, [1], 1, 0)
    assert abs(V.exact_variance(B, col, 0) - brute_force_variance(B, col, 0, 16)) < 1e-12


def test_probing_reduces_the_exact_variance():
    """4^4, m^2 = 0.1, p = 1 along dim 0: distance-1 and -2 colourings take 4
    and 8 colours, and each step of probing lowers the exact Z2 variance
    (Eq. (2) in its general form, itself pinned by brute force above)."""
    dims, m2 = [4, 4, 4, 4], 0.1
    B = np.linalg.inv(dense_laplacian_loops(dims, m2))[L.shift_map(dims, 0, 1), :]
    vh = V.exact_variance(B, np.zeros(256, int), 0)
    c1, m1 = greedy_colour(dims, 0, [1], 1, 0)
    c2, m2_ = greedy_colour(dims, 0, [1], 2, 0)
    v1 = V.exact_variance(B, c1, 0)
    v2 = V.exact_variance(B, c2, 0)
    assert (m1, m2_) == (4, 8)
    assert vh > 2 * v1 > 0 and v1 > 1.5 * v2 > 0


def test_unbiased_and_sample_variance():
    """Mean over many noise sets is within 5 sigma of the exact trace, and the
    sample variance approaches the exact variance (Sec. 2.2, Eq. (2))."""
    dims, m2, p = [4, 4, 4, 4], 0.1, 1
    B = np.linalg.inv(dense_laplacian_loops(dims, m2))[L.shift_map(dims, 0, p), :]
    col, m = greedy_colour(dims, 0, [p], 1, 0)
    S = 4000
    T = np.zeros(S)
    for s in range(S):
        z0 = rng.z2(123, s, 256)
        T[s] = sum((z0 * (col == c)) @ B @ (z0 * (col == c)) for c in range(m))
    exact_var = V.exact_variance(B, col, 0)
    assert abs(T.mean() - np.trace(B)) < 5 * np.sqrt(exact_var / S)
    sv = E.sample_variance(T[:, None])[0]
    assert abs(sv - exact_var) < 0.15 * exact_var


def test_z4_variance_formula():
    """Z4 noise shared by the 12 components of a site (Sec. 4.2 dilution):
    the sample variance of many estimates matches the exact formula."""
    dims = [2, 2, 2, 4]
    U = inputs.gauge_links(dims, 6)
    Bf = np.linalg.inv(dense_wilson_loops(dims, U, 0.12))
    perm = L.shift_map(dims, 2, 1)
    idx = (12 * perm[:, None] + np.arange(12)[None, :]).reshape(-1)
    B = Bf[idx, :]
    col = np.zeros(32, np.int32)
    S = 3000
    T = np.zeros(S, dtype=np.complex128)
    for s in range(S):
        z = rng.z4(5, s, 32)
        for a in range(12):
            v = np.zeros(384, np.complex128)
            v[a::12] = z
            T[s] += np.vdot(v, B @ v)
    ex = V.exact_variance(B, col, 1, dof=12)
    assert abs(np.mean(np.abs(T - T.mean()) ** 2) - ex) < 0.1 * ex


def test_table6_speedup_arithmetic():
    """Eq. (15) reproduces the printed speedups of Table 6 from its printed variances."""
    for r in read_golden("table6_speedup.txt"):
        p, k = int(r[0]), int(r[1])
        s = E.speedup_over_hutchinson(float(r[3]), float(r[5]), int(r[4]))
        assert abs(s - float(r[6])) < 0.005 * float(r[6]), (p, k)


def test_eq16_eq17_mean_what_sec43_says_at_equal_work():
    """Eqs. (16) and (17) against what they measure (Sec. 4.3): both compare
    estimators at the same number of solves.  4^4 Laplacian, m^2 = 0.1,
    p = 1 along dim 0: classical probing with the (0, 1) colouring (H_0,
    m_0 colours) and displaced probing with the (1, 1) colouring (H_p, m_p).
    Independent Z2 sets are drawn, each one's estimate z^T (B (.) H H^T) z
    formed from the dense B = P A^{-1}, and the sets are averaged in groups
    that cost the same budget of solves.  Eq. (17) must equal the observed
    standard deviation of a budget-M mean over |tr|, and Eq. (16) the ratio of
    the observed variances of the classical and displaced means at equal
    budget.  A missing square root, a transposed m_0 / m_p or m_p / M, or a
    missing trace each miss by far more than the sampling error."""
    from oracle import deflation as D
    dims, m2, mu, p = [4, 4, 4, 4], 0.1, 0, 1
    B = D.displacement_matrix(dims, mu, p) @ np.linalg.inv(D.dense_matrix(E.Laplacian(dims, m2)))
    tr = float(np.trace(B))
    c0, m0 = greedy_colour(dims, mu, [0], 1, 0)
    cp, mp = greedy_colour(dims, mu, [p], 1, 0)
    assert m0 != mp
    M = int(np.lcm(m0, mp)) * 4                        # the common budget of solves
    rng = np.random.default_rng(2021)
    trials = 3000

    def budget_means(col, m):
        Bm = B * (col[:, None] == col[None, :])
        k = M // m                                      # sets that the budget buys
        Z = rng.choice([-1.0, 1.0], size=(trials * k, B.shape[0]))
        T = np.einsum('ni,ni->n', Z @ Bm.T, Z)          # one estimate per set
        return T.reshape(trials, k).mean(axis=1), float(np.var(T, ddof=1))

    mean0, v0 = budget_means(c0, m0)
    meanp, vp = budget_means(cp, mp)
    # the per-set variances are the exact ones (Eq. (2) general form, pinned by enumeration)
    assert abs(v0 / V.exact_variance(B, c0, 0) - 1) < 0.05
    assert abs(vp / V.exact_variance(B, cp, 0) - 1) < 0.05
    nre_p = E.normalised_relative_error(vp, mp, M, tr)
    assert abs(np.std(meanp, ddof=1) / abs(tr) / nre_p - 1) < 0.06
    nre_0 = E.normalised_relative_error(v0, m0, M, tr)
    assert abs(np.std(mean0, ddof=1) / abs(tr) / nre_0 - 1) < 0.06
    s_cp = E.speedup_over_cp(v0, m0, vp, mp)
    assert abs(np.var(mean0, ddof=1) / np.var(meanp, ddof=1) / s_cp - 1) < 0.12
    assert s_cp > 1.0                                   # displaced probing wins for p = 1


def test_eq16_against_eq15_on_table6():
    """Eq. (16) is the ratio of two Eq. (15) speedups over the same Hutchinson
    variance: for every p of Table 6 and every pair of its colourings, with the
    printed variances and colour counts (Eq. (15) itself reproduces Table 6's
    printed speedups, above)."""
    rows = [r for r in read_golden("table6_speedup.txt")]
    by_p = {}
    for r in rows:
        by_p.setdefault(int(r[0]), []).append((float(r[3]), int(r[4]), float(r[5])))
    n = 0
    for p, rs in by_p.items():
        for (vh, ma, va) in rs:
            for (_, mb, vb) in rs:
                want = E.speedup_over_hutchinson(vh, vb, mb) / E.speedup_over_hutchinson(vh, va, ma)
                assert E.speedup_over_cp(va, ma, vb, mb) == pytest.approx(want, rel=1e-12)
                n += 1
    assert n > 500


# ---------------------------------------------------------------- gradient
def _estimate(op, col, m, seed, n_sets, kind, mu, p, tol, dilute=True):
    return E.probed_estimates(op, col, m, seed, n_sets, kind, mu, [p], tol, dilute).sum()


def test_laplacian_grad_m2_fd_and_closed_form():
    dims, m2, p = [4, 4, 4, 4], 0.1, 1
    col, m = greedy_colour(dims, 0, [p], 2, 0)
    g = Gr.grad_m2(E.Laplacian(dims, m2), col, m, 0, 2, 0, 0, p, 1e-13)
    h = 1e-5
    fd = (_estimate(E.Laplacian(dims, m2 + h), col, m, 0, 2, 0, 0, p, 1e-13)
          - _estimate(E.Laplacian(dims, m2 - h), col, m, 0, 2, 0, 0, p, 1e-13)) / (2 * h)
    assert abs(g - fd) < 1e-5 * abs(fd)
    # exact estimator (every site its own colour) -> closed form -sum cos(kp)/lambda^2
    col = np.arange(256, dtype=np.int32)
    g = Gr.grad_m2(E.Laplacian(dims, m2), col, 256, 0, 1, 0, 0, p, 1e-13)
    assert abs(g + free_laplacian_trace(dims, m2, 0, p, power=2)) < 1e-8
    assert abs(g - (-102.302723984847)) < 1e-8


def test_wilson_grad_kappa_and_links_fd():
    dims, kappa, p = [2, 2, 2, 4], 0.12, 1
    U = inputs.gauge_links(dims, 8)
    col, m = greedy_colour(dims, 2, [p], 1, 0)
    op = E.Wilson(dims, U, kappa)
    dk, G, Gb = Gr.grad_links(op, col, m, 3, 1, 1, 2, p, 1e-12, dilute=False)
    dk2 = Gr.grad_kappa(op, col, m, 3, 1, 1, 2, p, 1e-12, dilute=False)
    assert abs(dk - dk2) < 1e-12 * abs(dk)
    h = 1e-5
    f = lambda kap, Ul: _estimate(E.Wilson(dims, Ul, kap), col, m, 3, 1, 1, 2, p, 1e-12, dilute=False)
    fd = (f(kappa + h, U) - f(kappa - h, U)) / (2 * h)
    assert abs(dk - fd) < 1e-5 * abs(fd)
    r = np.random.default_rng(0)
    for _ in range(6):
        n, nu, a, b = r.integers(32), r.integers(4), r.integers(3), r.integers(3)
        for part in ("re", "im"):
            dU = np.zeros_like(U)
            dU[n, nu, a, b] = h if part == "re" else 1j * h
            fd = (f(kappa, U + dU) - f(kappa, U - dU)) / (2 * h)
            an = (G + Gb)[n, nu, a, b] if part == "re" else 1j * (G - Gb)[n, nu, a, b]
            assert abs(an - fd) < 1e-5 * max(abs(fd), 1e-3), (n, nu, a, b, part)


def test_wilson_grad_kappa_identity():
    """sum y^H H x = (1/kappa) sum (y^H x - y^H v), since H x = (x - v) / kappa."""
    dims, kappa, p = [2, 2, 2, 4], 0.11, 1
    U = inputs.gauge_links(dims, 2)
    op = E.Wilson(dims, U, kappa)
    col, m = greedy_colour(dims, 2, [p], 1, 0)
    lhs, rhs = 0.0, 0.0
    for v, x, y in Gr._probe_pairs(op, col, m, 1, 1, 1, 2, p, 1e-12, dilute=False):
        lhs += np.vdot(y, op.hop(x))
        rhs += (np.vdot(y, x) - np.vdot(y, v)) / kappa
    assert abs(lhs - rhs) < 1e-8 * abs(lhs)
