"""Even-odd trace estimation for the Laplacian (pt_trace_PAinv_eo), run by
its host twin (the same per-site arithmetic and steps; no GPU): the probed
estimates equal the oracle's (Eqs. (1), (5)) for Z2 noise, several
displacements, set offsets and colourings; iterations against the full
system; argument and iteration-limit errors."""
import numpy as np
import pytest

import oracle.estimator as OE
from oracle.colouring import greedy_colour


@pytest.mark.parametrize("dims,m2,mu,ps,k,noise,set0,n_sets", [
    ([4, 4, 4, 4], 0.1, 0, [0, 1, 2], 1, 0, 0, 2),
    ([6, 4, 2, 8], 0.05, 3, [1, 3], 2, 0, 3, 2),
    ([8, 8, 4, 4], 0.01, 1, [0, 4], 1, 0, 0, 1),
])
def test_estimates_match_the_oracle(ptlib, dims, m2, mu, ps, k, noise, set0, n_sets):
    col, m = greedy_colour(dims, mu, ps, k, 0)
    est, st = ptlib.trace_eo_host(dims, m2, col, m, mu, ps, noise, 1000, set0, n_sets, tol=1e-11)
    want = OE.probed_estimates(OE.Laplacian(dims, m2), col, m, 1000, n_sets, noise, mu, ps, 1e-13, set0=set0)
    assert np.allclose(est, want, rtol=1e-8, atol=1e-9 * np.abs(want).max())
    assert st["n_rhs"] == n_sets * m and st["n_noconv"] == 0 and st["max_relres"] <= 1e-11


def test_iterations_against_the_full_system(ptlib):
    """m^2 = 0.01 on 8x8x4x4: the even system's FP32 inner CG, restarted by the
    FP64 defect correction (inner tolerance 1e-5, as the engine's), takes
    fewer iterations than the oracle's unrestarted FP64 CG on the full system
    for the same probes (117 against 128); unrestarted FP64 CG on the even
    system takes half (16-17 against 32 per probe), which the restarts partly
    give back on a lattice this small (CG nearly terminates on its few
    distinct eigenvalues)."""
    from oracle.probes import probe
    dims, m2, mu = [8, 8, 4, 4], 0.01, 3
    col, m = greedy_colour(dims, mu, [1], 1, 0)
    _, st = ptlib.trace_eo_host(dims, m2, col, m, mu, [1], "z2", 7, 0, 1, tol=1e-10, delta=1e-5)
    full = eo64 = 0
    for c in range(m):
        v = probe(col, c, 7, 0, 0, 1, 0)
        full += OE.Laplacian(dims, m2).solve(v, 1e-10)[1]
        eo64 += int(ptlib.eo_solve_host(0, dims, v.reshape(1, -1), tol=1e-10, m2=m2)[1][0])
    assert st["inner_iters"] < full, (st["inner_iters"], full)
    assert eo64 <= 0.55 * full, (eo64, full)


def test_errors(ptlib):
    col = np.zeros(3 * 4 * 4 * 4, dtype=np.int32)
    with pytest.raises(ptlib.PtraceError):                                 # complex noise, real operator
        ptlib.trace_eo_host([4, 4, 4, 4], 0.1, np.zeros(256, np.int32), 1, 0, [1], "z4")
    with pytest.raises(ptlib.PtraceError):
        ptlib.trace_eo_host([3, 4, 4, 4], 0.1, col, 1, 0, [1])              # odd side
    with pytest.raises(ptlib.PtraceError):
        ptlib.trace_eo_host([4, 4, 4, 4], 0.1, np.zeros(256, np.int32), 1, 0, list(range(33)))
    with pytest.raises(ptlib.PtraceError) as ei:
        ptlib.trace_eo_host([4, 4, 4, 4], 0.01, np.zeros(256, np.int32), 1, 0, [1], tol=1e-14, maxit=2)
    assert ei.value.code == ptlib.PT_ERR_NOCONV


@pytest.mark.parametrize("dims,mu,ps", [
    ([2, 2, 2, 2], 2, [0, 1, -1]),                 # both neighbours along a side of 2 are one site
    ([4, 2, 4, 6], 3, [-2, 6, 13]),                # negative and wrapping displacements
    ([4, 4, 2, 2], 0, list(range(-16, 16))),       # the full 32 outputs per solve
])
def test_edge_cases_match_the_oracle(ptlib, dims, mu, ps):
    m2 = 0.2
    col, m = greedy_colour(dims, mu, [1], 1, 0)
    est, _ = ptlib.trace_eo_host(dims, m2, col, m, mu, ps, "z2", 11, 1, 2, tol=1e-11)
    want = OE.probed_estimates(OE.Laplacian(dims, m2), col, m, 11, 2, 0, mu, ps, 1e-13, set0=1)
    assert np.allclose(est, want, rtol=1e-8, atol=1e-9 * np.abs(want).max())
