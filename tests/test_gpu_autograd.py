"""torch.autograd wrapper of the adjoint gradient against plain torch autograd
through a dense Wilson operator on a tiny lattice (CPU, complex128), for a
real loss mixing Re T and Im T (pins the complex-gradient convention)."""
import numpy as np
import pytest

from oracle import lattice as OL
from oracle import operators as OO
from oracle.colouring import greedy_colour
from oracle.probes import probe
from paper_2106_01275_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_01275_gb300 import build
    build.build()
    from paper_2106_01275_gb300 import ptrace
    return ptrace


def dense_trace_torch(kappa, U, dims, col, m, mu, p, seed):
    """T = sum_{c,a} v^H P A^{-1} v with a dense, differentiable torch A."""
    import torch
    g, _ = OO.gammas()
    gam = [torch.tensor(x) for x in g]
    I4 = torch.eye(4, dtype=torch.complex128)
    N = int(np.prod(dims))
    xs = OL.coords(dims)
    blocks = {}
    A = torch.eye(12 * N, dtype=torch.complex128)
    rows = []
    for i in range(N):
        row = [torch.zeros((12, 12), dtype=torch.complex128) for _ in range(N)]
        row[i] = row[i] + torch.eye(12, dtype=torch.complex128)
        for nu in range(4):
            yf = xs[i].copy(); yf[nu] += 1
            yb = xs[i].copy(); yb[nu] -= 1
            sf = -1.0 if (nu == 3 and yf[3] == dims[3]) else 1.0
            sb = -1.0 if (nu == 3 and yb[3] < 0) else 1.0
            jf = int(OL.index_of(yf, dims)); jb = int(OL.index_of(yb, dims))
            row[jf] = row[jf] - kappa * sf * torch.kron(I4 - gam[nu], U[i, nu])
            row[jb] = row[jb] - kappa * sb * torch.kron(I4 + gam[nu], U[jb, nu].conj().T.contiguous())
        rows.append(torch.cat(row, dim=1))
    A = torch.cat(rows, dim=0)
    perm = OL.shift_map(dims, mu, p)
    idx = torch.tensor((12 * perm[:, None] + np.arange(12)[None, :]).reshape(-1))
    T = 0
    for c in range(m):
        for a in range(12):
            v = torch.tensor(probe(col, c, seed, 0, 1, 12, a).reshape(-1))
            x = torch.linalg.solve(A, v)
            T = T + torch.vdot(v, x[idx])
    return T


def test_autograd_matches_dense_torch(pt):
    import torch
    from paper_2106_01275_gb300.autograd import ProbeSpec, wilson_trace
    dims, kappa0, mu, p = [2, 2, 2, 4], 0.12, 2, 1
    U0 = inputs.gauge_links(dims, 21)
    colv, m = greedy_colour(dims, mu, [p], 1, 0)
    # reference: dense torch autograd on the CPU
    kap_r = torch.tensor(kappa0, dtype=torch.float64, requires_grad=True)
    U_r = torch.tensor(U0, requires_grad=True)
    T_r = dense_trace_torch(kap_r, U_r, dims, colv, m, mu, p, 11)
    L_r = T_r.real + 0.3 * T_r.imag
    L_r.backward()
    # library: adjoint gradient through the autograd wrapper
    ctx = pt.Context(0)
    spec = ProbeSpec(ctx, dims, torch.as_tensor(colv).cuda(), m, mu, p, "z4", 11, 0, 1, True, "fp64", 1e-12, 5000)
    kap = torch.tensor(kappa0, dtype=torch.float64, requires_grad=True)
    U = torch.tensor(U0).cuda().requires_grad_(True)
    T = wilson_trace(kap, U, spec)
    L = T.real + 0.3 * T.imag
    L.backward()
    assert abs(T.item() - T_r.item()) <= 1e-9 * abs(T_r.item())
    assert abs(kap.grad.item() - kap_r.grad.item()) <= 1e-7 * abs(kap_r.grad.item())
    gU = U.grad.cpu().numpy()
    gU_r = U_r.grad.numpy()
    assert np.max(np.abs(gU - gU_r)) <= 1e-7 * np.max(np.abs(gU_r))


def test_laplacian_autograd_dm2(pt):
    import torch
    from paper_2106_01275_gb300.autograd import ProbeSpec, laplacian_trace
    import oracle.estimator as OE
    import oracle.gradient as OG
    dims, m2, p = [4, 4, 4, 4], 0.1, 1
    colv, m = greedy_colour(dims, 0, [p], 2, 0)
    ctx = pt.Context(0)
    spec = ProbeSpec(ctx, dims, torch.as_tensor(colv).cuda(), m, 0, p, "z2", 0, 0, 2, True, "mixed_fp32", 1e-12, 5000)
    m2t = torch.tensor(m2, dtype=torch.float64, requires_grad=True)
    T = laplacian_trace(m2t, spec)
    T.real.backward()
    want = OG.grad_m2(OE.Laplacian(dims, m2), colv, m, 0, 2, 0, 0, p, 1e-13)
    assert abs(m2t.grad.item() - want.real) <= 1e-8 * abs(want)
