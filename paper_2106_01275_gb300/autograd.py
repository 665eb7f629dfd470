"""torch.autograd wrapper of the probed trace estimate (not in the paper).

    T = sum_s est[s] = sum_v v^H P A(theta)^{-1} v      (Eqs. (1), (5), fixed probes)

The forward pass calls pt_grad, which solves A x = v and the adjoint system
A^+ y = P^T v for every probe and returns T, dT/dkappa (Wilson) or dT/dm^2
(Laplacian) and, for Wilson links, G = dT/dU and Gbar = dT/d conj(U) (entries
of U treated as free complex numbers).  No Krylov history is kept: only these
derivatives are saved for backward.

Gradient convention (PyTorch's, for a real loss L and incoming g = dL/dT in
torch's sense): for a real parameter x, dL/dx = Re(conj(g) dT/dx); for a
complex tensor U, grad_U = conj(g) * Gbar + g * conj(G).
"""
import torch

from . import ptrace as pt


class ProbeSpec:
    """Everything that fixes the probes and the solver of one estimate."""

    def __init__(self, ctx, dims, col, n_colours, mu, p, noise="z4", seed=0, set0=0, n_sets=1, dilute=True,
                 prec="mixed_fp32", tol=1e-10, maxit=20000, antiperiodic_t=True):
        self.ctx, self.dims, self.col, self.n_colours, self.mu, self.p = ctx, list(dims), col, n_colours, mu, p
        self.noise, self.seed, self.set0, self.n_sets, self.dilute = noise, seed, set0, n_sets, dilute
        self.prec, self.tol, self.maxit, self.antiperiodic_t = prec, tol, maxit, antiperiodic_t


class _WilsonTrace(torch.autograd.Function):
    @staticmethod
    def forward(fctx, kappa, U, spec):
        op = pt.wilson(spec.ctx, spec.dims, U.detach().contiguous(), float(kappa), spec.antiperiodic_t)
        est, dk, G, Gb, _ = pt.grad(op, spec.col, spec.n_colours, spec.mu, spec.p, spec.noise, spec.seed,
                                    spec.set0, spec.n_sets, spec.dilute, spec.prec, spec.tol, spec.maxit,
                                    links=U.requires_grad)
        op.close()
        fctx.dk = dk
        fctx.kappa_is_tensor = torch.is_tensor(kappa)
        if G is not None:
            fctx.save_for_backward(G, Gb)
        else:
            fctx.save_for_backward()
        return torch.tensor(complex(est.sum()), dtype=torch.complex128, device=U.device)

    @staticmethod
    def backward(fctx, g):
        grad_kappa = grad_U = None
        if fctx.needs_input_grad[0]:
            grad_kappa = (torch.conj(g) * fctx.dk).real.to(torch.float64)
        if fctx.needs_input_grad[1]:
            G, Gb = fctx.saved_tensors
            grad_U = torch.conj(g) * Gb + g * torch.conj(G)
        return grad_kappa, grad_U, None


class _LaplacianTrace(torch.autograd.Function):
    @staticmethod
    def forward(fctx, m2, spec):
        op = pt.laplacian(spec.ctx, spec.dims, float(m2))
        est, dm2, _, _, _ = pt.grad(op, spec.col, spec.n_colours, spec.mu, spec.p, spec.noise, spec.seed,
                                    spec.set0, spec.n_sets, spec.dilute, spec.prec, spec.tol, spec.maxit)
        op.close()
        fctx.dm2 = dm2
        return torch.tensor(complex(est.sum()), dtype=torch.complex128, device=spec.col.device)

    @staticmethod
    def backward(fctx, g):
        return (torch.conj(g) * fctx.dm2).real.to(torch.float64), None


def wilson_trace(kappa, U, spec):
    """Probed estimate of Tr(P A^{-1}) for the Wilson operator, differentiable
    in kappa (0-dim float64 tensor) and U (complex128 [N, 4, 3, 3] on the GPU)."""
    return _WilsonTrace.apply(kappa, U, spec)


def laplacian_trace(m2, spec):
    """Probed estimate of Tr(P A^{-1}) for the shifted Laplacian, differentiable in m^2."""
    return _LaplacianTrace.apply(m2, spec)
