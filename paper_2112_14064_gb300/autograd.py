"""Eigenvalues of the damped QEP as a differentiable function of sigma_e.

``qep_eigenvalues(sigma_e, ...)`` returns the eigenvalues nearest the target
(complex tensor).  Its backward pass calls ``rigaqep_grad_damping`` (device
kernel): with G[k, e] = d lambda_k / d sigma_e and the incoming gradient g of
the complex output (PyTorch's convention g = dL/dRe + i dL/dIm for a real
loss L), the gradient of the real input is

    dL / d sigma_e = sum_k Re( conj(g_k) G[k, e] ).

Eigenvectors are returned as a non-differentiable output.  Gradients of
repeated eigenvalues are undefined (first-order perturbation of a simple
eigenvalue only).
"""
import torch

from . import rigaqep


class _QEPEigs(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sigma_e, ne, p, block, neig, target, opts):
        prob = rigaqep.Problem(ne, p, block, sigma_e.detach().contiguous()).analyze()
        lam, X, eta, nconv, st = prob.eigs(neig, target, raise_on_noconv=True, **opts)
        ctx.prob = prob
        ctx.ne = ne
        ctx.save_for_backward(lam, X)
        ctx.mark_non_differentiable(X, eta)
        return lam, X, eta

    @staticmethod
    def backward(ctx, g_lam, g_X, g_eta):
        lam, X = ctx.saved_tensors
        grad = None
        if g_lam is not None and ctx.needs_input_grad[0]:
            G = ctx.prob.grad_damping(lam, X)                    # (neig, ne^2) complex
            grad = (torch.conj(g_lam)[:, None] * G).real.sum(0)
        ctx.prob.close()
        return grad, None, None, None, None, None, None


def qep_eigenvalues(sigma_e, ne, p, block, neig, target, **opts):
    """(lambda, X, eta) for the neig eigenpairs nearest target; lambda is
    differentiable with respect to sigma_e (float64 CUDA tensor of ne*ne)."""
    return _QEPEigs.apply(sigma_e, ne, p, block, neig, target, opts)
