"""torch.autograd.Functions for quantities of interest of the BDDC-preconditioned
solve A(theta) u = f, theta_e = log(coeff_e):

  compliance(theta, prob, f)           q = f^T u      (adjoint = u: no second solve)
  linear_functional(theta, prob, f, w) q = w^T u      (adjoint solve A lambda = w)

Forward: set-up and PCG solve through the C ABI (amb_setup, amb_solve).
Backward: the adjoint element gradient from amb_grad, computed only then: the
library context of the forward is kept until backward runs (it holds the
factors the adjoint solve reuses) and released right away when no gradient
is needed (grad mode off, or theta not requiring grad).  All arithmetic runs
in libamb.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


def _forward(ctx, theta, prob, f, opts):
    coeff = torch.exp(theta.detach().to(torch.float64)).cpu().numpy()
    c = B.Context.from_problem(prob, coeff=coeff, **opts)
    u, _ = c.solve(f)
    if ctx.needs_input_grad[0]:
        ctx.amb = c
    else:
        c.close()
        ctx.amb = None
    return u


def _take(ctx):
    c = ctx.amb
    ctx.amb = None
    if c is None:
        raise RuntimeError("backward of an amb Function ran twice or without a forward context")
    return c


class Compliance(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta: torch.Tensor, prob, f: np.ndarray, opts: dict):
        u = _forward(ctx, theta, prob, f, opts)
        return theta.new_tensor(float(np.dot(f, u)))

    @staticmethod
    def backward(ctx, grad_out):
        c = _take(ctx)
        try:
            g = c.grad(B.QOI_COMPLIANCE)
        finally:
            c.close()
        return grad_out * torch.from_numpy(g).to(grad_out.device, grad_out.dtype), None, None, None


class LinearFunctional(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta: torch.Tensor, prob, f: np.ndarray, w: np.ndarray, opts: dict):
        u = _forward(ctx, theta, prob, f, opts)
        ctx.w = w
        return theta.new_tensor(float(np.dot(w, u)))

    @staticmethod
    def backward(ctx, grad_out):
        c = _take(ctx)
        try:
            g = c.grad(B.QOI_GENERAL, dq_du=ctx.w)
        finally:
            c.close()
        return grad_out * torch.from_numpy(g).to(grad_out.device, grad_out.dtype), None, None, None, None


def compliance(theta: torch.Tensor, prob, f: np.ndarray, **opts) -> torch.Tensor:
    """q = f^T u(theta); f: full-grid nodal load vector (amb_load_vector)."""
    return Compliance.apply(theta, prob, f, opts)


def linear_functional(theta: torch.Tensor, prob, f: np.ndarray, w: np.ndarray, **opts) -> torch.Tensor:
    """q = w^T u(theta); f, w: full-grid nodal vectors (entries of Dirichlet nodes ignored)."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    return LinearFunctional.apply(theta, prob, f, w, opts)
