"""torch.autograd.Function for the compliance q = f^T u(theta) of the
BDDC-preconditioned solve, theta_e = log(coeff_e).

Forward: set-up and PCG solve through the C ABI (amb_setup, amb_solve);
backward: the adjoint element gradient from amb_grad (compliance: the
adjoint equals u, so no second solve).  All arithmetic runs in libamb.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


class Compliance(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta: torch.Tensor, prob, f: np.ndarray, opts: dict):
        coeff = torch.exp(theta.detach().to(torch.float64)).contiguous()
        c = B.Context.from_problem(prob, coeff=coeff.cpu().numpy(), **opts)
        u, info = c.solve(f)
        g = c.grad(B.QOI_COMPLIANCE)
        c.close()
        ctx.save_for_backward(torch.from_numpy(g).to(theta.device))
        return theta.new_tensor(float(np.dot(f, u)))

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g.to(grad_out.dtype), None, None, None


def compliance(theta: torch.Tensor, prob, f: np.ndarray, **opts) -> torch.Tensor:
    return Compliance.apply(theta, prob, f, opts)
