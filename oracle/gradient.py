"""Adjoint gradient of a quantity of interest q(u) w.r.t. the element
log-coefficients theta_e = log(kappa_e) (or log of Young's modulus).

With A(theta) u = f, f independent of theta, and A = sum_e exp(theta_e) K_e^hat:
    dq/dtheta_e = -kappa_e * lambda_e^T Khat u_e,   A lambda = dq/du.
For the compliance q = f^T u the adjoint is lambda = u.

This step is not in the paper (it differentiates the solve).  Pinned by
tests/test_oracle_gradient.py against central finite differences.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import fe


def element_gradient(prob, u_free, lam_free, coeff=None):
    """g_e = -coeff_e lambda_e^T Khat u_e.  Pinned by
    test_oracle_gradient.py::test_gradient_vs_central_fd."""
    coeff = prob.coeff if coeff is None else coeff
    khat = fe.reference_stiffness(prob.dofs_per_node, prob.h, prob.poisson_ratio)
    ue = fe.to_full(prob, u_free)[fe.element_dofs(prob)]
    le = fe.to_full(prob, lam_free)[fe.element_dofs(prob)]
    return -coeff * np.einsum("ea,ab,eb->e", le, khat, ue)


def compliance_and_gradient(prob, coeff=None):
    """Direct (sparse LU) compliance and its adjoint gradient.

    Pinned by test_oracle_gradient.py::test_gradient_vs_central_fd (central differences in log-
    coefficient space) and test_gradient_through_bddc_solution.
    """
    coeff = prob.coeff if coeff is None else coeff
    a = fe.assemble_global(prob, coeff)
    f = fe.load_vector(prob)
    u = spla.spsolve(a.tocsc(), f)
    return float(f @ u), element_gradient(prob, u, u, coeff)


def linear_qoi_and_gradient(prob, w_free, coeff=None):
    """A linear quantity of interest q = w^T u (w on the free dofs), by sparse
    LU, and its adjoint gradient: A lambda = w (A is symmetric), then the
    element formula above.

    Pinned by test_oracle_gradient.py::test_linear_qoi_gradient_vs_central_fd.
    """
    coeff = prob.coeff if coeff is None else coeff
    a = fe.assemble_global(prob, coeff).tocsc()
    f = fe.load_vector(prob)
    lu = spla.splu(a)
    u = lu.solve(f)
    lam = lu.solve(np.asarray(w_free, dtype=float))
    return float(w_free @ u), element_gradient(prob, u, lam, coeff)
