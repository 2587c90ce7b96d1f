"""Pins of the adjoint gradient (an addition to the method, not in the paper):
central finite differences in log-coefficient space."""
import numpy as np
import pytest

import amb_inputs as ai
from oracle import fe, gradient, solver


@pytest.mark.parametrize("dpn", [1, 3])
def test_gradient_vs_central_fd(dpn):
    prob = ai.toy(3, dpn, 81, split=(2, 1, 1), sigma=1.0)
    j0, g = gradient.compliance_and_gradient(prob)
    rng = np.random.default_rng(104)
    theta = np.log(prob.coeff)
    for _ in range(3):
        d = rng.standard_normal(theta.size)
        d /= np.linalg.norm(d)
        hstep = 1e-6
        jp, _ = gradient.compliance_and_gradient(prob, np.exp(theta + hstep * d))
        jm, _ = gradient.compliance_and_gradient(prob, np.exp(theta - hstep * d))
        fd = (jp - jm) / (2 * hstep)
        assert abs(fd - g @ d) <= 1e-6 * abs(fd)


def test_gradient_through_bddc_solution():
    prob = ai.toy(4, 1, 82, split=(2, 2, 1), sigma=1.5)
    h, res, f = solver.solve(prob, rtol=1e-12)
    g_pcg = gradient.element_gradient(prob, res.u, res.u)
    _, g_dir = gradient.compliance_and_gradient(prob)
    assert np.abs(g_pcg - g_dir).max() <= 1e-8 * np.abs(g_dir).max()


@pytest.mark.parametrize("dpn", [1, 3])
def test_linear_qoi_gradient_vs_central_fd(dpn):
    """q = w^T u for a seeded w: the adjoint gradient against central
    differences, and against the compliance formula when w = f."""
    prob = ai.toy(3, dpn, 83, split=(2, 1, 1), sigma=1.0)
    n = fe.free_dof_map(prob)[1].size
    w = np.random.default_rng(105).standard_normal(n)
    q0, g = gradient.linear_qoi_and_gradient(prob, w)
    theta = np.log(prob.coeff)
    rng = np.random.default_rng(106)
    for _ in range(3):
        d = rng.standard_normal(theta.size)
        d /= np.linalg.norm(d)
        hstep = 1e-6
        qp, _ = gradient.linear_qoi_and_gradient(prob, w, np.exp(theta + hstep * d))
        qm, _ = gradient.linear_qoi_and_gradient(prob, w, np.exp(theta - hstep * d))
        fd = (qp - qm) / (2 * hstep)
        assert abs(fd - g @ d) <= 1e-6 * max(abs(fd), 1e-3 * np.linalg.norm(g))
    f = fe.load_vector(prob)
    qf, gf = gradient.linear_qoi_and_gradient(prob, f)
    qc, gc = gradient.compliance_and_gradient(prob)
    assert abs(qf - qc) <= 1e-12 * abs(qc)
    assert np.abs(gf - gc).max() <= 1e-12 * np.abs(gc).max()
