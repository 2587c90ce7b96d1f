"""The torch.autograd.Function of the compliance (paper_1301_0191_gb300.autograd)
through the C ABI: the forward value equals the oracle compliance f^T u,
backward gives the oracle adjoint gradient with respect to log(coeff), and a
central difference of the Function itself along a seeded direction agrees
with the gradient to 1e-5 relative."""
import numpy as np
import pytest

import amb_inputs as ai
from oracle import gradient as og

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1301_0191_gb300 import binding
    return binding


@pytest.mark.parametrize("dpn", [1, 3])
def test_compliance_function(B, dpn):
    import torch
    from paper_1301_0191_gb300 import autograd as AG
    prob = ai.toy(3, dpn, 61 + dpn, split=(2, 2, 1), sigma=1.0)
    ctx = B.Context.from_problem(prob, adaptive=0)
    f = ctx.load_vector(prob.body)
    ctx.close()
    opts = dict(precision=B.FP64, pcg_rtol=1e-12)
    theta = torch.tensor(np.log(prob.coeff), dtype=torch.float64, requires_grad=True)
    q = AG.compliance(theta, prob, f, **opts)
    q.backward()
    q_ref, g_ref = og.compliance_and_gradient(prob)
    assert abs(float(q.detach()) - q_ref) <= 1e-10 * abs(q_ref)
    g = theta.grad.numpy()
    assert np.abs(g - g_ref).max() <= 1e-7 * np.abs(g_ref).max()
    # central difference of the Function along a seeded direction
    d = torch.from_numpy(np.random.default_rng(np.random.PCG64(62)).standard_normal(theta.numel()))
    h = 1e-5
    with torch.no_grad():
        qp = float(AG.compliance(theta + h * d, prob, f, **opts))
        qm = float(AG.compliance(theta - h * d, prob, f, **opts))
    fd = (qp - qm) / (2 * h)
    ad = float(np.dot(g, d.numpy()))
    assert abs(fd - ad) <= 1e-5 * abs(ad)


def test_linear_functional_and_no_grad(B):
    """q = w^T u through the general adjoint (AMB_QOI_GENERAL): value and
    gradient against the oracle's sparse-LU adjoint; under no_grad the
    Function gives the same value and keeps no context for a backward."""
    import torch
    from oracle import fe
    from paper_1301_0191_gb300 import autograd as AG
    prob = ai.toy(3, 3, 71, split=(2, 2, 1), sigma=1.0)
    ctx = B.Context.from_problem(prob, adaptive=0)
    f = ctx.load_vector(prob.body)
    ctx.close()
    free = fe.free_dof_map(prob)[1]
    w = np.random.default_rng(np.random.PCG64(72)).standard_normal(f.size)
    opts = dict(precision=B.FP64, pcg_rtol=1e-12)
    theta = torch.tensor(np.log(prob.coeff), dtype=torch.float64, requires_grad=True)
    q = AG.linear_functional(theta, prob, f, w, **opts)
    q.backward()
    q_ref, g_ref = og.linear_qoi_and_gradient(prob, w[free])
    assert abs(float(q.detach()) - q_ref) <= 1e-10 * abs(q_ref)
    assert np.abs(theta.grad.numpy() - g_ref).max() <= 1e-7 * np.abs(g_ref).max()
    with torch.no_grad():
        q2 = AG.linear_functional(theta, prob, f, w, **opts)
    assert not q2.requires_grad
    assert abs(float(q2) - float(q.detach())) <= 1e-12 * abs(q_ref)
