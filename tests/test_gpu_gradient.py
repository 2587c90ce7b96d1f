"""Adjoint gradient of the compliance on the 64^3 Poisson workload (4x4x4
substructures, log-GRF coefficients), through the C ABI:

- against central finite differences of Q = f^T u in 20 seeded directions
  d ~ N(0, I) (not normalized: |d| ~ 512) with h = 1e-5, 1e-5 relative (each
  Q from its own set-up + solve at rtol 1e-12).  With normalized directions
  and h = 1e-6 the compliance moves by about 1e-11 of itself, next to the
  solves' 1e-12, and the quotient's rounding error was 2e-3 (measured);
- against the oracle's adjoint gradient at 512 seeded sample elements and its
  compliance (tests/golden/config4_gradient.json, written from oracle/ only).
  The gradient is quadratic in u, so the solution's 1e-6 relative bound
  carries over: sampled entries within 1e-6 of the largest |g_e| (both sides
  solve to rtol 1e-12; measured 1e-7).

The gradient context is the two-level adaptive FP64 form.  The finite
differences use FP32-preconditioned, non-adaptive contexts: Q only depends
on the solution, which the FP64 PCG resolves to rtol 1e-12 either way.
"""
import json
import os

import numpy as np
import pytest

import amb_inputs as ai

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "config4_gradient.json")


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1301_0191_gb300 import binding
    return binding


def _compliance(B, prob, coeff, **opts):
    c = B.Context.from_problem(prob, coeff=coeff, pcg_rtol=1e-12, **opts)
    f = c.load_vector(prob.body)
    u, info = c.solve(f)
    assert info.rel_residual <= 1e-12
    return float(f @ u), c, info


def test_compliance_gradient_64cube(B):
    prob = ai.config(4)
    q0, ctx, info = _compliance(B, prob, prob.coeff, precision=B.FP64)
    g = ctx.grad(B.QOI_COMPLIANCE)
    ctx.close()
    assert g.shape == (prob.nx * prob.ny * prob.nz,)

    # oracle adjoint gradient and compliance
    with open(GOLD) as fh:
        gold = json.load(fh)
    idx = np.asarray(gold["sample_elements"])
    g_ref = np.asarray(gold["gradient_samples"])
    assert abs(q0 - gold["compliance"]) <= 1e-10 * abs(gold["compliance"])
    assert np.abs(g[idx] - g_ref).max() <= 1e-6 * gold["gradient_abs_max"]
    assert abs(np.abs(g).max() - gold["gradient_abs_max"]) <= 1e-6 * gold["gradient_abs_max"]

    # central finite differences along seeded N(0,1) directions in log(kappa)
    rng = np.random.default_rng(np.random.PCG64(104))
    h = 1e-5
    worst = 0.0
    for _ in range(20):
        d = rng.standard_normal(g.size)
        qp, cp, _ = _compliance(B, prob, prob.coeff * np.exp(h * d), precision=B.FP32, adaptive=0)
        cp.close()
        qm, cm, _ = _compliance(B, prob, prob.coeff * np.exp(-h * d), precision=B.FP32, adaptive=0)
        cm.close()
        fd = (qp - qm) / (2 * h)
        ad = float(g @ d)
        worst = max(worst, abs(fd - ad) / abs(ad))
    assert worst <= 1e-5, worst
