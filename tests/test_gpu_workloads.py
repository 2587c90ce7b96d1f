"""Full-size parity on the benchmark workloads against stored oracle values
(tests/golden/config*_oracle.json, written by tests/golden/make_golden.py from
oracle/ only).  Sampled outputs the oracle computed one by one: PCG
iterations, adaptive rows per face, the indicator, and the top pair
eigenvalues of the used columns.  The solution is checked through its true
FP64 residual.

FP64 form: eigenvalues within 1e-4 relative, selected rows per face and PCG
iterations within +-1 of the oracle.

FP32 form (factorizations and preconditioner in FP32, trailing updates on the
tensor cores in 3xTF32): the Schur complements carry FP32 rounding, which
moves the pair eigenvalues that sit on near-null directions of S (the large
ones) by up to a few per cent, and the iteration count of the 1e4-contrast
workload grows by a few.  The bounds below are the measured behaviour with a
margin: max eigenvalue deviation <= 5e-2 (measured 3.2e-2 and 3.6e-2), median
<= 5e-3 (measured 1.8e-4 and 1.8e-3), selected rows per face identical
within +-1, PCG iterations within +1 of the oracle (48^3: 38 vs 37; 16^3
channels: 16 vs 15, the FP64 form's count).  The constraint space (G = C_D
S_DD^-1 C_D^T, its inverse, the coarse basis) is FP64 in both forms; with it
in FP32 the 1e4-contrast channels workload took 18 to 34 iterations depending
on rounding order.
"""
import json
import os

import numpy as np
import pytest

import amb_inputs as ai

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1301_0191_gb300 import binding
    return binding


def _gold(i):
    with open(os.path.join(GOLD, f"config{i}_oracle.json")) as f:
        return json.load(f)


@pytest.mark.parametrize("index,precision,rtol_max,rtol_med,it_slack",
                         [(1, "fp64", 1e-4, 1e-4, 1), (2, "fp64", 1e-4, 1e-4, 1),
                          (1, "fp32", 5e-2, 5e-3, 1), (2, "fp32", 5e-2, 5e-3, 1)])
def test_workload_against_oracle(B, index, precision, rtol_max, rtol_med, it_slack):
    g = _gold(index)
    prob = ai.config(index)
    prec = B.FP64 if precision == "fp64" else B.FP32
    ctx = B.Context.from_problem(prob, precision=prec, lobpcg_tol=1e-6, lobpcg_maxit=200)
    f = ctx.load_vector(prob.body)
    u, info = ctx.solve(f)
    rep = ctx.report()
    ctx.close()
    assert info.rel_residual <= 1e-8 and info.true_rel_residual <= 1.01e-8
    assert -1 <= info.iterations - g["pcg_iterations"] <= it_slack, (info.iterations, g["pcg_iterations"])
    pairs = {(p["s"], p["t"]): p for p in rep["pairs"]}
    assert len(pairs) == len(g["pairs"])
    off = 0
    dev = []
    for (s, t), k_o, lam_o in zip(g["pairs"], g["n_selected"], g["lambda_top"]):
        pr = pairs[(s, t)]
        assert abs(pr["n_selected"] - k_o) <= 1
        for i in range(min(len(lam_o), pr["n_selected"] + 1)):
            if lam_o[i] >= 0.1 * prob.tau:
                dev.append((abs(pr["lam"][i] - lam_o[i]) / lam_o[i], (s, t), i))
        off += abs(pr["n_selected"] - k_o)
    worst = max(dev)
    assert worst[0] <= rtol_max, worst
    assert float(np.median([d[0] for d in dev])) <= rtol_med
    assert abs(rep["n_adaptive"][0] - g["n_adaptive"][0]) <= max(2, off)
    # the indicator omega is a pair eigenvalue: same bound
    assert abs(rep["omega_level"][0] - g["omega_level"][0]) <= rtol_max * g["omega_level"][0] + 1e-3
