"""Write tests/golden/*.json from the CPU oracle only (no CUDA path involved).

    python tests/golden/make_golden.py 1 2      # config indices

    python tests/golden/make_golden.py grad4     # compliance gradient of config 4

For each workload: PCG iterations and condition estimate of the adaptive
two-level method (Algorithm 3 + Algorithm 1, rtol 1e-8), adaptive rows and
indicator per level (eq. cond-ind-mlevel), the number of coarse dofs, and
the largest computed pair eigenvalue per face.  The 48^3 elasticity
workload takes about 20 minutes on 8 cores.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import amb_inputs as ai  # noqa: E402
import numpy as np  # noqa: E402

from oracle import gradient as og  # noqa: E402
from oracle import solver  # noqa: E402


def golden(index):
    prob = ai.config(index)
    t0 = time.perf_counter()
    h, res, f = solver.solve(prob)
    out = {
        "workload": prob.name, "config_index": index, "pcg_iterations": int(res.its),
        "rel_residual": float(res.rel_res), "cond_estimate": float(res.cond),
        "n_adaptive": [int(r.n_adaptive) for r in h.reports],
        "omega_level": [float(r.omega_tilde) for r in h.reports],
        "n_coarse": [int(l.n_coarse) for l in h.levels],
        "pairs": [[int(s), int(t)] for (s, t) in h.reports[0].pairs],
        "n_selected": [int(k) for k in h.reports[0].n_selected],
        "lambda_top": [[float(x) for x in lam[:4]] for lam in h.reports[0].lam],
        "oracle_seconds": time.perf_counter() - t0,
        "source": "oracle/ (tests/golden/make_golden.py)",
    }
    with open(os.path.join(HERE, f"config{index}_oracle.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    return out


def gradient_golden(index=4, n_samples=512):
    """Compliance Q = f^T u and its adjoint gradient dQ/dlog(kappa_e) (for the
    compliance the adjoint is lambda = u) at seeded sample elements.  u comes from
    the oracle's two-level BDDC + PCG without adaptive constraints at rtol
    1e-12 (the gradient does not depend on the preconditioner; a sparse LU of
    the 270,400-dof system takes far longer)."""
    prob = ai.config(index)
    t0 = time.perf_counter()
    h, res, f = solver.solve(prob, rtol=1e-12, adaptive=False)
    u = res.u
    g = og.element_gradient(prob, u, u)
    rng = np.random.default_rng(np.random.PCG64(104))
    idx = np.sort(rng.choice(g.size, size=n_samples, replace=False))
    out = {
        "workload": prob.name, "config_index": index, "compliance": float(f @ u),
        "pcg_iterations": int(res.its), "rel_residual": float(res.rel_res),
        "sample_elements": [int(i) for i in idx], "gradient_samples": [float(x) for x in g[idx]],
        "gradient_abs_max": float(np.abs(g).max()), "gradient_sum": float(g.sum()),
        "oracle_seconds": time.perf_counter() - t0,
        "source": "oracle/ (tests/golden/make_golden.py grad4)",
    }
    with open(os.path.join(HERE, f"config{index}_gradient.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    return out


if __name__ == "__main__":
    for a in sys.argv[1:] or ["1"]:
        if a.startswith("grad"):
            o = gradient_golden(int(a[4:]))
            print(o["workload"], o["compliance"], o["pcg_iterations"], o["oracle_seconds"])
            continue
        o = golden(int(a))
        print(o["workload"], o["pcg_iterations"], o["n_adaptive"], o["omega_level"])
