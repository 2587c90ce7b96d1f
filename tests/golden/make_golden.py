"""Write tests/golden/*.json from the CPU oracle only (no CUDA path involved).

    python tests/golden/make_golden.py 1 2      # config indices

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


if __name__ == "__main__":
    for a in sys.argv[1:] or ["1"]:
        o = golden(int(a))
        print(o["workload"], o["pcg_iterations"], o["n_adaptive"], o["omega_level"])
