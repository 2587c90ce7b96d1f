"""The set-up's host combinatorics (csrc/topology.cpp) run on up to 16 host
threads; every index writes only its own outputs, so the result must not
depend on the thread count.  amb_plan (host only) of the 96^3 three-level and
the 48^3 elasticity workloads, levels 1 and 2, is compared between one thread
(AMB_HOST_THREADS=1) and several, field by field."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import json, sys
sys.path.insert(0, ROOT)
import numpy as np
import amb_inputs as ai
from paper_1301_0191_gb300 import binding as B
out = {}
for idx in (2, 3):
    prob = ai.config(idx)
    parents = list(prob.sub_to_parent or [])
    nsub = [prob.n_subs(2 + i) for i in range(len(parents))]
    for level in range(1, len(parents) + 2):
        info, subs = B.plan(prob.nx, prob.ny, prob.nz, prob.dofs_per_node, prob.dirichlet_node_mask,
                            prob.elem_to_sub, prob.n_subs(1), levels=len(parents) + 2,
                            sub_to_parent=parents, n_sub=nsub, level=level)
        out[f"{idx}/{level}"] = [[getattr(info, f) for f, _ in info._fields_], subs.tolist()]
print(json.dumps(out))
"""


def _plan(threads):
    env = dict(os.environ, AMB_HOST_THREADS=str(threads))
    r = subprocess.run([sys.executable, "-c", SCRIPT.replace("ROOT", repr(ROOT))], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_host_combinatorics_do_not_depend_on_the_thread_count():
    pytest.importorskip("numpy")
    one, many = _plan(1), _plan(8)
    assert one.keys() == many.keys() and len(one) >= 3
    for key in one:
        assert one[key] == many[key], key
