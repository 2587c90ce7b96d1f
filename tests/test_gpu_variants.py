"""The constraint variants of Sec. 8.2 (Table 6) through the C ABI against the
oracle:

  * "c+e+f": corners plus arithmetic edge and face averages as the initial
    constraints, no adaptivity (AMB_CORNERS_EDGES_FACES): coarse space size,
    constraint row spaces per substructure, solution (1e-6 against a sparse
    direct solve), PCG iterations (+-1) and the condition estimate; two and
    three levels, both problem kinds, both precisions;
  * "3eigv": corners and edge averages plus the three leading pair
    eigenvectors of every face (tau below every positive eigenvalue, at most
    3 rows per face): the selections are exactly 3 per face and the
    iterations match the oracle's;
  * the library rejects face averages in an adaptive set-up (AMB_EINVAL).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import amb_inputs as ai
from oracle import fe, levels as olv, solver

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


def _check_solution(B, prob, ctx, h, res, f_free):
    f = ctx.load_vector(prob.body)
    u, info = ctx.solve(f)
    free = fe.free_dof_map(prob)[1]
    assert np.allclose(f[free], f_free, rtol=1e-12, atol=1e-16)
    ud = spla.spsolve(h.ops[0].tocsc(), f_free)
    assert info.rel_residual <= 1e-8
    assert np.linalg.norm(u[free] - ud) <= 1e-6 * np.linalg.norm(ud)
    assert abs(info.iterations - res.its) <= 1, (info.iterations, res.its)
    return info


@pytest.mark.parametrize("dpn,split,precision", [(1, (2, 2, 1), "fp64"), (3, (2, 2, 1), "fp64"),
                                                  (3, (2, 2, 2), "fp32"), (1, (3, 2, 2), "fp32")])
def test_corners_edges_faces_two_levels(B, dpn, split, precision):
    prob = ai.toy(4 if dpn == 1 else 3, dpn, 61, split=split, sigma=2.0)
    prec = B.FP64 if precision == "fp64" else B.FP32
    ctx = B.Context.from_problem(prob, adaptive=0, initial_constraints=B.CORNERS_EDGES_FACES, precision=prec)
    h, res, f_free = solver.solve(prob, adaptive=False, initial="cef")
    lev = h.levels[0]
    free = fe.free_dof_map(prob)[1]
    assert ctx.level_info(1).n_coarse == lev.n_coarse
    for s, sb in enumerate(lev.subs):
        dofs = ctx.export(B.X_SUB_DOFS, 1, s, np.int64)
        ni, ng, _, nc = ctx.export(B.X_SUB_SIZES, 1, s, np.int32)
        assert nc == sb.c.shape[0]
        pos = {int(d): i for i, d in enumerate(free[sb.gdofs])}
        perm = np.array([pos[int(d)] for d in dofs[ni:]])
        Cl = ctx.export(B.X_CONSTR, 1, s, np.float64).reshape(nc, ng)
        assert np.linalg.matrix_rank(np.vstack([Cl, sb.c[:, perm]]), tol=1e-10) == nc
    info = _check_solution(B, prob, ctx, h, res, f_free)
    assert abs(info.cond_estimate - res.cond) <= 1e-3 * res.cond + 0.05
    ctx.close()


@pytest.mark.parametrize("dpn", [1, 3])
def test_corners_edges_faces_three_levels(B, dpn):
    groups = [np.array([0, 2, 4]), np.array([0, 2]), np.array([0, 1])]
    prob = ai.toy(3, dpn, 62, split=(4, 2, 1), levels=3, groups=groups, sigma=1.0)
    ctx = B.Context.from_problem(prob, adaptive=0, initial_constraints=B.CORNERS_EDGES_FACES)
    h, res, f_free = solver.solve(prob, adaptive=False, initial="cef")
    for lvl in (1, 2):
        assert ctx.level_info(lvl).n_coarse == h.levels[lvl - 1].n_coarse
    _check_solution(B, prob, ctx, h, res, f_free)
    ctx.close()


@pytest.mark.parametrize("dpn,split", [(1, (2, 2, 1)), (3, (2, 2, 1))])
def test_three_eigenvectors_per_face(B, dpn, split):
    prob = ai.toy(4 if dpn == 1 else 3, dpn, 63, split=split, sigma=2.0)
    tau = 1e-9
    ctx = B.Context.from_problem(prob, tau=tau, max_adaptive_per_face=3, lobpcg_tol=1e-8, lobpcg_maxit=300)
    rep = ctx.report()
    h, res, f_free = solver.solve(prob, tau=tau, max_per_face=3)
    assert all(p["n_selected"] == 3 for p in rep["pairs"])
    assert h.reports[0].n_selected == [3] * len(rep["pairs"])
    assert rep["n_adaptive"][0] == h.reports[0].n_adaptive
    _check_solution(B, prob, ctx, h, res, f_free)
    ctx.close()


def test_face_averages_rejected_when_adaptive(B):
    prob = ai.toy(3, 1, 64, split=(2, 2, 1))
    with pytest.raises(B.AmbError) as e:
        B.Context.from_problem(prob, adaptive=1, initial_constraints=B.CORNERS_EDGES_FACES)
    assert e.value.status == B.EINVAL
