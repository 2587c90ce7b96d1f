"""Parity of the adaptive constraint rows themselves (Sec. 7.2, eq. d-def).

The library exports, per face, the rows it added (AMB_X_PAIR_ROWS: the
face-restricted, orthonormalized c_l) and the face's dof ids.  They are
compared with the oracle's rows of the same face:
  * the face dof ids exactly (index work: bit-exact);
  * the number of rows;
  * the row spaces, by principal angles <= 1e-4.
Eigenvectors are unique only up to rotations inside clusters, and a row is
selected only when its eigenvalue exceeds tau, so faces with an eigenvalue
within 1e-4 (relative) of tau, or a saturated face whose last selected and
first unselected eigenvalues are that close, admit several correct row sets
and are skipped (they are counted, and most faces must be compared).
FP64 form, LOBPCG to a relative residual of 1e-8 on meshes with edges and
corners on every face (2x2x1, 2x2x2, 3x2x2).
"""
import numpy as np
import pytest
import scipy.linalg as sla

import amb_inputs as ai
from oracle import fe, levels as olv, pair as opr

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


def _ambiguous(lam, tau, cap):
    lam = np.sort(np.asarray(lam))[::-1]
    if np.any(np.abs(lam - tau) <= 1e-4 * tau):
        return True
    if lam.size > cap and lam[cap - 1] > tau and lam[cap - 1] - lam[cap] <= 1e-4 * lam[cap - 1]:
        return True
    return False


@pytest.mark.parametrize("split,sub,dpn,seed,tau", [((2, 2, 1), 4, 1, 31, 2.0), ((2, 2, 1), 3, 3, 32, 3.0),
                                                     ((2, 2, 2), 4, 1, 33, 2.0), ((2, 2, 2), 3, 3, 34, 3.0),
                                                     ((3, 2, 2), 3, 1, 35, 2.0)])
def test_pair_rows_match_oracle(B, split, sub, dpn, seed, tau):
    cap = 10
    prob = ai.toy(sub, dpn, seed, split=split, sigma=2.0, tau=tau)
    ctx = B.Context.from_problem(prob, lobpcg_tol=1e-8, lobpcg_maxit=300, max_adaptive_per_face=cap)
    rep = ctx.report()
    pairs = [p for p in rep["pairs"] if p["level"] == 1]
    lev = olv.level_one(prob)
    lev.schur()
    free = fe.free_dof_map(prob)[1]
    opairs = opr.pairs_of(lev)
    assert [(p["s"], p["t"]) for p in pairs] == [(int(s), int(t)) for s, t in opairs]
    compared, rows_compared = 0, 0
    for idx, p in enumerate(pairs):
        res = opr.solve_pair(lev, p["s"], p["t"], tau, max_per_face=cap)
        raw = ctx.export(B.X_PAIR_ROWS, 1, idx, np.uint8)
        k = p["n_rows"]
        nf = raw.size // 8 // (k + 1)
        assert raw.size == 8 * nf * (k + 1)
        rows = raw[: 8 * k * nf].view(np.float64).reshape(k, nf)
        dofs = raw[8 * k * nf:].view(np.int64)
        assert np.array_equal(dofs, free[res.face_dofs]), (p["s"], p["t"])
        # a pair converges by its residual or by Ritz values that stay put to
        # 1e-10 (relative); one that stalls short of 1e-8 stops at a residual
        # set by rounding; the rows themselves are checked by principal angles
        assert p["converged"] == 1 or p["residual"] <= 1e-5, (p["s"], p["t"], p["residual"])
        if _ambiguous(res.lam, tau, cap):
            continue
        assert p["n_selected"] == res.n_selected
        assert k == res.rows.shape[0], (p["s"], p["t"], k, res.rows.shape[0])
        compared += 1
        if k == 0:
            continue
        assert np.allclose(rows @ rows.T, np.eye(k), atol=1e-10)
        ang = sla.subspace_angles(rows.T, res.rows.T)
        assert ang.max() <= 1e-4, (p["s"], p["t"], ang.max())
        rows_compared += k
    assert compared >= 0.75 * len(pairs)
    assert rows_compared > 0
    ctx.close()
