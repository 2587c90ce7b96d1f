"""Pins of the pair eigenproblem (Sec. 4, eq. eig-matrix, d-def, Prop. 1,
Corollary 1) on 2x1x1 meshes, where it can be brute-forced densely."""
import numpy as np
import pytest

import amb_inputs as ai
from oracle import levels as lv, pair as pr


def _level(prob, initial="ce"):
    lev = lv.level_one(prob, initial)
    lev.schur()
    return lev


@pytest.mark.parametrize("sub,dpn,seed", [(4, 1, 1), (4, 3, 2), (6, 1, 3), (5, 3, 4)])
def test_literal_equals_reduced(sub, dpn, seed):
    prob = ai.toy(sub, dpn, seed, sigma=1.5)
    lev = _level(prob)
    lam_l, _, _, _ = pr.literal(lev, 0, 1)
    lam_r, _, _, _ = pr.reduced(lev, 0, 1)
    lam_l = lam_l[lam_l > 1e-9 * lam_l.max()]
    lam_r = lam_r[lam_r > 1e-9 * lam_r.max()]
    assert lam_l.size == lam_r.size
    assert np.allclose(lam_l, lam_r, rtol=1e-8)


def test_literal_equals_reduced_2x2x1():
    prob = ai.toy(4, 3, 9, split=(2, 2, 1), sigma=1.0)
    lev = _level(prob)
    for (s, t) in pr.pairs_of(lev):
        lam_l = pr.literal(lev, s, t)[0]
        lam_r = pr.reduced(lev, s, t)[0]
        lam_l = lam_l[lam_l > 1e-9 * lam_l.max()]
        lam_r = lam_r[lam_r > 1e-9 * lam_r.max()]
        assert np.allclose(lam_l, lam_r, rtol=1e-8)


def test_all_shared_dofs_corners_gives_zero():
    prob = ai.toy(4, 3, 5)
    lev = _level(prob, initial="all_corners")
    lam, _, amat, _ = pr.literal(lev, 0, 1)
    assert np.abs(amat).max() < 1e-12
    assert np.abs(lam).max() < 1e-10


@pytest.mark.parametrize("dpn", [1, 3])
def test_prop1_sign_structure(dpn):
    prob = ai.toy(4, dpn, 6, sigma=2.0, split=(2, 2, 1))
    lev = _level(prob)
    lam, w, amat, info = pr.literal(lev, 0, 1)
    ns = lev.subs[0].n_g
    c = amat @ w[:, :3]
    cs, ct = c[:ns], c[ns:]
    assert np.allclose(cs[info["ps"]], -ct[info["pt"]], atol=1e-10 * np.abs(c).max())
    off_s = np.setdiff1d(np.arange(ns), info["ps"])
    assert off_s.size > 0
    assert np.abs(cs[off_s]).max() < 1e-10 * np.abs(c).max()
    # the reduced rows agree with the literal ones on f
    lam_r, jumps, nmat, info_r = pr.reduced(lev, 0, 1)
    cr = pr.rows_from_reduced(nmat, jumps[:, :3], info_r)
    for k in range(3):
        a, b = cs[info["ps"], k], cr[k]
        assert min(np.abs(a - b).max(), np.abs(a + b).max()) < 1e-7 * np.abs(a).max()


@pytest.mark.parametrize("dpn,tau", [(1, 3.0), (3, 3.0)])
def test_corollary1_added_rows(dpn, tau):
    """After adding the rows of the k largest eigenvalues, the largest
    eigenvalue of the constrained pair problem is lambda_{k+1}."""
    prob = ai.toy(4, dpn, 8, sigma=2.0, tau=tau)
    lev = _level(prob)
    res = pr.solve_pair(lev, 0, 1, tau, form="literal")
    k = res.n_selected
    assert k >= 1
    lev.add_adaptive(0, 1, res.face_dofs, res.rows)
    lev.coarse_basis()
    lam2 = pr.literal(lev, 0, 1)[0]
    assert abs(lam2[0] - res.lam[k]) < 1e-8 * res.lam[0]
