"""Pins of the non-adaptive and fixed-count variants of Sec. 8.2 (Table 6):
"c+e+f", corners plus arithmetic averages over every edge and every face as
the initial constraints, and "3eigv", three adaptive constraints per face in
place of the three face averages.

  * The face averages are one row per face and component, 1/n on exactly the
    free dofs of the face's nodes (found here by brute force from the
    partition: nodes touched by the elements of exactly the two substructures,
    box vertices and Dirichlet nodes removed).
  * More constraints cannot raise lambda_max(M A): the constrained spaces are
    nested (c+e+f inside c+e inside c), and lambda_max(M A) is the largest
    averaging energy over that space (Sec. 2, eq. def-omega); the spectrum
    stays >= 1.
  * With two substructures the pair problem is the global one (Lemma 1 and
    Corollary 1): lambda_max(M A) equals the first eigenvalue of the pair
    problem whose jump constraints D include the face averages; with "3eigv"
    it equals the pair problem's fourth eigenvalue.
"""
import numpy as np
import pytest

import amb_inputs as ai
from oracle import fe, levels as lv, pair as pr, solver
from test_oracle_face_rows import _face_full_dofs, _node_subs


def _precond_spectrum(h):
    n = h.levels[0].n
    m = np.column_stack([h.apply(e) for e in np.eye(n)])
    ev = np.linalg.eigvals(m @ h.ops[0].toarray())
    assert np.abs(ev.imag).max() < 1e-8 * np.abs(ev).max()
    return np.sort(ev.real)


@pytest.mark.parametrize("split,sub,dpn,seed", [((2, 2, 1), 4, 1, 51), ((2, 2, 1), 3, 3, 52), ((2, 2, 2), 3, 1, 53)])
def test_face_average_rows(split, sub, dpn, seed):
    prob = ai.toy(sub, dpn, seed, split=split, sigma=1.0)
    lev = lv.level_one(prob, "cef")
    free = fe.free_dof_map(prob)[1]
    node_subs = _node_subs(prob)
    faces = [ob for ob in lev.objects if ob.kind == "face"]
    assert len(faces) == len(pr.pairs_of(lev))
    for ob in faces:
        s, t = ob.subs
        want = _face_full_dofs(prob, s, t, node_subs)
        got = np.sort(np.concatenate([free[d] for d in ob.dofs]))
        assert np.array_equal(got, want)
        assert len(ob.dofs) == dpn
        for d, w, c in zip(ob.dofs, ob.weights, ob.comps):
            assert np.all(free[d] % dpn == c)
            assert np.allclose(w, 1.0 / d.size)
    # every substructure carries one row per component of each of its faces
    ce = lv.level_one(prob, "ce")
    for s, (sb, sb_ce) in enumerate(zip(lev.subs, ce.subs)):
        nf = sum(1 for ob in faces if s in ob.subs)
        assert sb.c.shape[0] == sb_ce.c.shape[0] + nf * dpn


@pytest.mark.parametrize("split,sub,dpn,seed", [((2, 2, 1), 4, 1, 54), ((2, 2, 1), 3, 3, 55)])
def test_more_constraints_cannot_raise_lambda_max(split, sub, dpn, seed):
    prob = ai.toy(sub, dpn, seed, split=split, sigma=2.0)
    top = {}
    for initial in ("c", "ce", "cef"):
        ev = _precond_spectrum(solver.Hierarchy(prob, adaptive=False, initial=initial))
        assert ev.min() >= 1.0 - 1e-10
        top[initial] = ev.max()
    assert top["cef"] <= top["ce"] * (1 + 1e-10) and top["ce"] <= top["c"] * (1 + 1e-10)
    assert top["cef"] < top["ce"]      # the face averages do remove energy here


@pytest.mark.parametrize("dpn", [1, 3])
def test_two_substructures_lambda_max_is_the_pair_eigenvalue(dpn):
    prob = ai.toy(4 if dpn == 1 else 3, dpn, 56, sigma=2.0)
    # c+e+f, no adaptive rows: the face averages are in the pair's D
    h = solver.Hierarchy(prob, adaptive=False, initial="cef")
    lam = pr.literal(h.levels[0], 0, 1)[0]
    assert abs(_precond_spectrum(h).max() - lam.max()) < 1e-7 * lam.max()
    # 3eigv: c+e and the three leading pair eigenvectors of every face
    h3 = solver.Hierarchy(prob, adaptive=True, initial="ce", tau=1e-9, max_per_face=3)
    rep = h3.reports[0]
    assert rep.n_selected == [3]
    assert abs(_precond_spectrum(h3).max() - rep.lam[0][3]) < 1e-7 * rep.lam[0][3]
