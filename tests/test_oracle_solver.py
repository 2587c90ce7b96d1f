"""Pins of the oracle's Algorithm 1 / Algorithm 3 / PCG (Sec. 3, 6, 8):
the solution against a sparse direct solve; the spectrum of the BDDC
preconditioned operator (>= 1, and its maximum equal to the pair eigenvalue
lambda_{k+1} when there are only two substructures: Lemma 1 + Corollary 1);
one PCG iteration when every interface dof is a corner; a 3-level method
with one level-2 substructure reproducing the 2-level iterates; the Lanczos
condition estimate against the dense spectrum."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import amb_inputs as ai
from oracle import fe, solver


def _dense_precond_spectrum(h):
    n = h.levels[0].n
    m = np.column_stack([h.apply(e) for e in np.eye(n)])
    a = h.ops[0].toarray()
    ev = np.linalg.eigvals(m @ a)
    assert np.abs(ev.imag).max() < 1e-8 * np.abs(ev).max()
    return np.sort(ev.real), m


@pytest.mark.parametrize("dpn,split", [(1, (2, 1, 1)), (3, (2, 1, 1)), (1, (2, 2, 1)), (3, (2, 2, 2))])
def test_solution_vs_direct(dpn, split):
    prob = ai.toy(4 if dpn == 1 or split != (2, 2, 2) else 3, dpn, 21, split=split, sigma=1.5)
    h, res, f = solver.solve(prob, rtol=1e-10)
    ud = spla.spsolve(h.ops[0].tocsc(), f)
    assert res.rel_res <= 1e-10
    assert np.linalg.norm(res.u - ud) <= 1e-8 * np.linalg.norm(ud)
    # the oracle's global operator equals the direct FE assembly
    assert abs(h.ops[0] - fe.assemble_global(prob)).max() < 1e-12 * abs(h.ops[0]).max()


@pytest.mark.parametrize("dpn,split,adaptive", [(1, (2, 1, 1), False), (3, (2, 1, 1), True),
                                                  (1, (2, 2, 1), True), (3, (2, 2, 1), False)])
def test_spectrum_at_least_one(dpn, split, adaptive):
    prob = ai.toy(4, dpn, 31, split=split, sigma=2.0, tau=3.0)
    h = solver.Hierarchy(prob, adaptive=adaptive)
    ev, m = _dense_precond_spectrum(h)
    assert np.allclose(m, m.T, atol=1e-10 * np.abs(m).max())
    assert ev.min() >= 1.0 - 1e-10
    if split == (2, 1, 1):
        # two substructures: the pair problem is the global one, so the
        # largest eigenvalue of M A is the first eigenvalue not removed
        rep = h.reports[0] if adaptive else solver.Hierarchy(prob, adaptive=True, tau=1e30).reports[0]
        k = rep.n_selected[0]
        assert abs(ev.max() - rep.lam[0][k]) < 1e-7 * ev.max()


def test_three_levels_spectrum():
    groups = [np.array([0, 2, 4]), np.array([0, 2]), np.array([0, 1])]
    prob = ai.toy(3, 1, 41, split=(4, 2, 1), levels=3, groups=groups, sigma=1.0, tau=2.0)
    h = solver.Hierarchy(prob)
    assert len(h.levels) == 2 and h.levels[1].n_subs == 2
    ev, _ = _dense_precond_spectrum(h)
    assert ev.min() >= 1.0 - 1e-10
    f = fe.load_vector(prob)
    res = solver.pcg(h.ops[0], f, h.apply, rtol=1e-10)
    ud = spla.spsolve(h.ops[0].tocsc(), f)
    assert np.linalg.norm(res.u - ud) <= 1e-8 * np.linalg.norm(ud)


@pytest.mark.parametrize("dpn", [1, 3])
def test_all_corners_one_iteration(dpn):
    prob = ai.toy(4, dpn, 51, split=(2, 2, 1), sigma=1.0)
    h, res, f = solver.solve(prob, rtol=1e-12, initial="all_corners", adaptive=False)
    assert res.its == 1
    assert res.rel_res <= 1e-12


def test_three_levels_single_top_sub_equals_two_levels():
    groups = [np.array([0, 2]), np.array([0, 2]), np.array([0, 1])]
    prob3 = ai.toy(3, 3, 61, split=(2, 2, 1), levels=3, groups=groups, sigma=1.0)
    prob2 = ai.toy(3, 3, 61, split=(2, 2, 1), levels=2, sigma=1.0)
    h3, r3, _ = solver.solve(prob3, rtol=1e-10)
    h2, r2, _ = solver.solve(prob2, rtol=1e-10)
    assert r3.its == r2.its
    assert np.allclose(r3.history, r2.history, rtol=1e-8, atol=1e-14)


def test_lanczos_condition_estimate():
    prob = ai.toy(4, 1, 71, split=(2, 2, 1), sigma=2.0)
    h = solver.Hierarchy(prob, adaptive=False)
    ev, _ = _dense_precond_spectrum(h)
    f = fe.load_vector(prob)
    res = solver.pcg(h.ops[0], f, h.apply, rtol=1e-14, maxit=400)
    assert abs(res.cond - ev.max() / ev.min()) < 1e-3 * ev.max()


def test_lower_tau_nests_constraints_and_lowers_lambda_max():
    """Lowering tau adds rows per face (the selected eigenvectors of a higher
    tau stay selected, so the constrained spaces are nested) and can only
    lower the largest eigenvalue of M A, which is the maximum of the
    averaging energy over the constrained space (Sec. 4); the smallest stays
    >= 1.  Adaptivity on this 1e4-contrast problem lowers the PCG iteration
    count against the initial constraints alone, and rows are capped per
    face (the paper's saturation at the cap)."""
    rng = np.random.default_rng(np.random.PCG64(81))
    prob = ai.toy(4, 1, 81, split=(2, 2, 1), sigma=0.0)
    prob.coeff = np.where(rng.random(prob.coeff.size) < 0.15, 1.0e4, 1.0)
    f = fe.load_vector(prob)
    lmax, rows, its = [], [], []
    for tau in (1e30, 30.0, 6.0, 2.0):
        h = solver.Hierarchy(prob, adaptive=True, tau=tau)
        ev, _ = _dense_precond_spectrum(h)
        assert ev.min() >= 1.0 - 1e-10
        lmax.append(ev.max())
        rows.append([int(k) for k in h.reports[0].n_selected])
        its.append(solver.pcg(h.ops[0], f, h.apply, rtol=1e-8).its)
    for a, b in zip(rows, rows[1:]):
        assert all(x <= y for x, y in zip(a, b))
    assert sum(rows[-1]) > sum(rows[0]) == 0
    for a, b in zip(lmax, lmax[1:]):
        assert b <= a * (1 + 1e-9)
    assert lmax[-1] < lmax[0] and its[-1] < its[0]
    hc = solver.Hierarchy(prob, adaptive=True, tau=1.01, max_per_face=2)
    assert max(hc.reports[0].n_selected) == 2
