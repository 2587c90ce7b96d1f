"""Set-up of Adaptive-Multilevel BDDC (Algorithm 3), the Multilevel BDDC
preconditioner (Algorithm 1) and PCG with the Lanczos condition estimate.

Algorithm 1 is applied literally on the full level spaces U_i (interiors
included): interior pre-correction (eq. ML-uIi), residual update
(eq. ML-rBi), substructure correction on W_Delta (eq. ML-wDi) as the
local Neumann problem with the coarse dofs fixed to zero, coarse right-hand
side (eq. ML-coarse, ML-ri+1), recursion, averaging (eq. ML-uBi-1),
interior post-correction (eq. ML-vIi) and the combined update (eq. ML-ui).
The top-level coarse problem is solved directly (dense Cholesky).

PCG (Sec. 8): u_0 = 0, stop at ||r_k||_2 <= rtol ||f||_2 (recursive r); the
condition estimate uses the extreme eigenvalues of the CG tridiagonal with
diagonal 1/alpha_k + beta_{k-1}/alpha_{k-1} and off-diagonal
sqrt(beta_k)/alpha_k.

Pinned by tests/test_oracle_solver.py: the solution against a sparse direct
solve, eigenvalues of the preconditioned operator >= 1, one-iteration
convergence when every interface dof is a corner, the 3-level method with a
single level-2 substructure reproducing the 2-level iterates, and the
Lanczos estimate against dense eigenvalues of the preconditioned operator.
"""
from __future__ import annotations

import dataclasses
import time
from typing import List

import numpy as np
import scipy.linalg as sla

from . import fe, levels as lv, pair as pr


@dataclasses.dataclass
class LevelReport:
    pairs: List[tuple]
    lam: List[np.ndarray]
    n_selected: List[int]
    omega_tilde: float         # max over pairs of lambda_{k+1} (after selection)
    n_adaptive: int


class Hierarchy:
    def __init__(self, prob, levels=None, tau=None, initial="ce", adaptive=True,
                 max_per_face=10, form="reduced", timers=None):
        """Algorithm 3.  Pinned by test_oracle_solver.py::test_solution_vs_direct,
        test_spectrum_at_least_one and test_three_levels_spectrum."""
        self.prob = prob
        self.nlev = prob.levels if levels is None else levels
        self.tau = prob.tau if tau is None else tau
        self.timers = {} if timers is None else timers
        self.levels: List[lv.Level] = []
        self.reports: List[LevelReport] = []
        t0 = time.perf_counter()
        lev = lv.level_one(prob, initial)
        self._tick("assembly", t0)
        for i in range(self.nlev - 1):
            t0 = time.perf_counter()
            lev.schur()
            self._tick("factor", t0)
            t0 = time.perf_counter()
            rep = self._adapt(lev, max_per_face, form) if adaptive else None
            self._tick("eigen", t0)
            t0 = time.perf_counter()
            lev.coarse_basis()
            self._tick("coarse", t0)
            self.levels.append(lev)
            self.reports.append(rep)
            if i < self.nlev - 2:
                t0 = time.perf_counter()
                lev = lv.level_next(lev, prob.sub_to_parent[i], prob.n_subs(i + 2),
                                    prob.cuts[i + 1], initial)
                self._tick("assembly", t0)
        t0 = time.perf_counter()
        self.ops = [l.operator() for l in self.levels]
        for l in self.levels:
            for sb in l.subs:
                ni = sb.n_i
                if ni:
                    ext = -sla.cho_solve(sb.aii_cho, sb.k[:ni, ni:] @ sb.psi)
                else:
                    ext = np.zeros((0, sb.psi.shape[1]))
                sb.phi = np.vstack([ext, sb.psi])
        self.top = sla.cho_factor(self.levels[-1].coarse_matrix(), lower=True)
        self._tick("coarse", t0)

    def _tick(self, key, t0):
        """Timing bookkeeping only."""
        self.timers[key] = self.timers.get(key, 0.0) + time.perf_counter() - t0

    def _adapt(self, lev, max_per_face, form) -> LevelReport:
        """Pinned by test_oracle_solver.py::test_spectrum_at_least_one (adaptive) and
        test_oracle_pair.py::test_corollary1_added_rows."""
        pairs = pr.pairs_of(lev)
        lams, nsel, after = [], [], []
        results = []
        for (s, t) in pairs:
            res = pr.solve_pair(lev, s, t, self.tau, max_per_face, form)
            results.append(res)
            lams.append(res.lam)
            nsel.append(res.n_selected)
            k = res.n_selected
            after.append(res.lam[k] if k < res.lam.size else 0.0)
        n_ad = 0
        for res in results:
            if res.rows.shape[0]:
                lev.add_adaptive(res.s, res.t, res.face_dofs, res.rows)
                n_ad += res.rows.shape[0]
        return LevelReport(pairs=pairs, lam=lams, n_selected=nsel,
                           omega_tilde=max(after) if after else 0.0, n_adaptive=n_ad)

    # ------------------------------------------------------------ Algorithm 1
    def apply(self, r: np.ndarray, i: int = 0) -> np.ndarray:
        """Algorithm 1.  Pinned by test_oracle_solver.py::test_spectrum_at_least_one (spectrum of M
        A >= 1), test_all_corners_one_iteration and
        test_three_levels_single_top_sub_equals_two_levels."""
        lev, a = self.levels[i], self.ops[i]
        u_i = np.zeros(lev.n)
        for sb in lev.subs:
            if sb.n_i:
                u_i[sb.idofs] = sla.cho_solve(sb.aii_cho, r[sb.idofs])       # eq. ML-uIi
        r_b = r - a @ u_i                                                      # eq. ML-rBi
        g = lev.average_transpose(r_b)
        w, r_next = [], np.zeros(lev.n_coarse)
        for sb, gs in zip(lev.subs, g):
            nc = sb.rc.size
            sol = sla.lu_solve(sb.neumann_lu, np.concatenate([gs, np.zeros(nc)]))
            w.append(sol[:sb.dofs.size])                                       # eq. ML-wDi
            np.add.at(r_next, sb.rc, sb.phi.T @ gs)                            # eq. ML-ri+1
        if i == len(self.levels) - 1:
            u_c = sla.cho_solve(self.top, r_next)
        else:
            u_c = self.apply(r_next, i + 1)
        z = [ws + sb.phi @ u_c[sb.rc] for ws, sb in zip(w, lev.subs)]
        u_b = lev.average(z)                                                   # eq. ML-uBi-1
        t = a @ u_b
        v_i = np.zeros(lev.n)
        for sb in lev.subs:
            if sb.n_i:
                v_i[sb.idofs] = sla.cho_solve(sb.aii_cho, t[sb.idofs])         # eq. ML-vIi
        return u_i + u_b - v_i                                                 # eq. ML-ui

    def report(self):
        """Bookkeeping only (no arithmetic)."""
        return self.reports


@dataclasses.dataclass
class PCGResult:
    u: np.ndarray
    its: int
    rel_res: float
    alphas: np.ndarray
    betas: np.ndarray
    cond: float
    history: np.ndarray


def lanczos_cond(alphas, betas) -> float:
    """Pinned by test_oracle_solver.py::test_lanczos_condition_estimate."""
    k = len(alphas)
    if k == 0:
        return 1.0
    d = np.empty(k)
    e = np.empty(max(k - 1, 0))
    for j in range(k):
        d[j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j < k - 1:
            e[j] = np.sqrt(betas[j]) / alphas[j]
    ev = sla.eigh_tridiagonal(d, e, eigvals_only=True)
    return float(ev.max() / ev.min())


def pcg(a, f, precond, rtol=1e-8, maxit=1000) -> PCGResult:
    """Pinned by test_oracle_solver.py::test_solution_vs_direct."""
    u = np.zeros_like(f)
    r = f.copy()
    nf = np.linalg.norm(f)
    hist = [1.0]
    alphas, betas = [], []
    if nf == 0:
        return PCGResult(u, 0, 0.0, np.array([]), np.array([]), 1.0, np.array(hist))
    z = precond(r)
    p = z.copy()
    rz = r @ z
    its = 0
    while its < maxit:
        q = a @ p
        alpha = rz / (p @ q)
        u += alpha * p
        r -= alpha * q
        its += 1
        alphas.append(alpha)
        rel = np.linalg.norm(r) / nf
        hist.append(rel)
        if rel <= rtol:
            break
        z = precond(r)
        rz_new = r @ z
        beta = rz_new / rz
        betas.append(beta)
        p = z + beta * p
        rz = rz_new
    return PCGResult(u, its, hist[-1], np.array(alphas), np.array(betas),
                     lanczos_cond(alphas, betas), np.array(hist))


def solve(prob, rtol=1e-8, **kw):
    """Set-up + PCG on the level-1 problem; returns (hierarchy, PCGResult, f).

    Pinned by test_oracle_solver.py::test_solution_vs_direct.
    """
    h = Hierarchy(prob, **kw)
    f = fe.load_vector(prob)
    t0 = time.perf_counter()
    res = pcg(h.ops[0], f, h.apply, rtol=rtol)
    h._tick("pcg", t0)
    return h, res, f
