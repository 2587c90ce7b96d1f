"""Pairwise generalized eigenproblems and adaptive constraint rows (Sec. 4, 7.2).

For adjacent substructures s, t (sharing a face), with W^st = W^s x W^t on
the interfaces, S^st = diag(S^s, S^t) (eq. global-S), E^st the pair
average (weights from s and t only, identity off Gamma^st, Sec. 7.2),
D the jump rows of the initial coarse dofs shared by s and t and
Pi = I - D^T (D D^T)^{-1} D, eq. eig-matrix reads

    Pi (I-E)^T S (I-E) Pi w = lambda Pi S Pi w,

solved in the factor space modulo null(Pi S Pi) (eq. eig-nullspace).  On
interface coordinates (I - P^st) is the identity, energies are given by S.
The rows to add are c_l = w_l^T Pi (I-E)^T S (I-E) Pi (eq. d-def), split as
[c^s, -c^s] (Prop. 1); entries off the face are dropped and the face block
orthonormalized by a reduced QR (Sec. 7.2).

Two forms are provided:
  * `literal`: the matrices above, dense, on Gamma^s + Gamma^t;
  * `reduced`: the same eigenvalues from the jump j = w^s - w^t on the shared
    dofs f: numerator j^T N j with N = D_t S^s_ff D_t + D_s S^t_ff D_s, and
    denominator the minimal pair energy for that jump, j^T H j with
    H = parallel sum of the Schur complements of S^s, S^t onto f,
    restricted to null(C_f).
Pinned by tests/test_oracle_pair.py: literal == reduced on 2x1x1 meshes,
all shared dofs as corners gives all eigenvalues 0, Prop. 1 sign structure,
and the Courant-Fischer property of the added rows (Corollary 1).
"""
from __future__ import annotations

import dataclasses
from typing import List

import numpy as np
import scipy.linalg as sla

DROP = 1.0e-12   # relative eigenvalue drop in pseudo-inverses / factor spaces


@dataclasses.dataclass
class PairResult:
    s: int
    t: int
    lam: np.ndarray          # eigenvalues, descending (all positive ones)
    rows: np.ndarray         # (k, n_face) orthonormal adaptive rows on the face dofs
    face_dofs: np.ndarray    # level dofs of the face-class nodes
    n_selected: int
    crows_full: np.ndarray = None  # (nsel, n_f) unprojected rows on f (before dropping)


def _factor_space_eig(a, b):
    """Eigenpairs of a w = lambda b w on the complement of null(b), descending.

    Pinned by test_oracle_pair.py::test_literal_equals_reduced.
    """
    sig, v = np.linalg.eigh(0.5 * (b + b.T))
    keep = sig > DROP * max(sig.max(), 0.0)
    t = v[:, keep] / np.sqrt(sig[keep])
    m = t.T @ a @ t
    lam, y = np.linalg.eigh(0.5 * (m + m.T))
    order = np.argsort(lam)[::-1]
    return lam[order], t @ y[:, order]


def shared_info(lev, s, t):
    """Index bookkeeping of the shared dofs.  Pinned by
    test_oracle_pair.py::test_all_shared_dofs_corners_gives_zero."""
    key = (min(s, t), max(s, t))
    sbs, sbt = lev.subs[s], lev.subs[t]
    f = np.intersect1d(sbs.gdofs, sbt.gdofs)
    ps = np.array([lev.gpos[s][int(d)] for d in f], dtype=np.int64)
    pt = np.array([lev.gpos[t][int(d)] for d in f], dtype=np.int64)
    face_nodes = lev.faces.get(key, np.array([], dtype=np.int64))
    face_dofs = np.sort(np.concatenate([lev.dofs_of_node[i] for i in face_nodes]).astype(np.int64)) \
        if face_nodes.size else np.array([], dtype=np.int64)
    shared = sorted(set(sbs.rc.tolist()) & set(sbt.rc.tolist()))
    cs = np.array([sbs.c[list(sbs.rc).index(k)] for k in shared]).reshape(len(shared), sbs.n_g)
    ct = np.array([sbt.c[list(sbt.rc).index(k)] for k in shared]).reshape(len(shared), sbt.n_g)
    ks = np.diag(sbs.k)[sbs.n_i:][ps]
    kt = np.diag(sbt.k)[sbt.n_i:][pt]
    return dict(f=f, ps=ps, pt=pt, face_dofs=face_dofs, cs=cs, ct=ct,
                ds=ks / (ks + kt), dt=kt / (ks + kt))


def literal(lev, s, t):
    """Dense eq. eig-matrix on Gamma^s + Gamma^t.  Returns (lam, W, A, info).

    Pinned by test_oracle_pair.py::test_literal_equals_reduced (two independent formulations agree)
    and test_all_shared_dofs_corners_gives_zero.
    """
    info = shared_info(lev, s, t)
    sbs, sbt = lev.subs[s], lev.subs[t]
    ns, nt = sbs.n_g, sbt.n_g
    n = ns + nt
    smat = np.zeros((n, n))
    smat[:ns, :ns] = sbs.s
    smat[ns:, ns:] = sbt.s
    e = np.eye(n)
    for a, b, wsa, wtb in zip(info["ps"], info["pt"], info["ds"], info["dt"]):
        e[a, a], e[a, ns + b] = wsa, wtb
        e[ns + b, a], e[ns + b, ns + b] = wsa, wtb
    d = np.hstack([info["cs"], -info["ct"]])
    if d.shape[0]:
        pi = np.eye(n) - d.T @ np.linalg.solve(d @ d.T, d)
    else:
        pi = np.eye(n)
    ie = np.eye(n) - e
    amat = pi @ ie.T @ smat @ ie @ pi
    bmat = pi @ smat @ pi
    lam, w = _factor_space_eig(amat, bmat)
    return lam, w, amat, info


def _schur_onto(smat, keep_pos):
    """Pinned by test_oracle_pair.py::test_literal_equals_reduced."""
    n = smat.shape[0]
    other = np.setdiff1d(np.arange(n), keep_pos)
    sff = smat[np.ix_(keep_pos, keep_pos)]
    if other.size == 0:
        return sff
    soo = smat[np.ix_(other, other)]
    sof = smat[np.ix_(other, keep_pos)]
    return sff - sof.T @ sla.cho_solve(sla.cho_factor(soo, lower=True), sof)


def _pinv_psd(m):
    """Pinned by test_oracle_pair.py::test_literal_equals_reduced."""
    sig, v = np.linalg.eigh(0.5 * (m + m.T))
    keep = sig > DROP * max(sig.max(), 0.0)
    return (v[:, keep] / sig[keep]) @ v[:, keep].T


def reduced(lev, s, t):
    """Same positive eigenvalues as `literal`, from the jump on the shared dofs.
    Returns (lam, J, N, info) with J the jumps (columns) of the eigenvectors,
    normalized so that j^T H j = 1.

    Pinned by test_oracle_pair.py::test_literal_equals_reduced.
    """
    info = shared_info(lev, s, t)
    sbs, sbt = lev.subs[s], lev.subs[t]
    ps, pt, ds, dt = info["ps"], info["pt"], info["ds"], info["dt"]
    nmat = (dt[:, None] * sbs.s[np.ix_(ps, ps)] * dt[None, :]
            + ds[:, None] * sbt.s[np.ix_(pt, pt)] * ds[None, :])
    hs = _schur_onto(sbs.s, ps)
    ht = _schur_onto(sbt.s, pt)
    hmat = hs - hs @ _pinv_psd(hs + ht) @ hs
    cf = info["cs"][:, ps] if info["cs"].shape[0] else np.zeros((0, ps.size))
    z = sla.null_space(cf) if cf.shape[0] else np.eye(ps.size)
    lam, y = _factor_space_eig(z.T @ nmat @ z, z.T @ hmat @ z)
    info["cf"] = cf
    return lam, z @ y, nmat, info


def rows_from_reduced(nmat, jumps, info):
    """c^s on f: P_C N j, with P_C the orthogonal projector onto null(C_f).

    Pinned by test_oracle_pair.py::test_prop1_sign_structure and test_corollary1_added_rows.
    """
    c = nmat @ jumps
    cf = info["cf"]
    if cf.shape[0]:
        c = c - cf.T @ np.linalg.solve(cf @ cf.T, cf @ c)
    return c.T


def face_rows(crows_f, info, lev):
    """Drop entries off the face-class dofs, orthonormalize (reduced QR).

    Pinned by test_oracle_face_rows.py (2x2x1 and 2x2x2 meshes, whose faces
    border edges and corners): the support equals the face nodes' free dofs
    found by brute force from the partition, the rows are orthonormal and
    span the face-restricted c_l; and by test_oracle_pair.py::test_corollary1_added_rows.
    """
    f = info["f"]
    face_dofs = info["face_dofs"]
    sel = np.isin(f, face_dofs)
    blk = crows_f[:, sel]                        # (k, n_face) in the order of f[sel]
    fd = f[sel]
    if blk.shape[0] == 0:
        return np.zeros((0, fd.size)), fd
    q, r = np.linalg.qr(blk.T, mode="reduced")
    dg = np.abs(np.diag(r))
    keep = dg >= 1.0e-10 * dg.max() if dg.size and dg.max() > 0 else np.zeros(dg.size, bool)
    return q[:, keep].T, fd


def solve_pair(lev, s, t, tau, max_per_face=10, form="reduced") -> PairResult:
    """Pinned by test_oracle_pair.py::test_corollary1_added_rows (after the k rows the pair maximum
    is lambda_{k+1})."""
    if form == "literal":
        lam, w, amat, info = literal(lev, s, t)
        pos = lam > 0
        lam, w = lam[pos], w[:, pos]
        nsel = int(min(max_per_face, np.sum(lam > tau)))
        c = (amat @ w[:, :nsel]).T                   # rows on Gamma^s + Gamma^t
        crows_f = c[:, info["ps"]]                   # s-copy on f
    else:
        lam, jumps, nmat, info = reduced(lev, s, t)
        pos = lam > 0
        lam, jumps = lam[pos], jumps[:, pos]
        nsel = int(min(max_per_face, np.sum(lam > tau)))
        crows_f = rows_from_reduced(nmat, jumps[:, :nsel], info)
    rows, fd = face_rows(crows_f, info, lev)
    return PairResult(s=s, t=t, lam=lam, rows=rows, face_dofs=fd, n_selected=nsel,
                      crows_full=crows_f)


def pairs_of(lev) -> List[tuple]:
    """Every pair sharing at least one face-class dof.

    Pinned by test_oracle_levels.py::test_classification_counts_2x2x2 (12 faces).
    """
    return sorted(k for k, nodes in lev.faces.items() if nodes.size)
