"""Pins of the adaptive rows' face restriction (Sec. 7.2) on meshes with edges.

The paper builds each row c_l = A w_l (eq. d-def), keeps only its entries on
the face shared by the two substructures (entries on corners and on edges,
the nodes shared by three or more substructures, are dropped), and
orthonormalizes the face block by a reduced QR.  On a 2x1x1 mesh there are
no edges and every shared non-corner node is a face node, so the drop is
invisible there; the 2x2x1 and 2x2x2 decompositions below have edges (nodes
shared by 3 or 4 substructures) and box-vertex corners on every face.

The face node set is recomputed here from the partition alone, by counting
which substructures' elements touch each node, and the box-vertex corners
from the cut planes: an independent brute force of Sec. 2's classification.
Checked for every pair:
  * the row support is exactly the free dofs of the face nodes of (s, t):
    no edge, corner or Dirichlet dof, and no face dof missing;
  * the rows are orthonormal;
  * their span equals the span of the face-restricted rows c_l (principal
    angles), and their number equals that block's numerical rank.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import amb_inputs as ai
from oracle import fe, levels as lv, pair as pr


def _node_subs(prob):
    """Substructures touching every node, from elem_to_sub only."""
    nx, ny, nz = prob.nx, prob.ny, prob.nz
    subs = [set() for _ in range(prob.n_nodes)]
    sub = prob.elem_to_sub.reshape(nz, ny, nx)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                s = int(sub[k, j, i])
                for dk in (0, 1):
                    for dj in (0, 1):
                        for di in (0, 1):
                            subs[(i + di) + (nx + 1) * ((j + dj) + (ny + 1) * (k + dk))].add(s)
    return subs


def _is_box_vertex(prob, node):
    nx, ny = prob.nx, prob.ny
    i = node % (nx + 1)
    j = (node // (nx + 1)) % (ny + 1)
    k = node // ((nx + 1) * (ny + 1))
    cuts = prob.cuts[0]
    return i in set(cuts[0].tolist()) and j in set(cuts[1].tolist()) and k in set(cuts[2].tolist())


def _face_full_dofs(prob, s, t, node_subs):
    """Full-grid dofs of the free face nodes of (s, t), by brute force."""
    dpn = prob.dofs_per_node
    out = []
    for node, ss in enumerate(node_subs):
        if ss != {s, t} or prob.dirichlet_node_mask[node] or _is_box_vertex(prob, node):
            continue
        out.extend(node * dpn + c for c in range(dpn))
    return np.array(sorted(out), dtype=np.int64)


def _edge_or_corner_full_dofs(prob, node_subs):
    dpn = prob.dofs_per_node
    out = set()
    for node, ss in enumerate(node_subs):
        if prob.dirichlet_node_mask[node] or len(ss) < 2:
            continue
        if len(ss) >= 3 or _is_box_vertex(prob, node):
            out.update(node * dpn + c for c in range(dpn))
    return out


CASES = [((2, 2, 1), 4, 1, 21, 2.0), ((2, 2, 1), 3, 3, 22, 2.0),
         ((2, 2, 2), 4, 1, 23, 2.0), ((2, 2, 2), 3, 3, 24, 2.0)]


@pytest.mark.parametrize("split,sub,dpn,seed,tau", CASES)
def test_face_rows_support_orthonormality_and_span(split, sub, dpn, seed, tau):
    prob = ai.toy(sub, dpn, seed, split=split, sigma=2.0, tau=tau)
    lev = lv.level_one(prob)
    lev.schur()
    free = fe.free_dof_map(prob)[1]
    node_subs = _node_subs(prob)
    off_face = _edge_or_corner_full_dofs(prob, node_subs)
    assert off_face, "the decomposition must have edges or corners on its faces"
    pairs = pr.pairs_of(lev)
    n_rows_total, n_pairs_with_edges = 0, 0
    for (s, t) in pairs:
        res = pr.solve_pair(lev, s, t, tau)
        want = _face_full_dofs(prob, s, t, node_subs)
        got = free[res.face_dofs]
        # the support: exactly the face dofs, in increasing dof order
        assert np.array_equal(got, want), (s, t)
        assert not (set(got.tolist()) & off_face)
        # the shared dofs of (s, t) include edge or corner dofs that were dropped
        info = pr.shared_info(lev, s, t)
        f_full = free[info["f"]]
        if set(f_full.tolist()) & off_face:
            n_pairs_with_edges += 1
        if res.n_selected == 0:
            assert res.rows.shape[0] == 0
            continue
        rows = res.rows
        assert rows.shape[1] == want.size
        # orthonormal
        assert np.allclose(rows @ rows.T, np.eye(rows.shape[0]), atol=1e-12)
        # span of the face-restricted unprojected rows c_l (columns matched by full dof id)
        col = {int(d): i for i, d in enumerate(f_full)}
        blk = res.crows_full[:, [col[int(d)] for d in want]]
        sv = np.linalg.svd(blk, compute_uv=False)
        rank = int(np.sum(sv >= 1e-10 * sv.max())) if sv.size and sv.max() > 0 else 0
        assert rows.shape[0] == rank
        ang = sla.subspace_angles(rows.T, blk.T)
        assert ang.max() < 1e-8, (s, t, ang.max())
        n_rows_total += rows.shape[0]
    assert n_rows_total > 0
    assert n_pairs_with_edges == len(pairs)


def test_face_rows_differ_from_rows_that_keep_edges():
    """The edge drop changes the constraint: on a face whose shared dofs include
    edge dofs, the rows restricted to the face are not the face part of an
    orthonormal basis of the rows on all shared dofs (so a build that kept the
    edge entries would be told apart by the support test above and by the
    constraint it adds)."""
    prob = ai.toy(4, 1, 25, split=(2, 2, 1), sigma=2.0, tau=2.0)
    lev = lv.level_one(prob)
    lev.schur()
    found = False
    for (s, t) in pr.pairs_of(lev):
        res = pr.solve_pair(lev, s, t, 2.0)
        if res.n_selected == 0:
            continue
        info = pr.shared_info(lev, s, t)
        sel = np.isin(info["f"], res.face_dofs)
        if sel.all():
            continue
        full = res.crows_full
        dropped = full[:, ~sel]
        if np.abs(dropped).max() > 1e-8 * np.abs(full).max():
            found = True
    assert found
