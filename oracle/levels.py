"""One decomposition level of (Adaptive-)Multilevel BDDC, dense FP64.

Follows the paper's definitions:
  * Sec. 2: nodes shared by >= 2 substructures form the interface Gamma; a
    face is the set of nodes shared by the same two substructures, an edge
    the nodes shared by the same set of more than two.  Corners are chosen
    by the box-vertex rule: interface nodes whose three coordinates each lie
    on a cut plane of the partition or on the domain boundary (the paper
    cites a face-based corner algorithm it does not describe, Sec. 7.1).
  * Sec. 7.1: initial constraints = corners + arithmetic edge averages.
  * Sec. 7 (stiffness scaling): the averaging weights are proportional to
    the diagonal of the substructure matrices before interior elimination.
  * Sec. 5 eq. local_saddle_point_problem: the coarse basis Psi^s and mu^s
    from [S C^T; C 0][Psi; mu] = [0; I]; coarse element matrix -mu^s.
  * Sec. 3: level-(i+1) elements are level-i substructures with these
    coarse matrices, level-(i+1) dofs are level-i coarse dofs.

Pinned by tests/test_oracle_levels.py (S^s null spaces, C Psi = I,
Psi^T S Psi = -mu, E^2 = E and the partition of unity, the coarse matrix
being SPD with Dirichlet data) and, end to end, by the solver pins.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional, Tuple

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import fe


@dataclasses.dataclass
class CoarseObject:
    kind: str                    # 'corner' | 'edge' | 'adaptive'
    subs: Tuple[int, ...]        # substructures that share it
    dofs: List[np.ndarray]       # per coarse dof: level dofs of its functional
    weights: List[np.ndarray]    # per coarse dof: weights of its functional
    comps: List[int]             # per coarse dof: component (-1 for adaptive)
    node: int = -1               # corner: level node id
    coord: Optional[np.ndarray] = None  # corner: mesh coordinates (element units)
    first: int = -1              # global id of its first coarse dof


@dataclasses.dataclass
class Sub:
    dofs: np.ndarray             # level dofs, ordered [interior, interface]
    n_i: int
    k: np.ndarray                # dense local matrix in that order
    c: np.ndarray = None         # constraint rows on the interface block
    rc: np.ndarray = None        # global coarse id of each row of c
    w: np.ndarray = None         # stiffness-scaling weights on the interface block
    s: np.ndarray = None         # Schur complement on the interface
    psi: np.ndarray = None       # coarse basis on the interface
    mu: np.ndarray = None
    ac: np.ndarray = None        # coarse element matrix Psi^T S Psi
    aii_cho: tuple = None
    neumann_lu: tuple = None

    @property
    def n_g(self) -> int:
        return self.dofs.size - self.n_i

    @property
    def gdofs(self) -> np.ndarray:
        return self.dofs[self.n_i:]

    @property
    def idofs(self) -> np.ndarray:
        return self.dofs[:self.n_i]


class Level:
    """Substructuring of one level given its elements and nodes."""

    def __init__(self, n, elem_dofs, elem_mat, elem_sub, n_subs, node_of_dof, comp_of_dof,
                 node_eligible, node_vertex, node_coord=None, initial="ce"):
        """Pinned through its steps below."""
        self.n = n
        self.elem_dofs = elem_dofs          # list of int arrays (-1 = absent dof)
        self.elem_mat = elem_mat            # callable e -> dense matrix
        self.elem_sub = np.asarray(elem_sub)
        self.n_subs = n_subs
        self.node_of_dof = np.asarray(node_of_dof)
        self.comp_of_dof = np.asarray(comp_of_dof)
        self.n_nodes = len(node_eligible)
        self.node_eligible = np.asarray(node_eligible, dtype=bool)
        self.node_vertex = np.asarray(node_vertex, dtype=bool)
        self.node_coord = node_coord
        self.initial = initial
        self._classify()
        self._local_matrices()
        self._initial_constraints()
        self._weights()

    # ---------------------------------------------------------------- Sec. 2
    def _classify(self):
        """Sec. 2 classification.  Pinned by test_oracle_levels.py::test_classification_counts_2x2x2
        (the paper's 12 faces of the 2x2x2 decomposition, Table 1) and
        test_box_vertex_corners_ragged_and_level_two (corner counts from the cut planes)."""
        rows, cols = [], []
        for e, d in enumerate(self.elem_dofs):
            d = d[d >= 0]
            nodes = np.unique(self.node_of_dof[d])
            rows.append(nodes)
            cols.append(np.full(nodes.size, self.elem_sub[e]))
        rows = np.concatenate(rows)
        cols = np.concatenate(cols)
        ns = sp.coo_matrix((np.ones(rows.size), (rows, cols)),
                           shape=(self.n_nodes, self.n_subs)).tocsr()
        ns.data[:] = 1.0
        ns.sum_duplicates()
        ns.data[:] = 1.0
        self.node_subs = [tuple(ns.indices[ns.indptr[i]:ns.indptr[i + 1]]) for i in range(self.n_nodes)]
        cnt = np.diff(ns.indptr)
        has_dof = np.zeros(self.n_nodes, dtype=bool)
        has_dof[self.node_of_dof] = True
        self.node_interface = (cnt >= 2) & has_dof
        if self.initial == "all_corners":
            self.node_corner = self.node_interface.copy()
        else:
            self.node_corner = self.node_interface & self.node_eligible & self.node_vertex
        groups: Dict[tuple, list] = {}
        for i in np.nonzero(self.node_interface & ~self.node_corner)[0]:
            groups.setdefault(self.node_subs[i], []).append(i)
        self.edges = {k: np.array(v) for k, v in groups.items() if len(k) >= 3}
        self.faces = {k: np.array(v) for k, v in groups.items() if len(k) == 2}
        self.dofs_of_node = [[] for _ in range(self.n_nodes)]
        for d in range(self.n):
            self.dofs_of_node[self.node_of_dof[d]].append(d)

    def _local_matrices(self):
        """Pinned by test_oracle_levels.py::test_floating_schur_null_space (rigid modes of a
        floating substructure)."""
        elems_of_sub = [[] for _ in range(self.n_subs)]
        for e in range(len(self.elem_dofs)):
            elems_of_sub[self.elem_sub[e]].append(e)
        iface_dof = self.node_interface[self.node_of_dof]
        self.subs: List[Sub] = []
        for s in range(self.n_subs):
            dl = np.unique(np.concatenate([self.elem_dofs[e] for e in elems_of_sub[s]]))
            dl = dl[dl >= 0]
            inter = dl[~iface_dof[dl]]
            gam = dl[iface_dof[dl]]
            order = np.concatenate([inter, gam])
            pos = -np.ones(self.n, dtype=np.int64)
            pos[order] = np.arange(order.size)
            k = np.zeros((order.size, order.size))
            for e in elems_of_sub[s]:
                d = self.elem_dofs[e]
                m = self.elem_mat(e)
                keep = d >= 0
                loc = pos[d[keep]]
                k[np.ix_(loc, loc)] += m[np.ix_(keep, keep)]
            self.subs.append(Sub(dofs=order, n_i=inter.size, k=0.5 * (k + k.T)))
        self.gpos = []   # per sub: level dof -> position in its interface block
        for sb in self.subs:
            g = {int(d): i for i, d in enumerate(sb.gdofs)}
            self.gpos.append(g)

    # ---------------------------------------------------------------- Sec. 7.1
    def _initial_constraints(self):
        """Sec. 7.1 corners + edge averages ("ce"); corners only ("c"); or, for
        the non-adaptive variant of Sec. 8.2 (Table 6, "c+e+f"), corners +
        arithmetic averages over every edge and every face, per component
        ("cef").  Pinned by test_oracle_levels.py::test_coarse_basis_identities
        (C Psi = I), test_oracle_solver.py::test_all_corners_one_iteration and
        test_oracle_face_averages.py (the face rows against the face nodes found
        by brute force; more constraints cannot raise lambda_max(M A))."""
        self.objects: List[CoarseObject] = []
        for i in np.nonzero(self.node_corner)[0]:
            dofs = self.dofs_of_node[i]
            coord = None if self.node_coord is None else self.node_coord[i]
            self.objects.append(CoarseObject(
                kind="corner", subs=self.node_subs[i], node=int(i), coord=coord,
                dofs=[np.array([d]) for d in dofs], weights=[np.ones(1) for _ in dofs],
                comps=[int(self.comp_of_dof[d]) for d in dofs]))
        groups = []
        if self.initial in ("ce", "cef"):
            groups += [("edge", key, self.edges[key]) for key in sorted(self.edges)]
        if self.initial == "cef":
            groups += [("face", key, self.faces[key]) for key in sorted(self.faces)]
        for kind, key, nodes in groups:
            alld = np.concatenate([self.dofs_of_node[i] for i in nodes]).astype(np.int64)
            comps = self.comp_of_dof[alld]
            if np.any(comps < 0):
                raise ValueError(f"scalar coarse dofs on an {kind}")
            dl, wl, cl = [], [], []
            for c in sorted(set(comps.tolist())):
                dd = np.sort(alld[comps == c])
                dl.append(dd)
                wl.append(np.full(dd.size, 1.0 / dd.size))
                cl.append(int(c))
            self.objects.append(CoarseObject(kind=kind, subs=key, dofs=dl, weights=wl, comps=cl))
        self._number_coarse()

    def _number_coarse(self):
        """Pinned by test_oracle_levels.py::test_coarse_basis_identities."""
        n = 0
        for ob in self.objects:
            ob.first = n
            n += len(ob.dofs)
        self.n_coarse = n
        for s, sb in enumerate(self.subs):
            rows, ids = [], []
            for ob in self.objects:
                if s not in ob.subs:
                    continue
                for q in range(len(ob.dofs)):
                    r = np.zeros(sb.n_g)
                    for d, wt in zip(ob.dofs[q], ob.weights[q]):
                        r[self.gpos[s][int(d)]] += wt
                    rows.append(r)
                    ids.append(ob.first + q)
            sb.c = np.array(rows).reshape(len(rows), sb.n_g)
            sb.rc = np.array(ids, dtype=np.int64)

    def add_adaptive(self, s: int, t: int, face_dofs: np.ndarray, rows: np.ndarray):
        """Append adaptive rows (functionals on the face dofs shared by s, t).

        Pinned by test_oracle_pair.py::test_corollary1_added_rows.
        """
        for r in rows:
            self.objects.append(CoarseObject(kind="adaptive", subs=(min(s, t), max(s, t)),
                                             dofs=[np.asarray(face_dofs)], weights=[np.asarray(r)],
                                             comps=[-1]))

    # ---------------------------------------------------------------- Sec. 7
    def _weights(self):
        """Pinned by test_oracle_levels.py::test_averaging_is_projection_onto_U (partition of
        unity)."""
        diag_sum = np.zeros(self.n)
        for sb in self.subs:
            np.add.at(diag_sum, sb.gdofs, np.diag(sb.k)[sb.n_i:])
        for sb in self.subs:
            sb.w = np.diag(sb.k)[sb.n_i:] / diag_sum[sb.gdofs]

    # ---------------------------------------------------------------- Sec. 2, 5
    def schur(self):
        """Pinned by test_oracle_levels.py::test_floating_schur_null_space."""
        for sb in self.subs:
            ni = sb.n_i
            kii, kig, kgg = sb.k[:ni, :ni], sb.k[:ni, ni:], sb.k[ni:, ni:]
            if ni:
                sb.aii_cho = sla.cho_factor(kii, lower=True)
                sb.s = kgg - kig.T @ sla.cho_solve(sb.aii_cho, kig)
            else:
                sb.s = kgg.copy()
            sb.s = 0.5 * (sb.s + sb.s.T)

    def coarse_basis(self):
        """eq. local_saddle_point_problem; coarse element matrices Psi^T S Psi = -mu.

        Pinned by test_oracle_levels.py::test_coarse_basis_identities (C Psi = I, Psi^T S Psi =
        -mu).
        """
        self._number_coarse()
        for sb in self.subs:
            nc, ng = sb.c.shape
            sad = np.zeros((ng + nc, ng + nc))
            sad[:ng, :ng] = sb.s
            sad[:ng, ng:] = sb.c.T
            sad[ng:, :ng] = sb.c
            rhs = np.zeros((ng + nc, nc))
            rhs[ng:] = np.eye(nc)
            sol = sla.solve(sad, rhs)
            sb.psi, sb.mu = sol[:ng], sol[ng:]
            ac = sb.psi.T @ sb.s @ sb.psi
            sb.ac = 0.5 * (ac + ac.T)
            # local Neumann problem on the whole substructure with the coarse dofs fixed
            n = sb.dofs.size
            kn = np.zeros((n + nc, n + nc))
            kn[:n, :n] = sb.k
            kn[n:, sb.n_i:n] = sb.c
            kn[sb.n_i:n, n:] = sb.c.T
            sb.neumann_lu = sla.lu_factor(kn)

    def coarse_matrix(self) -> np.ndarray:
        """Pinned by test_oracle_solver.py::test_three_levels_single_top_sub_equals_two_levels."""
        a = np.zeros((self.n_coarse, self.n_coarse))
        for sb in self.subs:
            a[np.ix_(sb.rc, sb.rc)] += sb.ac
        return 0.5 * (a + a.T)

    def operator(self) -> sp.csr_matrix:
        """The level problem's matrix, assembled from its elements.

        Pinned by test_oracle_solver.py::test_three_levels_spectrum and test_solution_vs_direct.
        """
        rows, cols, vals = [], [], []
        for e, d in enumerate(self.elem_dofs):
            keep = d >= 0
            dd = d[keep]
            m = self.elem_mat(e)[np.ix_(keep, keep)]
            rows.append(np.repeat(dd, dd.size))
            cols.append(np.tile(dd, dd.size))
            vals.append(m.ravel())
        a = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(self.n, self.n)).tocsr()
        return 0.5 * (a + a.T)

    # ---------------------------------------------------------------- E operator
    def average(self, z: List[np.ndarray]) -> np.ndarray:
        """E: W -> U.  Interface dofs get the weighted average of the
        substructure values, interior dofs keep their (unique) value.

        Pinned by test_oracle_levels.py::test_averaging_is_projection_onto_U (E U = U, E^2 = E).
        """
        u = np.zeros(self.n)
        for sb, zs in zip(self.subs, z):
            u[sb.idofs] = zs[:sb.n_i]
            np.add.at(u, sb.gdofs, sb.w * zs[sb.n_i:])
        return u

    def average_transpose(self, r: np.ndarray) -> List[np.ndarray]:
        """E^T.  Pinned by test_oracle_solver.py::test_spectrum_at_least_one (a wrong transpose
        breaks symmetry and the lower bound 1)."""
        out = []
        for sb in self.subs:
            g = np.empty(sb.dofs.size)
            g[:sb.n_i] = r[sb.idofs]
            g[sb.n_i:] = sb.w * r[sb.gdofs]
            out.append(g)
        return out


# -------------------------------------------------------------------- builders

def level_one(prob, initial="ce") -> Level:
    """Pinned by test_oracle_levels.py::test_classification_counts_2x2x2."""
    fmap, free = fe.free_dof_map(prob)
    d = prob.dofs_per_node
    ed = fmap[fe.element_dofs(prob)]
    khat = fe.reference_stiffness(d, prob.h, prob.poisson_ratio)
    coeff = prob.coeff
    n_nodes = prob.n_nodes
    nn = np.arange(n_nodes)
    i = nn % (prob.nx + 1)
    j = (nn // (prob.nx + 1)) % (prob.ny + 1)
    k = nn // ((prob.nx + 1) * (prob.ny + 1))
    cx, cy, cz = prob.cuts[0]
    vertex = np.isin(i, cx) & np.isin(j, cy) & np.isin(k, cz)
    coord = np.stack([i, j, k], axis=1)
    return Level(n=free.size, elem_dofs=list(ed), elem_mat=lambda e: coeff[e] * khat,
                 elem_sub=prob.elem_to_sub, n_subs=prob.n_subs(1),
                 node_of_dof=free // d, comp_of_dof=free % d,
                 node_eligible=np.ones(n_nodes, dtype=bool), node_vertex=vertex,
                 node_coord=coord, initial=initial)


def level_next(prev: Level, parent: np.ndarray, n_subs: int, cuts, initial="ce") -> Level:
    """Level i+1: elements are level-i substructures with matrices Psi^T S Psi,
    dofs are level-i coarse dofs; level-(i+1) nodes are level-i coarse objects.

    Pinned by test_oracle_solver.py::test_three_levels_single_top_sub_equals_two_levels,
    test_three_levels_spectrum and
    test_oracle_levels.py::test_box_vertex_corners_ragged_and_level_two (level-2 corners).
    """
    node_of_dof = np.empty(prev.n_coarse, dtype=np.int64)
    comp_of_dof = np.empty(prev.n_coarse, dtype=np.int64)
    eligible, vertex, coords = [], [], []
    for o, ob in enumerate(prev.objects):
        for q in range(len(ob.dofs)):
            node_of_dof[ob.first + q] = o
            comp_of_dof[ob.first + q] = ob.comps[q]
        is_corner = ob.kind == "corner"
        eligible.append(is_corner)
        if is_corner and ob.coord is not None:
            c = ob.coord
            vertex.append(bool(np.isin(c[0], cuts[0]) and np.isin(c[1], cuts[1]) and np.isin(c[2], cuts[2])))
            coords.append(c)
        else:
            vertex.append(False)
            coords.append(np.array([-1, -1, -1]))
    elem_dofs = [sb.rc for sb in prev.subs]
    mats = [sb.ac for sb in prev.subs]
    return Level(n=prev.n_coarse, elem_dofs=elem_dofs, elem_mat=lambda e: mats[e],
                 elem_sub=parent, n_subs=n_subs, node_of_dof=node_of_dof,
                 comp_of_dof=comp_of_dof, node_eligible=np.array(eligible),
                 node_vertex=np.array(vertex), node_coord=np.array(coords), initial=initial)
