"""Crops of a box-partitioned mesh for oracle checks of single faces.

The pair eigenproblem of a face (Sec. 4, eq. eig-matrix) depends only on
S^s, S^t, the stiffness diagonals of s and t on their shared dofs (the pair
weights of Sec. 7.2) and the corners and edge averages of s and t, that is
on the elements of s and t and on which substructures share each of their
nodes.  In a box partition every substructure that shares a node with s or
t lies in the block of partition cells one layer around s and t.  The oracle
run on that crop (same element matrices, Dirichlet nodes and cut planes)
therefore gives the full problem's S^s, S^t and pair eigenvalues, at the
cost of a few dozen substructures instead of all of them.
tests/test_oracle_crop.py checks this against the oracle on a whole mesh.

Index bookkeeping only: no step of the method is computed here.
"""
import dataclasses

import numpy as np

import amb_inputs as ai
from oracle import fe


@dataclasses.dataclass
class Crop(ai.Problem):
    """A crop of a problem's mesh whose elements keep the full mesh's size."""
    h_full: float = 1.0

    @property
    def h(self) -> float:
        return self.h_full


def box_of(prob, s):
    na, nb = (len(c) - 1 for c in prob.cuts[0][:2])
    return s % na, (s // na) % nb, s // (na * nb)


def crop_around(prob, s, t):
    """The partition cells one layer around s and t, as a problem of its own;
    returns it, the map of its level-1 substructures to the full ones, and the
    full-mesh dof id (node * dofs_per_node + component) of each of its free
    dofs."""
    cuts = prob.cuts[0]
    nbox = [len(c) - 1 for c in cuts]
    bs, bt = box_of(prob, s), box_of(prob, t)
    lo = [max(min(bs[a], bt[a]) - 1, 0) for a in range(3)]
    hi = [min(max(bs[a], bt[a]) + 1, nbox[a] - 1) for a in range(3)]
    e0 = [int(cuts[a][lo[a]]) for a in range(3)]
    e1 = [int(cuts[a][hi[a] + 1]) for a in range(3)]
    nx, ny, nz = (e1[a] - e0[a] for a in range(3))
    coeff = prob.coeff.reshape(prob.nz, prob.ny, prob.nx)[e0[2]:e1[2], e0[1]:e1[1], e0[0]:e1[0]].ravel()
    m3 = prob.dirichlet_node_mask.reshape(prob.nz + 1, prob.ny + 1, prob.nx + 1)
    mask = m3[e0[2]:e1[2] + 1, e0[1]:e1[1] + 1, e0[0]:e1[0] + 1].ravel().copy()
    ccuts = [np.asarray(cuts[a][lo[a]:hi[a] + 2]) - e0[a] for a in range(3)]
    crop = Crop(name="crop", nx=nx, ny=ny, nz=nz, dofs_per_node=prob.dofs_per_node, coeff=coeff,
                 poisson_ratio=prob.poisson_ratio, body=np.zeros((nx * ny * nz, prob.dofs_per_node)),
                 dirichlet_node_mask=mask, cuts=[ccuts], elem_to_sub=ai.tensor_partition(nx, ny, nz, ccuts),
                 sub_to_parent=[], levels=2, tau=prob.tau, h_full=prob.h)
    na, nb = hi[0] - lo[0] + 1, hi[1] - lo[1] + 1
    sub_map = {}
    for c in range(hi[2] - lo[2] + 1):
        for b in range(nb):
            for a in range(na):
                sub_map[a + na * (b + nb * c)] = \
                    (a + lo[0]) + nbox[0] * ((b + lo[1]) + nbox[1] * (c + lo[2]))
    d = prob.dofs_per_node
    free_crop = fe.free_dof_map(crop)[1]
    node, comp = free_crop // d, free_crop % d
    i = node % (nx + 1)
    j = (node // (nx + 1)) % (ny + 1)
    k = node // ((nx + 1) * (ny + 1))
    gnode = (i + e0[0]) + (prob.nx + 1) * ((j + e0[1]) + (prob.ny + 1) * (k + e0[2]))
    dof_map = gnode * d + comp
    assert not np.any(np.repeat(prob.dirichlet_node_mask.astype(bool), d)[dof_map])
    return crop, sub_map, dof_map
