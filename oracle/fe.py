"""Q1 (tri-linear hexahedral) finite elements on a uniform grid, FP64.

Sec. 2: the domain is discretized by conforming finite elements, one dof per
node (scalar problem) or three displacement dofs per node (linear
elasticity); the global SPD system is Au = f (eq. problem-full-space-algebraic).
Sec. 8.1 uses tri-linear hexahedra.

Element node a = ax + 2*ay + 4*az at local corner (ax, ay, az) in {0,1}^3;
element dof order a * dofs_per_node + component.

Pinned by tests/test_oracle_fe.py: exact symbolic integration (independent
of the quadrature below), rigid-body null spaces, a constant-strain patch
test and the total load.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

_GAUSS = (0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0))  # 2-point rule on [0, 1]


def _shape_gradients(xi, eta, zeta, h):
    """Gradients (8, 3) of the 8 tri-linear shape functions on a cube of side h.

    Pinned by test_oracle_fe.py::test_poisson_element_exact and test_elasticity_element_exact_block
    (exact symbolic integrals of the element matrices built from these gradients).
    """
    g = np.zeros((8, 3))
    for a in range(8):
        ax, ay, az = a & 1, (a >> 1) & 1, (a >> 2) & 1
        fx = xi if ax else 1.0 - xi
        fy = eta if ay else 1.0 - eta
        fz = zeta if az else 1.0 - zeta
        dx = 1.0 if ax else -1.0
        dy = 1.0 if ay else -1.0
        dz = 1.0 if az else -1.0
        g[a] = (dx * fy * fz / h, fx * dy * fz / h, fx * fy * dz / h)
    return g


def lame(young: float, nu: float):
    """Lame parameters of (E, nu).  Pinned by
    test_oracle_fe.py::test_elasticity_element_exact_block."""
    lam = young * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = young / (2.0 * (1.0 + nu))
    return lam, mu


def reference_stiffness(dofs_per_node: int, h: float, nu: float = 0.3) -> np.ndarray:
    """Element matrix for unit coefficient (kappa = 1 or Young's modulus E = 1).

    Pinned by test_oracle_fe.py::test_poisson_element_exact, test_elasticity_element_exact_block
    (exact integrals) and test_rigid_modes_null_space (six rigid modes span the null space).
    """
    nd = 8 * dofs_per_node
    k = np.zeros((nd, nd))
    wq = 0.125 * h ** 3  # weight of each of the 8 Gauss points times the element volume
    if dofs_per_node == 3:
        lam, mu = lame(1.0, nu)
        dmat = lam * np.outer([1, 1, 1, 0, 0, 0], [1, 1, 1, 0, 0, 0]).astype(float)
        dmat += mu * np.diag([2.0, 2.0, 2.0, 1.0, 1.0, 1.0])
    for xi in _GAUSS:
        for eta in _GAUSS:
            for zeta in _GAUSS:
                g = _shape_gradients(xi, eta, zeta, h)
                if dofs_per_node == 1:
                    k += wq * g @ g.T
                else:
                    b = np.zeros((6, 24))
                    for a in range(8):
                        gx, gy, gz = g[a]
                        c = 3 * a
                        b[0, c] = gx
                        b[1, c + 1] = gy
                        b[2, c + 2] = gz
                        b[3, c + 1], b[3, c + 2] = gz, gy
                        b[4, c], b[4, c + 2] = gz, gx
                        b[5, c], b[5, c + 1] = gy, gx
                    k += wq * b.T @ dmat @ b
    return 0.5 * (k + k.T)


def element_nodes(nx: int, ny: int, nz: int) -> np.ndarray:
    """(n_el, 8) global node ids of every element, element order i fastest.

    Pinned by test_oracle_fe.py::test_patch_constant_strain (wrong connectivity breaks the patch
    test).
    """
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    out = np.empty((i.size, 8), dtype=np.int64)
    for a in range(8):
        ax, ay, az = a & 1, (a >> 1) & 1, (a >> 2) & 1
        out[:, a] = (i + ax) + (nx + 1) * ((j + ay) + (ny + 1) * (k + az))
    return out


def element_dofs(prob) -> np.ndarray:
    """(n_el, 8*dpn) global full-grid dof ids (node * dpn + component).

    Pinned by test_oracle_fe.py::test_patch_constant_strain.
    """
    nodes = element_nodes(prob.nx, prob.ny, prob.nz)
    d = prob.dofs_per_node
    return (nodes[:, :, None] * d + np.arange(d)[None, None, :]).reshape(nodes.shape[0], 8 * d)


def free_dof_map(prob):
    """Map full-grid dof -> free dof index (-1 for Dirichlet dofs) and the free dof list.

    Pinned by test_oracle_fe.py::test_total_load and test_patch_constant_strain.
    """
    d = prob.dofs_per_node
    fixed = np.repeat(prob.dirichlet_node_mask.astype(bool), d)
    fmap = -np.ones(fixed.size, dtype=np.int64)
    free = np.nonzero(~fixed)[0]
    fmap[free] = np.arange(free.size)
    return fmap, free


def assemble_global(prob, coeff=None) -> sp.csr_matrix:
    """Global stiffness on free dofs, K = sum_e coeff_e * Khat scattered.

    Pinned by test_oracle_fe.py::test_patch_constant_strain (a linear field gives zero interior
    forces).
    """
    coeff = prob.coeff if coeff is None else coeff
    khat = reference_stiffness(prob.dofs_per_node, prob.h, prob.poisson_ratio)
    fmap, free = free_dof_map(prob)
    ed = fmap[element_dofs(prob)]
    nd = ed.shape[1]
    rows = np.repeat(ed, nd, axis=1).ravel()
    cols = np.tile(ed, (1, nd)).ravel()
    vals = (coeff[:, None] * khat.ravel()[None, :]).ravel()
    keep = (rows >= 0) & (cols >= 0)
    a = sp.coo_matrix((vals[keep], (rows[keep], cols[keep])), shape=(free.size, free.size))
    return a.tocsr()


def load_vector(prob) -> np.ndarray:
    """Consistent nodal loads of a per-element constant body force, on free dofs.
    For tri-linear shape functions on a box, the integral of N_a is V/8.

    Pinned by test_oracle_fe.py::test_total_load (the loads sum to body force times volume).
    """
    fmap, free = free_dof_map(prob)
    ed = element_dofs(prob)
    d = prob.dofs_per_node
    vals = np.repeat(prob.body[:, None, :], 8, axis=1).reshape(ed.shape) * (prob.h ** 3 / 8.0)
    full = np.zeros(prob.n_dofs_full)
    np.add.at(full, ed.ravel(), vals.ravel())
    return full[free]


def to_full(prob, u_free: np.ndarray) -> np.ndarray:
    """Index bookkeeping only (no arithmetic)."""
    fmap, free = free_dof_map(prob)
    out = np.zeros(prob.n_dofs_full)
    out[free] = u_free
    return out
