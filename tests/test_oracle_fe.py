"""Pins of the oracle's Q1 element (Sec. 2, Sec. 8.1: tri-linear hexahedra)
against things the quadrature code does not use: exact symbolic integration,
rigid-body null spaces, a constant-strain patch test and the total load."""
import numpy as np
import pytest
import sympy

import amb_inputs as ai
from oracle import fe


def _sympy_shapes():
    x, y, z = sympy.symbols("x y z")
    n = []
    for a in range(8):
        ax, ay, az = a & 1, (a >> 1) & 1, (a >> 2) & 1
        n.append((x if ax else 1 - x) * (y if ay else 1 - y) * (z if az else 1 - z))
    return (x, y, z), n


def test_poisson_element_exact():
    (x, y, z), n = _sympy_shapes()
    h = 0.25
    k = fe.reference_stiffness(1, h)
    for a in range(8):
        for b in range(8):
            integrand = sum(sympy.diff(n[a], v) * sympy.diff(n[b], v) for v in (x, y, z))
            exact = float(sympy.integrate(integrand, (x, 0, 1), (y, 0, 1), (z, 0, 1))) * h
            assert abs(k[a, b] - exact) < 1e-14
    # closed form of the unit-cube Q1 Laplacian: (4, 0, -1, -1)/12 by node distance
    for a in range(8):
        for b in range(8):
            dist = bin(a ^ b).count("1")
            assert abs(k[a, b] / h - [4, 0, -1, -1][dist] / 12.0) < 1e-14


def test_elasticity_element_exact_block():
    (x, y, z), n = _sympy_shapes()
    nu = 0.3
    lam = nu / ((1 + nu) * (1 - 2 * nu))
    mu = 1 / (2 * (1 + nu))
    h = 0.5
    k = fe.reference_stiffness(3, h, nu)
    v = (x, y, z)
    for a in (0, 3, 6):
        for b in (0, 5, 7):
            for i in range(3):
                for j in range(3):
                    # a(u, w) = int lam div u div w + 2 mu eps(u):eps(w); u = N_a e_i, w = N_b e_j
                    da = [sympy.diff(n[a], q) for q in v]
                    db = [sympy.diff(n[b], q) for q in v]
                    expr = lam * da[i] * db[j] + mu * (da[j] * db[i] + int(i == j) * sum(p * q for p, q in zip(da, db)))
                    exact = float(sympy.integrate(expr, (x, 0, 1), (y, 0, 1), (z, 0, 1))) * h
                    assert abs(k[3 * a + i, 3 * b + j] - exact) < 1e-13


def test_rigid_modes_null_space():
    k1 = fe.reference_stiffness(1, 0.1)
    assert np.abs(k1 @ np.ones(8)).max() < 1e-14
    assert np.linalg.matrix_rank(k1, tol=1e-12) == 7
    k3 = fe.reference_stiffness(3, 0.1, 0.3)
    pts = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], float)
    modes = []
    for c in range(3):
        m = np.zeros((8, 3)); m[:, c] = 1; modes.append(m.ravel())
    for axis in range(3):
        m = np.cross(np.eye(3)[axis], pts); modes.append(m.ravel())
    for m in modes:
        assert np.abs(k3 @ m).max() < 1e-13
    assert np.linalg.matrix_rank(k3, tol=1e-10) == 18


def test_patch_constant_strain():
    """A linear displacement field gives zero nodal forces at interior nodes."""
    prob = ai.toy(3, 3, 1, split=(1, 1, 1))
    prob.dirichlet_node_mask[:] = 0
    prob.coeff[:] = 1.0
    a = fe.assemble_global(prob)
    nn = np.arange(prob.n_nodes)
    i = nn % (prob.nx + 1); j = (nn // (prob.nx + 1)) % (prob.ny + 1); k = nn // ((prob.nx + 1) * (prob.ny + 1))
    grad = np.array([[0.3, -0.2, 0.1], [0.05, 0.4, -0.3], [0.2, 0.1, -0.1]])
    xyz = np.stack([i, j, k], 1) * prob.h
    u = (xyz @ grad.T).ravel()
    f = a @ u
    inner = (i > 0) & (i < prob.nx) & (j > 0) & (j < prob.ny) & (k > 0) & (k < prob.nz)
    assert np.abs(f.reshape(-1, 3)[inner]).max() < 1e-12


def test_total_load():
    prob = ai.toy(4, 1, 3)
    prob.dirichlet_node_mask[:] = 0
    f = fe.load_vector(prob)
    vol = prob.nx * prob.ny * prob.nz * prob.h ** 3
    assert abs(f.sum() - vol) < 1e-14
    prob3 = ai.toy(4, 3, 3)
    prob3.dirichlet_node_mask[:] = 0
    f3 = fe.load_vector(prob3).reshape(-1, 3)
    assert abs(f3[:, 2].sum() + vol) < 1e-14 and np.abs(f3[:, :2]).max() == 0
