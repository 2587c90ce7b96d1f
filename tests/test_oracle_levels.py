"""Pins of one oracle level: Schur-complement null spaces, the coarse basis
(eq. local_saddle_point_problem: C Psi = I, Psi^T S Psi = -mu, Sec. 5), the
averaging operator E (eq. E-onto-U: E U = U, E^2 = E) and the box-vertex
corner counts of the paper's 2x2x2 decomposition (12 faces, Table 1)."""
import numpy as np
import pytest

import amb_inputs as ai
from oracle import levels as lv


def _level(prob, initial="ce"):
    lev = lv.level_one(prob, initial)
    lev.schur()
    lev.coarse_basis()
    return lev


def _rigid_modes(lev, sb, prob):
    nodes = lev.node_of_dof[sb.gdofs]
    comp = lev.comp_of_dof[sb.gdofs]
    nx1, ny1 = prob.nx + 1, prob.ny + 1
    xyz = np.stack([nodes % nx1, (nodes // nx1) % ny1, nodes // (nx1 * ny1)], 1).astype(float)
    modes = []
    for c in range(3):
        modes.append((comp == c).astype(float))
    for ax in range(3):
        r = np.cross(np.eye(3)[ax], xyz)
        modes.append(r[np.arange(comp.size), comp])
    return np.array(modes).T


def test_floating_schur_null_space():
    prob = ai.toy(4, 1, 11)
    lev = _level(prob)
    s1 = lev.subs[1].s        # sub 1 does not touch x = 0: floating
    assert np.abs(s1 @ np.ones(s1.shape[0])).max() < 1e-10 * np.abs(s1).max()
    prob3 = ai.toy(4, 3, 11)
    lev3 = _level(prob3)
    sb = lev3.subs[1]
    r = _rigid_modes(lev3, sb, prob3)
    assert np.abs(sb.s @ r).max() < 1e-9 * np.abs(sb.s).max()
    # sub 0 is held by the Dirichlet face: its S is positive definite
    assert np.linalg.eigvalsh(lev3.subs[0].s).min() > 0


@pytest.mark.parametrize("dpn", [1, 3])
def test_coarse_basis_identities(dpn):
    prob = ai.toy(4, dpn, 5, split=(2, 2, 1))
    lev = _level(prob)
    for sb in lev.subs:
        nc = sb.c.shape[0]
        assert np.allclose(sb.c @ sb.psi, np.eye(nc), atol=1e-10)
        assert np.allclose(sb.psi.T @ sb.s @ sb.psi, -sb.mu, atol=1e-9 * np.abs(sb.mu).max())
    ac = lev.coarse_matrix()
    assert np.linalg.eigvalsh(ac).min() > 0


def test_averaging_is_projection_onto_U():
    prob = ai.toy(4, 3, 2, split=(2, 2, 1))
    lev = _level(prob)
    rng = np.random.default_rng(0)
    u = rng.standard_normal(lev.n)
    ru = [u[sb.dofs] for sb in lev.subs]
    assert np.allclose(lev.average(ru), u, atol=1e-13)          # E U = U (partition of unity)
    z = [rng.standard_normal(sb.dofs.size) for sb in lev.subs]
    ez = lev.average(z)
    assert np.allclose(lev.average([ez[sb.dofs] for sb in lev.subs]), ez, atol=1e-13)  # E^2 = E
    # weights sum to one on every interface dof
    acc = np.zeros(lev.n)
    for sb in lev.subs:
        np.add.at(acc, sb.gdofs, sb.w)
    iface = np.unique(np.concatenate([sb.gdofs for sb in lev.subs]))
    assert np.allclose(acc[iface], 1.0, atol=1e-14)


def test_classification_counts_2x2x2():
    prob = ai.config(1)
    lev = lv.level_one(prob)
    # 3x3x3 box vertices, minus the 9 Dirichlet ones on x = 0, minus the 4 owned by one substructure
    assert int(lev.node_corner.sum()) == 14
    assert len(lev.edges) == 6
    assert len(lev.faces) == 12
    # every edge is shared by 4 substructures, every face by 2
    assert all(len(k) == 4 for k in lev.edges)


def test_box_vertex_corners_ragged_and_level_two():
    """Corner counts by the box-vertex rule, counted by hand from the cut
    planes.  Ragged 3 x 2 x 1 boxes (x cuts 0, 2, 5, 9; y cuts 0, 4, 9; one z
    box) with the Dirichlet face x = 0: vertices on x = 2 and x = 5 (y = 0,
    4, 9; z = 0, 9) are interface nodes, on x = 9 only y = 4 is (shared by
    two boxes) -> 6 + 6 + 2 = 14.  The face between the boxes (0,0) and
    (0,1) is one node wide (x = 1); its nodes on z = 0 and z = 9 are no
    vertices.  Level 2 of the 4 x 2 x 1 toy grouped 2 x 1 x 1: the level-2
    vertices on the shared plane x = 6 are (y, z) in {0, 6} x {0, 3} -> 4
    corners; the level-1 corners at y = 3 are not."""
    rng = np.random.default_rng(np.random.PCG64(21))
    coeff = np.exp(rng.standard_normal(9 ** 3))
    prob = ai._make("ragged", 9, None, 1, coeff, 2, 3.0,
                    cuts1=[np.array([0, 2, 5, 9]), np.array([0, 4, 9]), np.array([0, 9])])
    lev = lv.level_one(prob)
    assert int(lev.node_corner.sum()) == 14
    n1 = prob.nx + 1
    for z in (0, 9):
        node = 1 + n1 * (4 + n1 * z)
        assert lev.node_interface[node] and not lev.node_corner[node]
    groups = [np.array([0, 2, 4]), np.array([0, 2]), np.array([0, 1])]
    toy = ai.toy(3, 3, 41, split=(4, 2, 1), levels=3, groups=groups, sigma=1.0, tau=2.0)
    from oracle import solver
    h = solver.Hierarchy(toy)
    # level 1 (cuts x 0,3,6,9,12; y 0,3,6; z 0,3): x = 3, 6, 9 give 3 x 3 x 2 = 18, x = 12 only y = 3 -> 20
    assert int(h.levels[0].node_corner.sum()) == 20
    assert int(h.levels[1].node_corner.sum()) == 4


@pytest.mark.parametrize("dpn,split,initial", [(1, (2, 2, 1), "ce"), (3, (2, 2, 1), "ce"), (3, (2, 2, 2), "c")])
def test_assumption_1_constrained_problems_are_definite(dpn, split, initial):
    """Assumption 1: with the initial constraints every substructure's
    energy is positive on the constrained space null(C), floating or not,
    although S itself is singular for floating substructures (constants,
    rigid modes).  Without constraints a floating substructure breaks it."""
    import scipy.linalg as sla
    prob = ai.toy(3, dpn, 17, split=split)
    lev = lv.level_one(prob, initial)
    lev.schur()
    floating = 0
    for sb in lev.subs:
        z = sla.null_space(sb.c)
        lam = np.linalg.eigvalsh(z.T @ sb.s @ z)
        assert lam.min() > 1e-8 * lam.max()
        lam_s = np.linalg.eigvalsh(sb.s)
        if lam_s.min() < 1e-10 * lam_s.max():
            floating += 1
    assert floating > 0          # the case the assumption is about is present
