"""The library's host combinatorics (amb_plan: Sec. 2 classification with
the box-vertex corner rule, the initial constraints of Sec. 7.1, the
level-(i+1) nodes from the level-i coarse objects of Sec. 3) against the
oracle's levels, on the CPU: counts of substructures, faces, edges, corner
nodes, level and coarse dofs, and per substructure n_I, n_Gamma, corner
dofs and coarse dofs.  Irregular and ragged box partitions, substructures
without interior dofs, scalar and elasticity problems, both initial
constraint sets, and levels 2 and 3 of non-adaptive hierarchies."""
import numpy as np
import pytest

import amb_inputs as ai
from oracle import levels as olv, pair as opr, solver


def _cases():
    rng = np.random.default_rng(np.random.PCG64(7))
    yield "toy221", ai.toy(3, 1, 1, split=(2, 2, 1))
    yield "toy222_elast", ai.toy(2, 3, 2, split=(2, 2, 2))
    yield "ragged", ai._make("ragged", 9, None, 1, np.ones(729), 2, 10.0,
                             cuts1=[np.array([0, 2, 5, 9]), np.array([0, 4, 9]), np.array([0, 9])])
    yield "thin", ai._make("thin", 6, None, 1, np.ones(216), 2, 10.0,
                           cuts1=[np.array([0, 1, 4, 5, 6]), np.array([0, 3, 6]), np.array([0, 6])])
    cuts = [ai.irregular_cuts(14, 4, 2, 5, rng) for _ in range(3)]
    yield "irregular", ai._make("irr", 14, None, 1, np.ones(14 ** 3), 2, 10.0, cuts1=cuts)
    cuts = [ai.irregular_cuts(10, 3, 2, 5, rng) for _ in range(3)]
    yield "irregular_elast", ai._make("irr3", 10, None, 3, np.ones(1000), 2, 10.0, cuts1=cuts)


def _initial(B, initial):
    return {"c": B.CORNERS, "ce": B.CORNERS_EDGES, "cef": B.CORNERS_EDGES_FACES}[initial]


@pytest.mark.parametrize("initial", ["ce", "c", "cef"])
@pytest.mark.parametrize("name,prob", list(_cases()))
def test_level_one_plan_matches_oracle(name, prob, initial):
    from paper_1301_0191_gb300 import binding as B
    info, subs = B.plan(prob.nx, prob.ny, prob.nz, prob.dofs_per_node, prob.dirichlet_node_mask,
                        prob.elem_to_sub, prob.n_subs(1), initial=_initial(B, initial))
    lev = olv.level_one(prob, initial=initial)
    _compare(info, subs, lev, name)


def _compare(info, subs, lev, name):
    assert info.n_subs == lev.n_subs
    assert info.n_dofs == lev.n
    assert info.n_corner_nodes == int(lev.node_corner.sum())
    assert info.n_edges == len(lev.edges)
    assert info.n_pairs == len(opr.pairs_of(lev))
    assert info.n_coarse == lev.n_coarse
    for s, sb in enumerate(lev.subs):
        n_crn = int(np.sum(lev.node_corner[lev.node_of_dof[sb.gdofs]]))
        assert tuple(subs[s]) == (sb.n_i, sb.n_g, n_crn, sb.c.shape[0]), (name, s)
    assert info.sum_ni == sum(sb.n_i for sb in lev.subs)
    assert info.schur_words == float(sum(sb.n_g ** 2 for sb in lev.subs))


def test_plan_rejects_a_non_box_partition():
    from paper_1301_0191_gb300 import binding as B
    prob = ai.toy(2, 1, 3, split=(2, 1, 1))
    e2s = prob.elem_to_sub.copy()
    e2s[0] = 1 - e2s[0]
    with pytest.raises(B.AmbError) as ei:
        B.plan(prob.nx, prob.ny, prob.nz, 1, prob.dirichlet_node_mask, e2s, 2)
    assert ei.value.status == B.EINVAL


def _multilevel_cases():
    g3 = [np.array([0, 2, 4]), np.array([0, 2]), np.array([0, 1])]
    yield "scalar_4x2x1_to_2", ai.toy(3, 1, 41, split=(4, 2, 1), levels=3, groups=g3)
    g = [np.array([0, 2, 4])] * 3
    yield "elast_4x4x4_to_2x2x2", ai.toy(2, 3, 42, split=(4, 4, 4), levels=3, groups=g)
    yield "scalar_4x4x4_to_2x2x2", ai.toy(2, 1, 43, split=(4, 4, 4), levels=3, groups=g)
    rng = np.random.default_rng(np.random.PCG64(44))
    cuts = [ai.irregular_cuts(16, 4, 3, 5, rng) for _ in range(3)]
    yield "irregular_to_2x2x2", ai._make("irr", 16, None, 1, np.ones(16 ** 3), 3, 10.0, groups=g, cuts1=cuts)


@pytest.mark.parametrize("initial", ["ce", "cef"])
@pytest.mark.parametrize("name,prob", list(_multilevel_cases()))
def test_level_two_plan_matches_oracle(name, prob, initial):
    """Level 2 of a non-adaptive three-level hierarchy: the nodes are the
    level-1 corners, edges (and faces, with face averages), only level-1
    corners may become corners."""
    from paper_1301_0191_gb300 import binding as B
    h = solver.Hierarchy(prob, adaptive=False, initial=initial)
    info, subs = B.plan(prob.nx, prob.ny, prob.nz, prob.dofs_per_node, prob.dirichlet_node_mask,
                        prob.elem_to_sub, prob.n_subs(1), levels=3, sub_to_parent=prob.sub_to_parent,
                        n_sub=[prob.n_subs(2)], level=2, initial=_initial(B, initial))
    _compare(info, subs, h.levels[1], name)
    # level 1 of the same hierarchy
    info1, subs1 = B.plan(prob.nx, prob.ny, prob.nz, prob.dofs_per_node, prob.dirichlet_node_mask,
                          prob.elem_to_sub, prob.n_subs(1), levels=3, sub_to_parent=prob.sub_to_parent,
                          n_sub=[prob.n_subs(2)], level=1, initial=_initial(B, initial))
    _compare(info1, subs1, h.levels[0], name)


def test_plan_rejects_bad_levels():
    from paper_1301_0191_gb300 import binding as B
    prob = list(_multilevel_cases())[0][1]
    args = (prob.nx, prob.ny, prob.nz, prob.dofs_per_node, prob.dirichlet_node_mask, prob.elem_to_sub,
            prob.n_subs(1))
    for level in (0, 3):
        with pytest.raises(B.AmbError) as ei:
            B.plan(*args, levels=3, sub_to_parent=prob.sub_to_parent, n_sub=[prob.n_subs(2)], level=level)
        assert ei.value.status == B.EINVAL
    with pytest.raises(B.AmbError) as ei:                  # three levels need the parent map
        B.plan(*args, levels=3, level=1)
    assert ei.value.status == B.EINVAL


@pytest.mark.parametrize("name,prob", list(_multilevel_cases())[:2])
def test_level_two_plan_corners_only(name, prob):
    """Level 2 with corners as the only initial constraints: its nodes are
    the level-1 corners alone."""
    from paper_1301_0191_gb300 import binding as B
    h = solver.Hierarchy(prob, adaptive=False, initial="c")
    info, subs = B.plan(prob.nx, prob.ny, prob.nz, prob.dofs_per_node, prob.dirichlet_node_mask,
                        prob.elem_to_sub, prob.n_subs(1), levels=3, sub_to_parent=prob.sub_to_parent,
                        n_sub=[prob.n_subs(2)], level=2, initial=B.CORNERS)
    _compare(info, subs, h.levels[1], name)


def test_bench_workload_sizes():
    """The 48^3 elasticity workload (4 x 4 x 4 boxes of 12^3 elements, the
    x = 0 node plane clamped), by counting nodes: a box's nodes on outer,
    unclamped faces are its own, so a box at the far corner has 12^3
    interior nodes and a box with no free outer face 11^3.  The
    factorization work equals the bench line's algorithmic flop count, which
    came from the same sizes through amb_level_info on the GPU."""
    from paper_1301_0191_gb300 import binding as B
    p = ai.config(2)
    info, subs = B.plan(p.nx, p.ny, p.nz, p.dofs_per_node, p.dirichlet_node_mask, p.elem_to_sub, p.n_subs(1))
    assert (info.n_subs, info.n_pairs) == (64, 144)
    assert info.n_dofs == 3 * 48 * 49 * 49                     # the x = 0 node plane is clamped
    assert info.max_ni == 3 * 12 ** 3 and int(subs[:, 0].min()) == 3 * 11 ** 3
    assert (info.max_ngamma, info.max_ndelta) == (2598, 2574)
    assert info.factor_flops == 5776528886316.0
