"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

Tolerances (FP64 path): Schur complements and coarse matrices 1e-9
relative to their largest entry, entry by entry (coarse matrices after
matching the constraint rows one to one); solution 1e-6 relative to a sparse direct solve at
the 1e-8 PCG tolerance; pair eigenvalues above tau/10 within 1e-4
relative (LOBPCG residual 1e-8); PCG iterations and selected constraint
counts within +-1 (several results are correct at ties, Sec. 4).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import amb_inputs as ai
from oracle import fe, gradient as og, levels as olv, pair as opr, solver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1301_0191_gb300 import binding
    return binding


def _free(prob):
    return fe.free_dof_map(prob)[1]


def _ctx(B, prob, **kw):
    return B.Context.from_problem(prob, **kw)


@pytest.mark.parametrize("dpn,split,seed", [(1, (2, 2, 1), 3), (3, (2, 2, 1), 4), (3, (2, 2, 2), 5), (1, (3, 2, 2), 6)])
def test_schur_and_coarse_matrices(B, dpn, split, seed):
    prob = ai.toy(4 if dpn == 1 else 3, dpn, seed, split=split, sigma=1.5)
    ctx = _ctx(B, prob, adaptive=0)
    lev = olv.level_one(prob)
    lev.schur()
    lev.coarse_basis()
    free = _free(prob)
    info = ctx.level_info(1)
    assert info.n_subs == lev.n_subs and info.n_coarse == lev.n_coarse
    assert info.n_corner_nodes == int(lev.node_corner.sum())
    corners = ctx.export(B.X_CORNERS, 1, 0, np.int64)
    ocorner = np.sort(free[np.concatenate([lev.dofs_of_node[i] for i in np.nonzero(lev.node_corner)[0]])])
    assert np.array_equal(np.sort(corners), ocorner)
    for s, sb in enumerate(lev.subs):
        dofs = ctx.export(B.X_SUB_DOFS, 1, s, np.int64)
        ni, ng, ncrn, nc = ctx.export(B.X_SUB_SIZES, 1, s, np.int32)
        assert ni == sb.n_i and ng == sb.n_g and nc == sb.c.shape[0]
        assert np.array_equal(np.sort(dofs[:ni]), np.sort(free[sb.idofs]))
        # map the oracle interface order onto the library's
        g_lib = dofs[ni:]
        pos = {int(d): i for i, d in enumerate(free[sb.gdofs])}
        perm = np.array([pos[int(d)] for d in g_lib])
        S = ctx.export(B.X_SCHUR, 1, s, np.float64).reshape(ng, ng, order="F")
        So = sb.s[np.ix_(perm, perm)]
        assert np.abs(S - So).max() <= 1e-9 * np.abs(So).max()
        Ac = ctx.export(B.X_COARSE_EL, 1, s, np.float64).reshape(nc, nc, order="F")
        ev, evo = np.linalg.eigvalsh(Ac), np.linalg.eigvalsh(sb.ac)
        assert np.allclose(ev, evo, rtol=1e-8, atol=1e-9 * np.abs(evo).max())
        Cl = ctx.export(B.X_CONSTR, 1, s, np.float64).reshape(nc, ng)
        # same row space (constraint functionals), in the library's interface order
        Co = sb.c[:, perm]
        assert np.linalg.matrix_rank(np.vstack([Cl, Co]), tol=1e-10) == nc
        # the initial constraints are unique functionals (corner dofs, edge
        # averages): match the rows one to one, then A_c entry by entry
        cperm = []
        for row in Cl:
            hit = np.nonzero(np.abs(Co - row).max(axis=1) <= 1e-12)[0]
            assert hit.size == 1
            cperm.append(int(hit[0]))
        Aco = sb.ac[np.ix_(cperm, cperm)]
        assert np.abs(Ac - Aco).max() <= 1e-9 * np.abs(Aco).max()
    ctx.close()


def _oracle_pairs(prob, tau):
    lev = olv.level_one(prob)
    lev.schur()
    out = {}
    for (s, t) in opr.pairs_of(lev):
        lam, _, _, _ = opr.reduced(lev, s, t)
        out[(s, t)] = np.sort(lam[lam > 0])[::-1]
    return out


@pytest.mark.parametrize("dpn,split,seed,tau", [(1, (2, 1, 1), 7, 2.0), (3, (2, 1, 1), 8, 3.0),
                                                 (1, (2, 2, 2), 9, 3.0), (3, (2, 2, 1), 10, 3.0)])
def test_pair_eigenvalues_and_selection(B, dpn, split, seed, tau):
    prob = ai.toy(5 if dpn == 1 else 4, dpn, seed, split=split, sigma=2.0, tau=tau)
    ctx = _ctx(B, prob, lobpcg_tol=1e-6, lobpcg_maxit=300)
    rep = ctx.report()
    ref = _oracle_pairs(prob, tau)
    assert len(rep["pairs"]) == len(ref)
    for pr in rep["pairs"]:
        lo = ref[(pr["s"], pr["t"])]
        lam = pr["lam"]
        # the columns the method uses: the selected ones and lambda_{k+1}
        k = min(len(lam), len(lo), pr["n_selected"] + 1)
        for i in range(k):
            if lo[i] >= 0.1 * tau:
                assert abs(lam[i] - lo[i]) <= 1e-4 * lo[i], (pr["s"], pr["t"], i, lam[i], lo[i])
        nsel_o = int(min(10, np.sum(lo > tau)))
        assert abs(pr["n_selected"] - nsel_o) <= 1
        assert pr["converged"] == 1
    ctx.close()


@pytest.mark.parametrize("dpn,split,seed,adaptive", [(1, (2, 2, 1), 11, 1), (3, (2, 2, 1), 12, 1),
                                                      (3, (2, 2, 2), 13, 0), (1, (3, 3, 2), 14, 1)])
def test_solution_and_iterations(B, dpn, split, seed, adaptive):
    prob = ai.toy(4 if dpn == 1 else 3, dpn, seed, split=split, sigma=2.0, tau=3.0)
    ctx = _ctx(B, prob, adaptive=adaptive, lobpcg_tol=1e-8, lobpcg_maxit=300)
    f = ctx.load_vector(prob.body)
    u, info = ctx.solve(f)
    h, res, f_free = solver.solve(prob, adaptive=bool(adaptive))
    free = _free(prob)
    assert np.allclose(f[free], f_free, rtol=1e-12, atol=1e-16)
    ud = spla.spsolve(h.ops[0].tocsc(), f_free)
    assert info.rel_residual <= 1e-8 and info.true_rel_residual <= 1e-7
    assert np.linalg.norm(u[free] - ud) <= 1e-6 * np.linalg.norm(ud)
    assert abs(info.iterations - res.its) <= 1, (info.iterations, res.its)
    assert abs(info.cond_estimate - res.cond) <= 1e-3 * res.cond + 0.05
    if adaptive:
        rep = ctx.report()
        assert abs(rep["n_adaptive"][0] - h.reports[0].n_adaptive) <= max(1, len(rep["pairs"]) // 10)
    ctx.close()


def test_config1_end_to_end(B):
    prob = ai.config(1)
    ctx = _ctx(B, prob, lobpcg_tol=1e-8, lobpcg_maxit=300)
    f = ctx.load_vector(prob.body)
    u, info = ctx.solve(f)
    h, res, f_free = solver.solve(prob)
    free = _free(prob)
    ud = spla.spsolve(h.ops[0].tocsc(), f_free)
    assert np.linalg.norm(u[free] - ud) <= 1e-6 * np.linalg.norm(ud)
    assert abs(info.iterations - res.its) <= 1
    rep = ctx.report()
    assert abs(rep["n_adaptive"][0] - h.reports[0].n_adaptive) <= 2
    ctx.close()


@pytest.mark.parametrize("dpn", [1, 3])
def test_three_levels(B, dpn):
    """Three levels (4x2x1 substructures in 2x1x1 level-2 groups): the level-2
    corners are the level-1 corners on level-2 box vertices; coarse objects,
    pair eigenvalues and selections on both levels match the oracle."""
    groups = [np.array([0, 2, 4]), np.array([0, 2]), np.array([0, 1])]
    prob = ai.toy(3, dpn, 41, split=(4, 2, 1), levels=3, groups=groups, sigma=1.0, tau=2.0)
    ctx = _ctx(B, prob, lobpcg_tol=1e-8, lobpcg_maxit=300)
    f = ctx.load_vector(prob.body)
    u, info = ctx.solve(f)
    rep = ctx.report()
    h, res, f_free = solver.solve(prob)
    free = _free(prob)
    ud = spla.spsolve(h.ops[0].tocsc(), f_free)
    assert np.linalg.norm(u[free] - ud) <= 1e-6 * np.linalg.norm(ud)
    assert abs(info.iterations - res.its) <= 1, (info.iterations, res.its)
    same_selection = True
    for lev in (1, 2):
        li, ol, orep = ctx.level_info(lev), h.levels[lev - 1], h.reports[lev - 1]
        assert li.n_dofs == ol.n
        assert li.n_corner_nodes == int(ol.node_corner.sum())
        assert li.n_edges == len(ol.edges) and li.n_faces == len(ol.faces)
        gp = {(p["s"], p["t"]): p for p in rep["pairs"] if p["level"] == lev}
        assert sorted(gp) == sorted((int(s), int(t)) for s, t in orep.pairs)
        for (s, t), lo, k_o in zip(orep.pairs, orep.lam, orep.n_selected):
            pr = gp[(int(s), int(t))]
            assert abs(pr["n_selected"] - k_o) <= 1
            if same_selection:
                lo = np.sort(np.asarray(lo))[::-1]
                for i in range(min(len(lo), len(pr["lam"]), pr["n_selected"] + 1)):
                    if lo[i] >= 0.1 * prob.tau:
                        assert abs(pr["lam"][i] - lo[i]) <= 1e-4 * lo[i], (lev, s, t, i, pr["lam"][i], lo[i])
        # level-2 elements carry the level-1 adaptive rows: compare their
        # eigenvalues only when the level-1 selections agree
        same_selection = same_selection and all(
            gp[(int(s), int(t))]["n_selected"] == k_o for (s, t), k_o in zip(orep.pairs, orep.n_selected))
    li2 = ctx.level_info(2)
    assert li2.n_subs == 2
    ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_runs_are_bitwise_reproducible(B, precision):
    """Assembly, factorizations, LOBPCG and PCG use no atomics or
    order-dependent reductions: two set-ups + solves of the same problem give
    identical bits (two-level and three-level hierarchies)."""
    prec = B.FP64 if precision == "fp64" else B.FP32
    groups = [np.array([0, 2, 4]), np.array([0, 2]), np.array([0, 1])]
    for prob in (ai.toy(4, 3, 17, split=(2, 2, 2), sigma=1.5, tau=3.0),
                 ai.toy(3, 1, 41, split=(4, 2, 1), levels=3, groups=groups, sigma=1.0, tau=2.0)):
        out = []
        for _ in range(2):
            c = _ctx(B, prob, precision=prec)
            f = c.load_vector(prob.body)
            u, info = c.solve(f)
            rep = c.report()
            out.append((u, info.iterations, [p["lam"] for p in rep["pairs"]], rep["n_adaptive"]))
            c.close()
        (u0, i0, l0, n0), (u1, i1, l1, n1) = out
        assert i0 == i1 and n0 == n1
        assert np.array_equal(u0, u1)
        assert all(np.array_equal(np.asarray(a), np.asarray(b)) for a, b in zip(l0, l1))


def test_fp32_preconditioner_reaches_fp64_tolerance(B):
    prob = ai.toy(4, 3, 15, split=(2, 2, 2), sigma=1.5, tau=3.0)
    c64 = _ctx(B, prob, lobpcg_tol=1e-8)
    c32 = _ctx(B, prob, precision=B.FP32, lobpcg_tol=1e-5)
    f = c64.load_vector(prob.body)
    u64, i64 = c64.solve(f)
    u32, i32 = c32.solve(f)
    assert i32.rel_residual <= 1e-8 and i32.true_rel_residual <= 1e-7
    assert np.linalg.norm(u32 - u64) <= 1e-6 * np.linalg.norm(u64)
    assert i32.iterations <= i64.iterations + 3
    c64.close()
    c32.close()


def test_fp32_form_three_levels(B):
    """FP32 form on three levels (elasticity, 4x2x1 substructures in two
    level-2 groups): PCG reaches the FP64 tolerance, the solution matches the
    sparse direct solve to 1e-6, and the selections per face match the FP64
    form within +-1 on both levels."""
    groups = [np.array([0, 2, 4]), np.array([0, 2]), np.array([0, 1])]
    prob = ai.toy(3, 3, 41, split=(4, 2, 1), levels=3, groups=groups, sigma=1.0, tau=2.0)
    c64 = _ctx(B, prob, lobpcg_tol=1e-8, lobpcg_maxit=300)
    c32 = _ctx(B, prob, precision=B.FP32, lobpcg_tol=1e-6, lobpcg_maxit=300)
    f = c64.load_vector(prob.body)
    u64, i64 = c64.solve(f)
    u32, i32 = c32.solve(f)
    r64, r32 = c64.report(), c32.report()
    c64.close()
    c32.close()
    assert i32.rel_residual <= 1e-8 and i32.true_rel_residual <= 1e-7
    free = _free(prob)
    h, res, f_free = solver.solve(prob)
    ud = spla.spsolve(h.ops[0].tocsc(), f_free)
    assert np.linalg.norm(u32[free] - ud) <= 1e-6 * np.linalg.norm(ud)
    assert i32.iterations <= i64.iterations + 3
    sel64 = {(p["level"], p["s"], p["t"]): p["n_selected"] for p in r64["pairs"]}
    sel32 = {(p["level"], p["s"], p["t"]): p["n_selected"] for p in r32["pairs"]}
    assert sel64.keys() == sel32.keys()
    assert all(abs(sel64[k] - sel32[k]) <= 1 for k in sel64)


def test_compliance_gradient(B):
    prob = ai.toy(3, 1, 16, split=(2, 2, 1), sigma=1.0)
    ctx = _ctx(B, prob)
    f = ctx.load_vector(prob.body)
    ctx.solve(f)
    g = ctx.grad(B.QOI_COMPLIANCE)
    _, g_ref = og.compliance_and_gradient(prob)
    assert np.abs(g - g_ref).max() <= 1e-7 * np.abs(g_ref).max()
    # general QoI with dq/du = f equals the compliance adjoint
    g2 = ctx.grad(B.QOI_GENERAL, dq_du=f)
    assert np.abs(g2 - g_ref).max() <= 1e-6 * np.abs(g_ref).max()
    ctx.close()


def test_schur_apply(B):
    import torch
    prob = ai.toy(4, 3, 17, split=(2, 2, 1))
    ctx = _ctx(B, prob, adaptive=0)
    n = ctx.level_info(1).n_subs
    sizes = [int(ctx.export(B.X_SUB_SIZES, 1, s, np.int32)[1]) for s in range(n)]
    for width in (1, 7):
        x = torch.randn(sum(sizes) * width, dtype=torch.float64, device="cuda")
        y = torch.empty_like(x)
        ctx.schur_apply(1, width, x, y)
        xh, yh = x.cpu().numpy(), y.cpu().numpy()
        o = 0
        for s, ng in enumerate(sizes):
            S = ctx.export(B.X_SCHUR, 1, s, np.float64).reshape(ng, ng, order="F")
            X = xh[o:o + ng * width].reshape(ng, width, order="F")
            Y = yh[o:o + ng * width].reshape(ng, width, order="F")
            assert np.abs(Y - S @ X).max() <= 1e-12 * np.abs(S).max() * ng
            o += ng * width
    ctx.close()


def test_schur_apply_fp32_tensor_cores(B):
    """FP32 form, widths 64 and 100 (tensor cores, 3xTF32, K in chunks of 256):
    Y = S X against the FP64 product of the exported FP32 S with the same X,
    within the 3xTF32 accumulation error (64 units of 2^-24 relative to sum |S||X|;
    the measured rms is a few units)."""
    import torch
    prob = ai.toy(6, 3, 19, split=(2, 2, 1))   # n_G up to ~500: two K chunks
    ctx = _ctx(B, prob, adaptive=0, precision=B.FP32)
    n = ctx.level_info(1).n_subs
    sizes = [int(ctx.export(B.X_SUB_SIZES, 1, s, np.int32)[1]) for s in range(n)]
    assert max(sizes) > 256
    gen = torch.Generator(device="cuda").manual_seed(9)
    for width in (64, 100):
        x = torch.randn(sum(sizes) * width, dtype=torch.float32, device="cuda", generator=gen)
        y = torch.empty_like(x)
        ctx.schur_apply(1, width, x, y)
        xh, yh = x.cpu().numpy().astype(np.float64), y.cpu().numpy().astype(np.float64)
        o = 0
        for s, ng in enumerate(sizes):
            S = ctx.export(B.X_SCHUR, 1, s, np.float64).reshape(ng, ng, order="F")   # the FP32 S, exported as FP64
            X = xh[o:o + ng * width].reshape(ng, width, order="F")
            Y = yh[o:o + ng * width].reshape(ng, width, order="F")
            bound = 64 * 2.0 ** -24 * (np.abs(S) @ np.abs(X)) + 1e-30
            assert np.all(np.abs(Y - S @ X) <= bound), (width, s)
            o += ng * width
    ctx.close()


def test_host_made_failures(B):
    prob = ai.toy(3, 1, 18, split=(2, 1, 1))
    bad = prob.coeff.copy()
    bad[3] = -1.0
    with pytest.raises(B.AmbError) as e:
        B.Context.from_problem(prob, coeff=bad)
    assert e.value.status == B.EINVAL
    ctx = _ctx(B, prob, pcg_maxit=1, adaptive=0)
    f = ctx.load_vector(prob.body)
    with pytest.raises(B.AmbError) as e:
        ctx.solve(f)
    assert e.value.status == B.ENOCONV
    fn = f.copy()
    fn[5] = np.nan
    with pytest.raises(B.AmbError):
        ctx.solve(fn)
    ctx.close()
