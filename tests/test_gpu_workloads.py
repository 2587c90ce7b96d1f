"""Full-size parity on the benchmark workloads against stored oracle values
(tests/golden/config*_oracle.json, written by tests/golden/make_golden.py from
oracle/ only).  Sampled outputs the oracle computed one by one: PCG
iterations, adaptive rows per face, the indicator, and the top pair
eigenvalues of the used columns.  The solution is checked against a sparse
direct solve (16^3) or through its residual in the oracle's own assembly (48^3).

FP64 form: eigenvalues within 1e-4 relative, selected rows per face and PCG
iterations within +-1 of the oracle.

FP32 form (factorizations and preconditioner in FP32, trailing updates on the
tensor cores in 3xTF32): the Schur complements carry FP32 rounding, which
moves the pair eigenvalues that sit on near-null directions of S.  The
rigid modes of floating substructures are projected out of the B products
(exact for the FP64 S), which removes most of it: on the 48^3 elasticity
workload the deviation is 1.3e-4 at most and 1.9e-6 in the median (3.2e-2 and
1.8e-4 without the projection).  The 1e4-contrast channels have further
near-null modes (the stiff channels inside floating substructures) that no
projection removes: 3.0e-3 at most, 2.7e-4 in the median.  LOBPCG itself
agrees with its own FP32 pencil to <= 1e-7 (test_gpu_fp32_form.py), so these
are the FP32 pencil's errors.  Bounds (measured behaviour with a margin):
48^3 max 5e-4, median 2e-5; 16^3 channels max 1e-2, median 2e-3; selected
rows per face identical within +-1, PCG iterations within +1 of the oracle
(48^3: 38 vs 37; 16^3 channels: 16 vs 15, the FP64 form's count).  The constraint space (G = C_D
S_DD^-1 C_D^T, its inverse, the coarse basis) is FP64 in both forms; with it
in FP32 the 1e4-contrast channels workload took 18 to 34 iterations depending
on rounding order.
"""
import json
import os

import numpy as np
import pytest

import amb_inputs as ai
from crops import crop_around
from oracle import fe

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1301_0191_gb300 import binding
    return binding


def _gold(i):
    with open(os.path.join(GOLD, f"config{i}_oracle.json")) as f:
        return json.load(f)


@pytest.mark.parametrize("index,precision,rtol_max,rtol_med,it_slack",
                         [(1, "fp64", 1e-4, 1e-4, 1), (2, "fp64", 1e-4, 1e-4, 1),
                          (1, "fp32", 1e-2, 2e-3, 1), (2, "fp32", 5e-4, 2e-5, 1)])
def test_workload_against_oracle(B, index, precision, rtol_max, rtol_med, it_slack):
    g = _gold(index)
    prob = ai.config(index)
    prec = B.FP64 if precision == "fp64" else B.FP32
    ctx = B.Context.from_problem(prob, precision=prec, lobpcg_tol=1e-6, lobpcg_maxit=200)
    f = ctx.load_vector(prob.body)
    u, info = ctx.solve(f)
    rep = ctx.report()
    ctx.close()
    assert info.rel_residual <= 1e-8 and info.true_rel_residual <= 1.01e-8
    assert -1 <= info.iterations - g["pcg_iterations"] <= it_slack, (info.iterations, g["pcg_iterations"])
    free = fe.free_dof_map(prob)[1]
    if index == 1:
        # the solution against a sparse direct solve of the oracle's assembly (4,624 dofs)
        import scipy.sparse.linalg as spla
        ud = spla.spsolve(fe.assemble_global(prob).tocsc(), fe.load_vector(prob))
        assert np.linalg.norm(u[free] - ud) <= 1e-6 * np.linalg.norm(ud)
    else:
        # 345,744 dofs: the solution through its residual in the oracle's own assembly and load
        # (a sparse direct solve of 3-D elasticity at this size takes minutes and tens of GB)
        f_o = fe.load_vector(prob)
        true_rel = np.linalg.norm(f_o - fe.assemble_global(prob) @ u[free]) / np.linalg.norm(f_o)
        assert true_rel <= 1.01e-8, true_rel
    pairs = {(p["s"], p["t"]): p for p in rep["pairs"]}
    assert len(pairs) == len(g["pairs"])
    off = 0
    dev = []
    for (s, t), k_o, lam_o in zip(g["pairs"], g["n_selected"], g["lambda_top"]):
        pr = pairs[(s, t)]
        assert abs(pr["n_selected"] - k_o) <= 1
        for i in range(min(len(lam_o), pr["n_selected"] + 1)):
            if lam_o[i] >= 0.1 * prob.tau:
                dev.append((abs(pr["lam"][i] - lam_o[i]) / lam_o[i], (s, t), i))
        off += abs(pr["n_selected"] - k_o)
    worst = max(dev)
    assert worst[0] <= rtol_max, worst
    assert float(np.median([d[0] for d in dev])) <= rtol_med
    assert abs(rep["n_adaptive"][0] - g["n_adaptive"][0]) <= max(2, off)
    # the indicator omega is a pair eigenvalue: same bound
    assert abs(rep["omega_level"][0] - g["omega_level"][0]) <= rtol_max * g["omega_level"][0] + 1e-3


# ---------------------------------------------------------------------------
# 96^3 Poisson, 512 irregular boxes (6..14 elements a side), slabs of 1e6,
# three levels: too large for the whole oracle, so the oracle computes sampled
# outputs one by one, on crops of the mesh around the sampled faces
# (tests/crops.py; the locality it relies on is pinned by test_oracle_crop.py).

def test_irregular_three_level_workload_sampled(B):
    """Every check is collected and reported together.  FP64 form: S^s to
    1e-9 and pair eigenvalues above tau/10 to 1e-4 relative, selected rows
    +-1 against the oracle on the sampled faces.  Both forms: the 1e-8
    residual in the oracle's own assembly, and Algorithm 3's selection rule
    and indicator on every face of both levels."""
    from oracle import levels as olv, pair as opr

    prob = ai.config(3)
    tau, cap = prob.tau, 10
    a_full = fe.assemble_global(prob)
    f_o = fe.load_vector(prob)
    free = fe.free_dof_map(prob)[1]          # the library's vectors live on all mesh dofs
    bad, res = [], {}
    for name, prec in (("fp64", B.FP64), ("fp32", B.FP32)):
        ctx = B.Context.from_problem(prob, precision=prec, lobpcg_tol=1e-6, lobpcg_maxit=200)
        f = ctx.load_vector(prob.body)
        assert np.allclose(f[free], f_o, rtol=1e-12, atol=1e-16)
        u, info = ctx.solve(f)
        rep = ctx.report()
        # the solution through its residual in the oracle's own FP64 assembly
        true_rel = np.linalg.norm(f_o - a_full @ u[free]) / np.linalg.norm(f_o)
        if not (info.rel_residual <= 1e-8 and true_rel <= 1.01e-8):
            bad.append((name, "residual", info.rel_residual, true_rel))
        # Algorithm 3's selection on every level: the leading eigenvalues above
        # tau, at most `cap` of them; the indicator (eq. cond-ind-mlevel) is the
        # largest first eigenvalue left out
        assert rep["n_levels"] == 2
        assert sum(1 for p in rep["pairs"] if p["level"] == 1) == 1344
        for lvl in (1, 2):
            om = 0.0
            for p in (q for q in rep["pairs"] if q["level"] == lvl):
                lam, k = p["lam"], p["n_selected"]
                # the used values (selected and the indicator) descending; at
                # the tail, directions dropped as B-null report 0 after
                # negative rounding-level values
                ok = bool(np.all(np.diff(lam[:k + 1]) <= 0.0))
                ok = ok and bool(np.all(lam[:k] > tau)) and k <= cap
                if k < len(lam):
                    ok = ok and (k == cap or lam[k] <= tau)
                    om = max(om, lam[k])
                if not ok:
                    bad.append((name, "selection", lvl, p["s"], p["t"], k, lam[:k + 2].tolist()))
            if rep["omega_level"][lvl - 1] != om:
                bad.append((name, "indicator", lvl, rep["omega_level"][lvl - 1], om))
        res[name] = (ctx, info, rep)
        if name != "fp64":
            continue
        # LOBPCG on the FP64 form: the stiff-slab faces (lambda_1 ~ 3e5)
        # converge by their Ritz values; a pair that ends with a residual
        # above 1e-2 has not found its eigenvectors (measured: 12 of 1344)
        lost = [(p["s"], p["t"]) for p in rep["pairs"] if p["level"] == 1 and p["residual"] > 1e-2]
        print(f"fp64 level-1 pairs with residual > 1e-2: {len(lost)} of 1344")
        if len(lost) > 27:
            bad.append(("lobpcg", len(lost), lost[:10]))
        # sampled against the oracle on crops: the face with the most rows, the
        # face with the largest pair eigenvalue, the face that sets the
        # indicator (its lambda_{k+1} is the level's omega, just below tau),
        # a seeded random face
        lv1 = [p for p in rep["pairs"] if p["level"] == 1]
        picks = [max(lv1, key=lambda p: (p["n_selected"], p["lam"][0])),
                 max(lv1, key=lambda p: p["lam"][0]),
                 max(lv1, key=lambda p: p["lam"][p["n_selected"]] if p["n_selected"] < len(p["lam"]) else 0.0),
                 lv1[int(np.random.default_rng(np.random.PCG64(3)).integers(len(lv1)))]]
        seen = set()
        for p in picks:
            s, t = p["s"], p["t"]
            if (s, t) in seen:
                continue
            seen.add((s, t))
            crop, sub_map, dof_map = crop_around(prob, s, t)
            inv = {v: k for k, v in sub_map.items()}
            lev = olv.level_one(crop)
            lev.schur()
            for sub in (s, t):
                sb = lev.subs[inv[sub]]
                dofs = ctx.export(B.X_SUB_DOFS, 1, sub, np.int64)
                ni, ng = (int(x) for x in ctx.export(B.X_SUB_SIZES, 1, sub, np.int32)[:2])
                assert ni == sb.n_i and ng == sb.n_g
                assert np.array_equal(np.sort(dofs[:ni]), np.sort(dof_map[sb.idofs]))
                pos = {int(dd): i for i, dd in enumerate(dof_map[sb.gdofs])}
                perm = np.array([pos[int(dd)] for dd in dofs[ni:]])
                S = ctx.export(B.X_SCHUR, 1, sub, np.float64).reshape(ng, ng, order="F")
                err = np.abs(S - sb.s[np.ix_(perm, perm)]).max() / np.abs(sb.s).max()
                if not err <= 1e-9:
                    bad.append(("schur", sub, err))
            cs, ct = inv[s], inv[t]
            r = opr.solve_pair(lev, min(cs, ct), max(cs, ct), tau, max_per_face=cap)
            lo = np.sort(r.lam)[::-1]
            dev = [abs(p["lam"][i] - lo[i]) / lo[i]
                   for i in range(min(len(lo), len(p["lam"]), p["n_selected"] + 1)) if lo[i] >= 0.1 * tau]
            if abs(p["n_selected"] - r.n_selected) > 1 or max(dev, default=0.0) > 1e-4:
                bad.append(("pair", s, t, p["n_selected"], r.n_selected, max(dev, default=0.0)))
            print(f"pair {(s, t)}: rows {p['n_selected']} (oracle {r.n_selected}), lam1 {p['lam'][0]:.8g} "
                  f"(oracle {lo[0]:.8g}), max rel dev {max(dev, default=0.0):.2e}")
    # the FP32 form against the FP64 form: iterations within +-2 and adaptive
    # rows per level within 2% (the FP32 pencil moves eigenvalues near tau)
    (_, i64, r64), (_, i32, r32) = res["fp64"], res["fp32"]
    if abs(i32.iterations - i64.iterations) > 2:
        bad.append(("iterations", i64.iterations, i32.iterations))
    for lvl in range(2):
        if abs(r32["n_adaptive"][lvl] - r64["n_adaptive"][lvl]) > max(2, 0.02 * r64["n_adaptive"][lvl]):
            bad.append(("rows", lvl, r64["n_adaptive"][lvl], r32["n_adaptive"][lvl]))
    print(f"its fp64 {i64.iterations} fp32 {i32.iterations}; rows {r64['n_adaptive']} / {r32['n_adaptive']}; "
          f"omega {r64['omega_level']} / {r32['omega_level']}")
    for c, _, _ in res.values():
        c.close()
    for b in bad:
        print("violation:", b)
    assert not bad, bad
