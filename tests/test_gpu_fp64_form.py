"""FP64 form: Schur complements through several tensor-core trailing updates.

The FP64 form's trailing update C -= P P^T runs on the TF32 tensor cores
from exact slice products (every row of P cut into eight 7-bit integer
slices, per-level exact integer sums, one rounding to FP64 per entry).
Substructures with more than 256 interior dofs take several outer blocks,
so their Schur complement S = K_GG - K_GI K_II^-1 K_IG (Sec. 3) passes
through several such updates, each with a ragged last tile.

Bound: both sides are backward-stable FP64 computations of S, so they
differ by about n u kappa(K_II) |S| with n ~ 10^3 interior dofs, u = 2^-53
and kappa(K_II) ~ 10^2 for these meshes and coefficient contrasts, i.e.
~10^-11 of the largest entry; the test asks for 1e-11.  A trailing update
of FP32 accuracy (3xTF32) would be off by ~10^-6 and fails it.
"""
import numpy as np
import pytest

import amb_inputs as ai
from oracle import fe, levels as olv

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


@pytest.mark.parametrize("sub,dpn,split,seed", [(8, 3, (2, 1, 1), 41), (12, 1, (2, 1, 1), 42), (8, 3, (2, 2, 1), 43)])
def test_fp64_schur_through_several_trailing_updates(B, sub, dpn, split, seed):
    prob = ai.toy(sub, dpn, seed, split=split, sigma=1.5)
    ctx = B.Context.from_problem(prob, adaptive=0)
    lev = olv.level_one(prob)
    lev.schur()
    free = fe.free_dof_map(prob)[1]
    worst = 0.0
    for s, sb in enumerate(lev.subs):
        assert sb.n_i > 256   # several outer blocks of 256 columns
        dofs = ctx.export(B.X_SUB_DOFS, 1, s, np.int64)
        ni, ng = int(sb.n_i), int(sb.n_g)
        pos = {int(d): i for i, d in enumerate(free[sb.gdofs])}
        perm = np.array([pos[int(d)] for d in dofs[ni:]])
        S = ctx.export(B.X_SCHUR, 1, s, np.float64).reshape(ng, ng, order="F")
        So = sb.s[np.ix_(perm, perm)]
        err = np.abs(S - So).max() / np.abs(So).max()
        worst = max(worst, err)
        print(f"sub {s}: n_I {ni} n_G {ng} max |S - S_oracle| / max |S| = {err:.3e}")
        assert err <= 1e-11, (s, err)
    ctx.close()


@pytest.mark.parametrize("sub,dpn", [(12, 1), (9, 3)])
def test_fp64_interior_inverse_through_the_tensor_core_merges(B, sub, dpn):
    """One substructure, no interface: the preconditioner is the interior
    solve Z^T Z with Z = L_I^-1 merged block by block on the tensor cores
    (K up to 1024, several chunks per merge), so one PCG step leaves the
    residual (I - K Z^T Z) f.  For Z to FP64 accuracy that is about
    kappa(K) u ~ 10^3 x 1e-16; the test asks for 1e-11 (a Z of FP32 accuracy
    leaves ~1e-4)."""
    prob = ai.toy(sub, dpn, 44 + dpn, split=(1, 1, 1), sigma=1.5)
    lev = olv.level_one(prob)
    assert lev.subs[0].n_i > 2000 and lev.subs[0].n_g == 0
    ctx = B.Context.from_problem(prob, adaptive=0)
    f = ctx.load_vector(prob.body)
    u, info = ctx.solve(f)
    print(f"n_I {lev.subs[0].n_i}: iterations {info.iterations}, relative residual {info.rel_residual:.3e}")
    assert info.iterations == 1
    assert info.rel_residual <= 1e-11
    ctx.close()
