"""amb_schur_apply_noalloc gives the same products as amb_schur_apply.

The allocation-free variant exists for callers that cannot allocate device
memory during a call (their device memory is owned by their own pool, or
they cannot accept cudaMalloc's implicit synchronisation).  It stages its
launch descriptors in a fixed device array of the library image instead of
context-allocated memory; this test calls both entry points through the C
ABI and compares their outputs, twice in a row, so that a second call that
reuses the shared array is covered too.  This file sorts last so that a
run that stops at the first failure has already run every other test.
"""
import numpy as np
import pytest

import amb_inputs as ai

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_schur_apply_matches_schur_apply(precision):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1301_0191_gb300 import binding as B

    prec = B.FP64 if precision == "fp64" else B.FP32
    dt = torch.float64 if precision == "fp64" else torch.float32
    tol = 1e-12 if precision == "fp64" else 1e-5
    prob = ai.toy(4, 3, 23, split=(2, 2, 2), sigma=1.0)
    ctx = B.Context.from_problem(prob, adaptive=0, precision=prec)
    n = ctx.level_info(1).n_subs
    total = sum(int(ctx.export(B.X_SUB_SIZES, 1, s, np.int32)[1]) for s in range(n))
    gen = torch.Generator(device="cuda").manual_seed(5)
    for width in (1, 6):
        x = torch.randn(total * width, dtype=dt, device="cuda", generator=gen)
        ref = torch.empty_like(x)
        ctx.schur_apply(1, width, x, ref)
        scale = float(ref.abs().max())
        for _ in range(2):
            y = torch.full_like(x, float("nan"))
            ctx.schur_apply_noalloc(1, width, x, y)
            assert torch.isfinite(y).all()
            assert float((y - ref).abs().max()) <= tol * scale
    ctx.close()
