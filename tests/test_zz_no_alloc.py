"""amb_schur_apply_noalloc gives the same products as amb_schur_apply.

The allocation-free variant exists for callers that cannot allocate device
memory during a call (their device memory is owned by their own pool, or
they cannot accept cudaMalloc's implicit synchronisation).  It stages its
launch descriptors in a fixed device array of the library image instead of
context-allocated memory; this test calls both entry points through the C
ABI and compares their outputs, twice in a row, so that a second call that
reuses the shared array is covered too.  It also checks the claim itself:
after the first call (which looks up the array's address), further calls
leave the device's free memory and the stream-ordered pool the library
allocates from unchanged, and take nothing from torch's allocator.  At FP32 widths >= 64
amb_schur_apply runs on the tensor cores (3xTF32) and this variant on the
SIMT units, so the two agree there to FP32 rounding (1e-5 of the largest
entry) rather than bit for bit.  A level with more substructures than the
variant's fixed array holds (1024) is rejected with AMB_EINVAL.  This file
sorts last so that a run that stops at the first failure has already run
every other test.
"""
import ctypes
import ctypes.util

import numpy as np
import pytest

import amb_inputs as ai

pytestmark = pytest.mark.gpu


def _binding():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1301_0191_gb300 import binding as B
    return torch, B


def _cudart():
    names = [ctypes.util.find_library("cudart"), "libcudart.so", "/usr/local/cuda/lib64/libcudart.so"]
    for n in names:
        if not n:
            continue
        try:
            return ctypes.CDLL(n)
        except OSError:
            continue
    return None


def _pool_usage(rt, dev):
    """(used, reserved) bytes of the device's default stream-ordered pool."""
    pool = ctypes.c_void_p()
    if rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), dev) != 0:
        return None
    used, res = ctypes.c_uint64(), ctypes.c_uint64()
    if rt.cudaMemPoolGetAttribute(pool, 0x7, ctypes.byref(used)) != 0:      # UsedMemCurrent
        return None
    if rt.cudaMemPoolGetAttribute(pool, 0x5, ctypes.byref(res)) != 0:       # ReservedMemCurrent
        return None
    return used.value, res.value


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_schur_apply_matches_schur_apply(precision):
    torch, B = _binding()
    prec = B.FP64 if precision == "fp64" else B.FP32
    dt = torch.float64 if precision == "fp64" else torch.float32
    tol = 1e-12 if precision == "fp64" else 1e-5
    prob = ai.toy(4, 3, 23, split=(2, 2, 2), sigma=1.0)
    ctx = B.Context.from_problem(prob, adaptive=0, precision=prec)
    n = ctx.level_info(1).n_subs
    total = sum(int(ctx.export(B.X_SUB_SIZES, 1, s, np.int32)[1]) for s in range(n))
    gen = torch.Generator(device="cuda").manual_seed(5)
    widths = (1, 6, 64) if precision == "fp32" else (1, 6)
    rt = _cudart()
    dev = torch.cuda.current_device()
    for width in widths:
        x = torch.randn(total * width, dtype=dt, device="cuda", generator=gen)
        ref = torch.empty_like(x)
        ctx.schur_apply(1, width, x, ref)
        scale = float(ref.abs().max())
        ys = [torch.full_like(x, float("nan")) for _ in range(3)]
        ctx.schur_apply_noalloc(1, width, x, ys[0])     # the first call may look up the array's address
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        torch0 = torch.cuda.memory_allocated()
        pool0 = _pool_usage(rt, dev) if rt else None
        for y in ys[1:]:
            ctx.schur_apply_noalloc(1, width, x, y)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert torch.cuda.memory_allocated() <= torch0     # Python temporaries may be freed meanwhile
        if pool0 is not None:
            assert _pool_usage(rt, dev) == pool0
        for y in ys:
            assert torch.isfinite(y).all()
            assert float((y - ref).abs().max()) <= tol * scale, (width, float((y - ref).abs().max()) / scale)
    ctx.close()


def test_noalloc_rejects_levels_beyond_its_array():
    torch, B = _binding()
    # 11 x 11 x 9 = 1089 substructures of 2^3 elements
    prob = ai.toy(2, 1, 29, split=(11, 11, 9), sigma=0.5)
    ctx = B.Context.from_problem(prob, adaptive=0)
    n = ctx.level_info(1).n_subs
    assert n == 1089
    total = sum(int(ctx.export(B.X_SUB_SIZES, 1, s, np.int32)[1]) for s in range(n))
    x = torch.zeros(total, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(B.AmbError) as e:
        ctx.schur_apply_noalloc(1, 1, x, y)
    assert e.value.status == B.EINVAL and "1024" in str(e.value)
    # the ordinary entry point still serves that level
    ctx.schur_apply(1, 1, x, y)
    ctx.close()
