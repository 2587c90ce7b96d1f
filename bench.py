"""Benchmark: adaptive-BDDC set-up + solve to a 1e-8 relative residual on the
3D elasticity workload (48^3 Q1 hexahedra, 4x4x4 substructures of 12^3
elements, lognormal Young's modulus sigma 1.5, nu 0.3, clamped face, unit
body force, two levels, adaptive faces at tau = 10), plus the batched
Schur-apply roofline fraction.

One step = amb_setup + amb_solve through the C ABI with coefficients and
right-hand side already in HBM.  The factor working set (tens of GB) is far
larger than the 129 MB L2, so no flush is needed between steps.

--impl reference times the CPU FP64 oracle on a bounded sample of the same
workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import amb_inputs as ai  # noqa: E402

METRIC = "adaptive-BDDC setup+solve s to 1e-8 rel. residual; Schur-apply % of roofline"
WORKLOAD = "elasticity48_4x4x4_lognormal"
# DRAM bytes per 128 x 128 output tile of the tensor-core trailing update, from one ncu capture of that kernel
# on the 2x2x2 corner block of the 48^3 workload (its first launch, the update after the first 256 columns:
# 699.54 MB read + 536.97 MB written over 9424 tiles; None when the kernel has changed since)
TC_TRAFFIC_PER_TILE = 1236.51e6 / 9424
TC_OUTER, TC_TILE = 256, 128
# DRAM bytes (read + write) of one B apply of the LOBPCG operator products on the 48^3 workload, from one
# 1-pass ncu capture of the timed step (None when the kernel has changed since)
TRAFFIC_GEMM_DF_B = 1.11e9 + 0.040e9


def max_over_ranks(ms, world, device):
    """The slowest rank's time per step: every rank runs one replica of the workload, so the job's time is
    the maximum (all-reduce MAX over the process group; the identity on one rank)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def tc_tiles(n_i, n_g, n_d):
    """Output tiles of all trailing updates of one set-up: the interior factorization (columns 0..n_I of the
    (n_I + n_G)-square matrix) and the corner-constrained Neumann one (columns n_I..n_I + n_D), one update per
    256-column outer block, lower-triangular tiles of the remaining rows."""
    t = 0
    for ni, ng, nd in zip(n_i.astype(int), n_g.astype(int), n_d.astype(int)):
        n = ni + ng
        for c0, c1 in ((0, ni), (ni, ni + nd)):
            for j1 in range(c0 + TC_OUTER, c1 + TC_OUTER, TC_OUTER):
                rem = n - min(j1, c1)
                tm = -(-rem // TC_TILE)
                if rem > 0:
                    t += tm * (tm + 1) // 2
    return t


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# cuBLAS GEMM rates measured on this machine's GB300 with `bench.py --measure-peaks` (8192^3, best of
# three, torch matmul): TF32 tensor cores 1052 TFLOP/s, FP64 1.10 TFLOP/s, FP32 without tensor cores
# 69.7 TFLOP/s, BF16 2015 TFLOP/s (MEASURED_PEAKS.json's BF16 burst: 1913).  The TF32 peak below is
# the driver's measured BF16 burst times the measured TF32/BF16 ratio (0.522; nominal 1.1/2.25 = 0.489).
MEASURED_TF32_PER_BF16 = 1051.8 / 2015.5
MEASURED_FP64_TFLOPS = 1.10


def measure_peaks():
    """cuBLAS GEMM throughput (through torch) for the roofline denominators."""
    def rate(dtype, n, reps, tf32=True):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        a = torch.randn(n, n, device="cuda", dtype=dtype)
        b = torch.randn(n, n, device="cuda", dtype=dtype)
        for _ in range(3):
            a @ b
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            a @ b
        e1.record()
        torch.cuda.synchronize()
        return 2 * n ** 3 / (e0.elapsed_time(e1) / reps * 1e-3) / 1e12
    out = {"tf32_tflops": max(rate(torch.float32, 8192, 20) for _ in range(3)),
           "fp32_no_tensor_tflops": max(rate(torch.float32, 8192, 5, False) for _ in range(2)),
           "fp64_tflops": max(rate(torch.float64, 8192, 3) for _ in range(2)),
           "bf16_tflops": max(rate(torch.bfloat16, 8192, 20) for _ in range(3)),
           "method": "cuBLAS GEMM through torch, 8192^3, best of several"}
    print(json.dumps(out))


# ---------------------------------------------------------------- clocks
class Clocks:
    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, gpu_index=0):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9 or p[0] != str(gpu_index):
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        busy = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- oracle sample
# PCG iterations of the oracle on the full workloads (tests/golden for 48^3; the 96^3 three-level workload is
# too large for the whole oracle, so its estimate uses the library's FP64-form count, 30; so does the 64^3
# Poisson workload of the gradient, whose stored oracle run solved to 1e-12 for the gradient check)
ORACLE_ITS = {"c2": 37, "c3": 30, "c4": 30}
CONFIG_INDEX = {"c2": 2, "c2block": 2, "c3": 3, "c4": 4}


def oracle_sample(prob, its_full=37):
    """The CPU oracle on a bounded sample of the workload, an ESTIMATE of the
    whole oracle's time: set-up of the 2x2x1 block of level-1 substructures at
    the clamped face (same substructure shapes and coefficient field) and one
    Algorithm-1 application, scaled by (substructures / 4) and by the PCG
    iteration count on the full workload."""
    from oracle import fe, solver
    sub = ai.sub_block(prob, (2, 2, 1))
    t0 = time.perf_counter()
    h = solver.Hierarchy(sub)
    t_setup = time.perf_counter() - t0
    f = fe.load_vector(sub)
    t1 = time.perf_counter()
    z = h.apply(f)
    _ = h.ops[0] @ z
    t_iter = time.perf_counter() - t1
    scale = prob.n_subs(1) / 4.0
    est = scale * (t_setup + its_full * t_iter)
    return est, time.perf_counter() - t0, dict(t_setup=t_setup, t_iter=t_iter)


def oracle_full_c1():
    """The whole oracle (set-up of all 8 substructures, every pair eigenproblem, PCG to 1e-8) on the 16^3
    channels workload, timed: a complete run, not an extrapolation."""
    from oracle import solver
    prob = ai.config(1)
    t0 = time.perf_counter()
    _, res, _ = solver.solve(prob)
    return time.perf_counter() - t0, res.its


def cpu_threads():
    try:
        from threadpoolctl import threadpool_info
        return max(int(i.get("num_threads", 1)) for i in threadpool_info()) or os.cpu_count()
    except Exception:
        return os.cpu_count()


# ---------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-form", action="store_true")
    ap.add_argument("--workload", default="c2", choices=["c2", "c2block", "c3", "c4"],
                    help="c2: the 48^3 elasticity workload; c3: the 96^3 Poisson workload on 512 irregular "
                         "boxes, three levels; c4: the 64^3 Poisson workload on a Gaussian random field, with "
                         "the compliance gradient (amb_grad) in every step; c2block: a corner block of the c2 "
                         "substructures (same shapes; 2x1x1 holds ~0.5 GB on the device), for profiler captures")
    ap.add_argument("--block", default="2,1,1", help="substructures per axis of the c2block workload")
    ap.add_argument("--profile", action="store_true",
                    help="warm-up + timed steps only (no e2e, family timing, Schur sweep or baselines)")
    ap.add_argument("--measure-peaks", action="store_true",
                    help="print the cuBLAS GEMM rates (TF32, FP32, FP64, BF16) used as roofline peaks, then exit")
    args = ap.parse_args()
    if args.measure_peaks:
        measure_peaks()
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    prob = ai.config(CONFIG_INDEX[args.workload])
    workload = prob.name
    its_full = ORACLE_ITS[args.workload if args.workload in ORACLE_ITS else "c2"]
    with_grad = args.workload == "c4"
    if args.workload == "c2block":
        prob = ai.sub_block(prob, tuple(int(v) for v in args.block.split(",")))
        workload = prob.name
    sample_desc = (f"ESTIMATE, not a complete run: oracle set-up of 4 of {prob.n_subs(1)} level-1 substructures "
                   f"(2x2x1 block at the clamped face) + one Algorithm-1 application, scaled by "
                   f"{prob.n_subs(1) / 4:g} and by {its_full} PCG iterations"
                   + ("; the compliance gradient (one element loop) is not in it" if args.workload == "c4" else ""))

    if args.impl == "reference":
        if rank != 0:
            return
        for _ in range(args.warmup):
            oracle_sample(prob, its_full)
        vals, wall = [], 0.0
        for _ in range(args.steps):
            est, w, _ = oracle_sample(prob, its_full)
            vals.append(est)
            wall += w
        v = statistics.mean(vals)
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * v, "higher_is_better": False,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": workload, "levels": prob.levels, "tau": prob.tau},
                "estimate": True,
                "cpu_baseline": {"kind": "oracle", "value": v, "unit": "s", "cores": cpu_threads(),
                                 "sample": sample_desc, "sample_wall_s_total": wall},
                "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1301_0191_gb300 import binding as B

    prec = B.FP32 if args.precision == "fp32" else B.FP64
    coeff_d = torch.tensor(prob.coeff, dtype=torch.float64, device="cuda")
    # right-hand side: consistent loads of the unit body force, computed once by the library
    c0 = B.Context.from_problem(prob, adaptive=0, precision=prec)
    f_h = c0.load_vector(prob.body)
    c0.close()
    f_d = torch.tensor(f_h, device="cuda")
    u_d = torch.empty_like(f_d)
    opts = dict(precision=prec, lobpcg_maxit=200, lobpcg_tol=1e-6, pcg_rtol=1e-8)

    g_d = torch.empty(prob.n_el, dtype=torch.float64, device="cuda") if with_grad else None

    def step(timing=0):
        c = B.Context.from_problem(prob, coeff=coeff_d, timing_events=timing, **opts)
        _, info = c.solve(f_d, out=u_d)
        if with_grad:
            c.grad(B.QOI_COMPLIANCE, out=g_d)
        return c, info

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        c, info = step()
        c.close()
    clocks = Clocks()
    barrier()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    e0.record()
    infos = []
    for _ in range(args.steps):
        c, info = step()
        infos.append(info)
        launches += c.stats()["kernels_launched"]
        c.close()
    e1.record()
    barrier()
    clk = clocks.stop(local)
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, "cuda")
    if args.profile:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": ms * 1e-3, "unit": "s", "profile_run": True,
                              "config": {"workload": workload}, "pcg_iterations": infos[-1].iterations,
                              "gpu_launches": int(launches / args.steps)}))
        if world > 1:
            dist.destroy_process_group()
        return

    # end to end: host coefficients / rhs / solution, copies inside the timed region
    coeff_h = np.ascontiguousarray(prob.coeff)
    u_h = np.empty_like(f_h)
    g_h = np.empty(prob.n_el) if with_grad else None
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        c = B.Context.from_problem(prob, coeff=coeff_h, **opts)
        c.solve(f_h, out=u_h)
        if with_grad:
            c.grad(B.QOI_COMPLIANCE, out=g_h)
        c.close()
    barrier()
    e2e_s = (time.perf_counter() - t0) / args.steps
    h2d = coeff_h.nbytes + f_h.nbytes + prob.dirichlet_node_mask.nbytes + prob.elem_to_sub.nbytes
    d2h = u_h.nbytes + (g_h.nbytes if with_grad else 0)

    # kernel-family timing (separate, untimed run with CUDA events per family)
    c, info = step(timing=1)
    st = c.stats()
    li = c.level_info(1)
    rep = c.report()
    peaks, src = _peaks()
    fams = st["families"]
    fp = "fp32" if prec == B.FP32 else "fp64"
    # SIMT FP32: 152 SMs x 128 lanes x 2 flops x max SM clock; FP64: the measured cuBLAS FP64 GEMM rate
    alu_peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12 if fp == "fp32" else MEASURED_FP64_TFLOPS
    # TF32 tensor peak: the measured dense BF16 burst times the measured cuBLAS TF32/BF16 ratio
    tf32_peak = peaks["bf16_tflops"] * MEASURED_TF32_PER_BF16
    # per-substructure sizes of level 1: (n_I, n_Gamma, n_corner, n_c)
    sz = np.array([c.export(B.X_SUB_SIZES, 1, s, np.int32)[:4] for s in range(li.n_subs)], dtype=np.float64)
    n_i, n_g, n_d = sz[:, 0], sz[:, 1], sz[:, 1] - sz[:, 2]
    sizes = [int(v) for v in n_g]
    # factorization a2-a5: algorithmic flops sum(n_I^3/3 + n_I^2 n_G + n_I n_G^2 + n_D^3/3)
    fact_flops = float(np.sum(n_i ** 3 / 3 + n_i ** 2 * n_g + n_i * n_g ** 2 + n_d ** 3 / 3))
    f_ms = fams["factor"]["ms"]
    factorization = {"algorithmic_flops": fact_flops, "ms": f_ms,
                     "TFLOP/s": fact_flops / (f_ms * 1e-3) / 1e12 if f_ms > 0 else None,
                     "tf32_peak": tf32_peak, "frac_of_tf32_peak": fact_flops / (f_ms * 1e-3) / 1e12 / tf32_peak
                     if f_ms > 0 else None, "trtri_ms": fams["trtri"]["ms"],
                     "note": "factor family = Cholesky of A_II (whose trailing updates also form S) and of S_DD; "
                             "the explicit triangular inverses (trtri) are timed apart"}
    # the step's dominant kernel: the LOBPCG operator products (k_gemm_df, the A and B applies: FP32 S times
    # the FP64 block with the sum carried in FP32 pairs on the SIMT units).  Algorithmic work: 2 n k w flops
    # per product; algorithmic bytes: each substructure's S (B) and each pair side's S_ff (A) once per apply.
    lop = fams["lobpcg_products"]
    roofline = None
    if lop["ms"] > 0:
        ach = lop["flops"] / (lop["ms"] * 1e-3) / 1e12
        gbs = lop["bytes"] / (lop["ms"] * 1e-3) / 1e9
        sm_mhz = peaks.get("sm_max_mhz", 2070.0)
        if fp == "fp32":
            # FP32-pair multiply-adds: 11 FP32 instructions each (product split by an FMA, TwoSum, low word)
            pair_peak = 152 * 128 * sm_mhz * 1e6 / 11 * 2 / 1e12
            peak, peak_src = pair_peak, (f"derived FP32-pair multiply-add rate: 152 SMs x 128 FP32 lanes x "
                                         f"{sm_mhz:g} MHz / 11 instructions per multiply-add x 2 flops")
        else:
            peak, peak_src = alu_peak, "measured cuBLAS FP64 GEMM rate (1.10 TFLOP/s)"
        roofline = {"kernel": "k_gemm_df: LOBPCG A and B products S X (factor-precision S, FP64 block, "
                              "FP32-pair accumulation on the SIMT units)",
                    "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                    "frac_of_plain_fp32_simt": ach / alu_peak,
                    "traffic": TRAFFIC_GEMM_DF_B if args.workload == "c2" and fp == "fp32" else None,
                    "traffic_note": "DRAM bytes of one full B apply (all 144 pairs) from one ncu capture of the "
                                    "timed step (1-pass dram__bytes_read.sum + write); the algorithmic bytes of "
                                    "that apply (S of every substructure once) are 1.06e9",
                    "algorithmic_GB/s": gbs, "hbm_frac_algorithmic": gbs / peaks["hbm_gbs"],
                    "algorithmic_flops": lop["flops"], "algorithmic_bytes": lop["bytes"],
                    "launches": lop["launches"], "ms": lop["ms"], "peak_source": peak_src,
                    "units": "flops = 2 per multiply-add of S X, counted over the active columns; bytes = each "
                             "substructure's S (B) and each pair side's face block (A) once per apply"}
    # the factorization's kernel: the tensor-core trailing update (FP32 form)
    tc = fams["tc_trailing"]
    if fp == "fp32" and tc["ms"] > 0:
        ach = tc["flops"] / (tc["ms"] * 1e-3) / 1e12
        roofline_factor = {"kernel": "k_tc_syrk (+ k_tc_split): Cholesky trailing update C -= P P^T, 3xTF32 on tcgen05",
                    "bound": "tensor", "achieved": ach, "peak": tf32_peak, "unit": "TFLOP/s", "frac": ach / tf32_peak,
                    "tensor_pipe_frac": 3.0 * ach / tf32_peak,
                    "traffic": TC_TRAFFIC_PER_TILE * tc_tiles(n_i, n_g, n_d) / (tc["launches"] // 2)
                    if TC_TRAFFIC_PER_TILE and tc["launches"] >= 2 else None,
                    "traffic_note": "k_tc_syrk DRAM bytes per launch (each update = one k_tc_split + one k_tc_syrk "
                                    "launch): bytes per 128x128 tile from one ncu capture of one launch on the 2x2x2 "
                                    "corner block (9424 tiles) x this step's tiles / updates; the split pass is not "
                                    "included",
                    "algorithmic_bytes_per_tile": 2 * 4 * TC_TILE * TC_TILE,
                    "launches": tc["launches"], "ms": tc["ms"],
                    "peak_source": f"{src} bf16 dense burst x nominal TF32/BF16 ratio (of {src})",
                    "units": "flops = 2 per lower-triangle multiply-add; tensor_pipe_frac counts the three TF32 "
                             "products of each"}
    else:
        achieved = fact_flops / (f_ms * 1e-3) / 1e12 if f_ms > 0 else None
        roofline_factor = {"kernel": "batched partial Cholesky (k_chol_diag + k_gemm panel/trailing, FP64)",
                    "bound": "alu",
                    "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                    "frac": achieved / alu_peak if achieved else None, "traffic": None,
                    "peak_source": f"nominal {fp} rate"}
    # Algorithm-1 preconditioner: bytes per application streamed by the GEMVs (triangles of the explicit
    # inverses, K_IG twice, Psi twice)
    esz_f = 4 if fp == "fp32" else 8
    nc = sz[:, 3]
    pre_bytes = esz_f * float(np.sum(n_i ** 2 + n_d ** 2 + 2 * n_i * n_g + 2 * n_g * nc))
    pre = fams["precond"]
    # one application before the first PCG iteration and one after each non-final one
    precond = {"bytes_per_apply": pre_bytes, "applies": int(info.iterations), "ms": pre["ms"]}
    precond["GB/s"] = pre_bytes * precond["applies"] / (pre["ms"] * 1e-3) / 1e9 if pre["ms"] > 0 else None
    precond["hbm_frac"] = precond["GB/s"] / peaks["hbm_gbs"] if precond["GB/s"] else None
    # Schur apply at widths 1, 30, 180 (headline 2)
    tdt = torch.float32 if prec == B.FP32 else torch.float64
    esz = 4 if prec == B.FP32 else 8
    schur = {}
    for width in (1, 30, 180):
        x = torch.randn(sum(sizes) * width, dtype=tdt, device="cuda")
        y = torch.empty_like(x)
        for _ in range(3):
            c.schur_apply(1, width, x, y)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(10):
            c.schur_apply(1, width, x, y)
        b.record()
        torch.cuda.synchronize()
        t = a.elapsed_time(b) / 10 * 1e-3
        byts = sum(n * n * esz + 2 * n * width * esz for n in sizes)
        flops = sum(2.0 * n * n * width for n in sizes)
        schur[f"w{width}"] = {"ms": t * 1e3, "GB/s": byts / t / 1e9, "hbm_frac": byts / t / 1e9 / peaks["hbm_gbs"],
                              "TFLOP/s": flops / t / 1e12, "alu_frac": flops / t / 1e12 / alu_peak}
        if prec == B.FP32 and width >= 64:
            # tensor cores, 3xTF32: three TF32 products per useful multiply-add
            schur[f"w{width}"].update({"path": "tensor cores (3xTF32)",
                                       "tensor_pipe_frac": 3.0 * flops / t / 1e12 / tf32_peak})
    c.close()

    fp64_form = None
    if not args.no_fp64_form and prec == B.FP32:
        # one untimed FP64 step first: it pays the one-time tile tuning of the FP64 products, as the
        # warm-up steps do for the FP32 form
        # (the untimed step records the kernel families with CUDA events)
        fam64 = None
        for timed in (False, True):
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            c64 = B.Context.from_problem(prob, coeff=coeff_d, precision=B.FP64, lobpcg_maxit=200, lobpcg_tol=1e-6,
                                         timing_events=0 if timed else 1)
            _, i64 = c64.solve(f_d, out=u_d)
            b.record()
            torch.cuda.synchronize()
            if not timed:
                fam64 = c64.stats()["families"]
            c64.close()
        fp64_form = {"s": a.elapsed_time(b) * 1e-3, "iterations": i64.iterations,
                     "speedup_fp32": a.elapsed_time(b) / ms, "warmup": 1}
        tr = fam64["tc_trailing"]
        if tr["ms"] > 0:
            # the trailing updates C -= P P^T from exact slice products (k_oz_split + k_oz_gemm): FP64-accurate
            # flops (2 per lower-triangle multiply-add) per second, against the measured FP64 GEMM rate; each
            # multiply-add is 36 TF32 slice products, against the TF32 tensor peak
            rate = tr["flops"] / (tr["ms"] * 1e-3) / 1e12
            fp64_form["trailing_update"] = {
                "kernel": "k_oz_gemm (+ k_oz_split): C -= P P^T from eight 7-bit digit slices per entry on tcgen05",
                "ms": tr["ms"], "launches": tr["launches"], "fp64_tflops": rate,
                "vs_fp64_gemm_peak": rate / MEASURED_FP64_TFLOPS, "slice_product_tflops": 36 * rate,
                "tensor_frac": 36 * rate / tf32_peak,
                "note": "family time of the untimed FP64 step (CUDA events); the timed step runs without events"}
        fp64_form["families_ms"] = {k: round(v["ms"], 1) for k, v in fam64.items() if v["ms"] > 0}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        est, wall, parts = oracle_sample(prob, its_full)
        cpu = {"value": est, "unit": "s", "cores": cpu_threads(), "kind": "oracle", "estimate": True,
               "sample": sample_desc, "sample_wall_s": wall}
        # one complete oracle run beside it (16^3 channels, two levels, adaptive), and the library on the same
        # workload in both forms, set-up + solve, inputs on the host
        t_or, its_or = oracle_full_c1()
        p1 = ai.config(1)
        gpu_s = {}
        for name, pr1 in (("fp64", B.FP64), ("fp32", B.FP32)):
            for _ in range(2):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                c1 = B.Context.from_problem(p1, precision=pr1, lobpcg_maxit=200, lobpcg_tol=1e-6)
                f1 = c1.load_vector(p1.body)
                _, i1 = c1.solve(f1)
                c1.close()
                torch.cuda.synchronize()
                gpu_s[name] = {"s": time.perf_counter() - t0, "pcg_iterations": i1.iterations}
        cpu["complete_run"] = {"workload": p1.name, "oracle_s": t_or, "oracle_pcg_iterations": its_or,
                               "cores": cpu_threads(), "library_e2e": gpu_s,
                               "note": "the whole oracle, set-up (all pair eigenproblems) + PCG to 1e-8, timed; "
                                       "the library's times are the second of two runs, host inputs"}
    if rank == 0:
        last = infos[-1]
        line = {"metric": METRIC, "value": ms * 1e-3, "unit": "s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == B.FP32 else "f64",
                "data": "synthetic",
                "config": {"workload": workload, "levels": prob.levels, "tau": prob.tau, "dofs": int(li.n_dofs),
                           **({"step": "set-up + solve + compliance gradient"} if with_grad else {}),
                           "substructures": li.n_subs, "pairs": li.n_pairs, "l2": "working set >> L2 (no flush)",
                           "replicas": "one independent problem per GPU"},
                "pcg_iterations": last.iterations, "rel_residual": last.rel_residual,
                "true_rel_residual": last.true_rel_residual, "cond_estimate": last.cond_estimate,
                "n_adaptive": rep["n_adaptive"], "omega": rep["omega"],
                "phase_ms": st["phase_ms"],
                "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
                "gpu_launches": int(launches / args.steps), "clocks": clk, "roofline": roofline,
                "roofline_factor": roofline_factor,
                "schur_apply": schur, "factorization": factorization, "precond": precond,
                "families": {k: {"ms": v["ms"], "launches": v["launches"]} for k, v in fams.items()},
                "fp64_form": fp64_form, "cpu_baseline": cpu}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
