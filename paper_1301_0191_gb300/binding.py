"""Thin ctypes binding of libamb.so (include/amb.h): argument marshalling only.

Every computation happens in the CUDA library; this module converts numpy
arrays / torch tensors into pointers and C structs and back.  Importing it
without the built library raises, so a missing extension fails loudly.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from .build import LIB

OK, EINVAL, ENOMEM, ENOTSPD, EASSUMPTION, ENOCONV, ETIMEOUT, ECUDA = range(8)
FP64, FP32 = 0, 1
CORNERS, CORNERS_EDGES, CORNERS_EDGES_FACES = 1, 2, 3
QOI_COMPLIANCE, QOI_GENERAL = 0, 1
MAX_EIG, MAX_LEVELS, FAM_N = 16, 8, 9
X_SUB_DOFS, X_SUB_SIZES, X_SCHUR, X_COARSE_EL, X_CONSTR, X_CORNERS, X_PAIR_ROWS = range(1, 8)
FAMILIES = ("factor", "trtri", "schur", "lobpcg", "precond", "operator", "coarse", "tc_trailing", "lobpcg_products")


class Mesh(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("h", C.c_double),
                ("dofs_per_node", C.c_int32), ("dirichlet_node_mask", C.c_void_p)]


class Coeffs(C.Structure):
    _fields_ = [("coeff", C.c_void_p), ("poisson_ratio", C.c_double)]


class Partition(C.Structure):
    _fields_ = [("elem_to_sub", C.c_void_p), ("n_sub1", C.c_int32), ("sub_to_parent", C.c_void_p),
                ("n_sub", C.c_void_p)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("initial_constraints", C.c_int32), ("adaptive", C.c_int32),
                ("max_adaptive_per_face", C.c_int32), ("lobpcg_maxit", C.c_int32), ("lobpcg_tol", C.c_double),
                ("pcg_rtol", C.c_double), ("pcg_maxit", C.c_int32), ("seed", C.c_uint64),
                ("cuda_stream", C.c_void_p), ("timing_events", C.c_int32)]


class SolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("rel_residual", C.c_double), ("true_rel_residual", C.c_double),
                ("cond_estimate", C.c_double), ("ms", C.c_double)]


class PairReport(C.Structure):
    _fields_ = [("level", C.c_int32), ("s", C.c_int32), ("t", C.c_int32), ("n_computed", C.c_int32),
                ("n_selected", C.c_int32), ("n_rows", C.c_int32), ("converged", C.c_int32),
                ("iterations", C.c_int32), ("lambda_", C.c_double * MAX_EIG), ("residual", C.c_double)]


class Report(C.Structure):
    _fields_ = [("n_levels", C.c_int32), ("n_pairs", C.c_int32), ("omega_level", C.c_double * MAX_LEVELS),
                ("omega", C.c_double), ("n_adaptive", C.c_int32 * MAX_LEVELS),
                ("n_coarse", C.c_int32 * MAX_LEVELS), ("pcg_iterations", C.c_int32),
                ("cond_estimate", C.c_double), ("pairs", PairReport * 1)]


class LevelSizes(C.Structure):
    _fields_ = [("n_subs", C.c_int32), ("n_pairs", C.c_int32), ("n_corner_nodes", C.c_int32),
                ("n_edges", C.c_int32), ("n_faces", C.c_int32), ("n_dofs", C.c_int64), ("n_coarse", C.c_int64),
                ("sum_ni", C.c_int64), ("sum_ngamma", C.c_int64), ("max_ni", C.c_int64),
                ("max_ngamma", C.c_int64), ("max_ndelta", C.c_int64), ("factor_flops", C.c_double),
                ("schur_words", C.c_double)]


class KernelStats(C.Structure):
    _fields_ = [("ms", C.c_double * FAM_N), ("launches", C.c_int64 * FAM_N), ("flops", C.c_double * FAM_N),
                ("bytes", C.c_double * FAM_N), ("phase_ms", C.c_double * 8), ("kernels_launched", C.c_int64),
                ("tuned_shapes", C.c_int64), ("tuning_runs", C.c_int64), ("graph_replays", C.c_int64)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"libamb.so is not built ({LIB}); run __graft_entry__.build()")
        L = C.CDLL(LIB)
        vp, i32, d, sz = C.c_void_p, C.c_int32, C.c_double, C.POINTER(C.c_size_t)
        L.amb_default_options.argtypes = [C.POINTER(Options)]
        L.amb_setup.argtypes = [C.POINTER(vp), C.POINTER(Mesh), C.POINTER(Coeffs), C.POINTER(Partition), i32, d,
                                C.POINTER(Options)]
        L.amb_solve.argtypes = [vp, vp, vp, C.POINTER(SolveInfo)]
        L.amb_load_vector.argtypes = [vp, vp, vp]
        L.amb_eigen_report.argtypes = [vp, vp, sz]
        L.amb_grad.argtypes = [vp, i32, vp, vp]
        L.amb_schur_apply.argtypes = [vp, i32, i32, vp, vp]
        L.amb_schur_apply_noalloc.argtypes = [vp, i32, i32, vp, vp]
        L.amb_schur_apply_noalloc.restype = C.c_int
        L.amb_level_info.argtypes = [vp, i32, C.POINTER(LevelSizes)]
        L.amb_plan.argtypes = [C.POINTER(Mesh), C.POINTER(Partition), i32, i32, i32, C.POINTER(LevelSizes), vp]
        L.amb_export.argtypes = [vp, i32, i32, i32, vp, sz]
        L.amb_stats.argtypes = [vp, C.POINTER(KernelStats)]
        L.amb_last_error.argtypes = [vp]
        L.amb_last_error.restype = C.c_char_p
        L.amb_destroy.argtypes = [vp]
        for f in ("amb_setup", "amb_solve", "amb_load_vector", "amb_eigen_report", "amb_grad", "amb_schur_apply",
                  "amb_level_info", "amb_plan", "amb_export", "amb_stats"):
            getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


class AmbError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"status {status}: {msg}")
        self.status = status


def _ptr(a) -> int:
    """Address of a C-contiguous numpy array or torch tensor."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous()
        return a.data_ptr()
    assert isinstance(a, np.ndarray) and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def default_options(**kw) -> Options:
    o = Options()
    lib().amb_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def plan(nx, ny, nz, dofs_per_node, dirichlet_node_mask, elem_to_sub, n_sub1, levels=2, sub_to_parent=(),
         n_sub=(), level=1, initial=CORNERS_EDGES):
    """Host-only plan of one level with the initial constraints (amb_plan):
    the level's sizes and, per substructure, (n_I, n_Gamma, corner dofs,
    coarse dofs).  No GPU."""
    mask = np.ascontiguousarray(dirichlet_node_mask, dtype=np.uint8)
    e2s = np.ascontiguousarray(elem_to_sub, dtype=np.int32)
    parents = [np.ascontiguousarray(p, dtype=np.int32) for p in sub_to_parent]
    arr = (C.c_void_p * max(1, len(parents)))(*[_ptr(p) for p in parents])
    ns = np.ascontiguousarray(list(n_sub) or [0], dtype=np.int32)
    mesh = Mesh(nx, ny, nz, 1.0 / nx, dofs_per_node, _ptr(mask))
    part = Partition(_ptr(e2s), n_sub1, C.cast(arr, C.c_void_p) if parents else None, _ptr(ns) if parents else None)
    n_level = ([n_sub1] + [int(v) for v in n_sub])[level - 1] if 1 <= level <= len(parents) + 1 else 1
    info = LevelSizes()
    subs = np.zeros((n_level, 4), dtype=np.int32)
    st = lib().amb_plan(C.byref(mesh), C.byref(part), levels, initial, level, C.byref(info), _ptr(subs))
    if st != OK:
        raise AmbError(st, "amb_plan rejected the input")
    return info, subs


class Context:
    """One library context: set-up on construction, then solve/report/grad."""

    def __init__(self, nx, ny, nz, h, dofs_per_node, dirichlet_node_mask, coeff, poisson_ratio, elem_to_sub,
                 n_sub1, levels, tau, sub_to_parent=(), n_sub=(), options: Optional[Options] = None, **opts):
        self._keep = []
        mask = np.ascontiguousarray(dirichlet_node_mask, dtype=np.uint8)
        e2s = np.ascontiguousarray(elem_to_sub, dtype=np.int32)
        if not hasattr(coeff, "data_ptr"):
            coeff = np.ascontiguousarray(coeff, dtype=np.float64)
        self._keep += [mask, e2s, coeff]
        mesh = Mesh(nx, ny, nz, h, dofs_per_node, _ptr(mask))
        co = Coeffs(_ptr(coeff), poisson_ratio)
        parents = [np.ascontiguousarray(p, dtype=np.int32) for p in sub_to_parent]
        self._keep += parents
        arr = (C.c_void_p * max(1, len(parents)))(*[_ptr(p) for p in parents])
        ns = np.ascontiguousarray(list(n_sub) or [0], dtype=np.int32)
        self._keep += [arr, ns]
        part = Partition(_ptr(e2s), n_sub1, C.cast(arr, C.c_void_p) if parents else None,
                         _ptr(ns) if parents else None)
        o = options if options is not None else default_options(**opts)
        self.options = o
        self.dofs_per_node = dofs_per_node
        self.n_nodes = (nx + 1) * (ny + 1) * (nz + 1)
        self.n_el = nx * ny * nz
        self.h = C.c_void_p()
        st = lib().amb_setup(C.byref(self.h), C.byref(mesh), C.byref(co), C.byref(part), levels, tau, C.byref(o))
        if st != OK:
            msg = self.last_error()
            self.close()
            raise AmbError(st, msg)

    @classmethod
    def from_problem(cls, prob, coeff=None, levels=None, tau=None, **opts):
        """Convenience constructor from an amb_inputs.Problem."""
        c = prob.coeff if coeff is None else coeff
        return cls(prob.nx, prob.ny, prob.nz, prob.h, prob.dofs_per_node, prob.dirichlet_node_mask, c,
                   prob.poisson_ratio, prob.elem_to_sub, prob.n_subs(1), prob.levels if levels is None else levels,
                   prob.tau if tau is None else tau, prob.sub_to_parent,
                   [prob.n_subs(i + 2) for i in range(len(prob.sub_to_parent))], **opts)

    def last_error(self) -> str:
        m = lib().amb_last_error(self.h)
        return m.decode() if m else ""

    def _check(self, st):
        if st != OK:
            raise AmbError(st, self.last_error())

    def close(self):
        if self.h:
            lib().amb_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ calls
    def load_vector(self, body, out=None):
        body = body if hasattr(body, "data_ptr") else np.ascontiguousarray(body, dtype=np.float64)
        out = np.zeros(self.n_nodes * self.dofs_per_node) if out is None else out
        self._check(lib().amb_load_vector(self.h, _ptr(body), _ptr(out)))
        return out

    def solve(self, rhs, out=None, allow_noconv=False):
        rhs = rhs if hasattr(rhs, "data_ptr") else np.ascontiguousarray(rhs, dtype=np.float64)
        out = np.zeros(self.n_nodes * self.dofs_per_node) if out is None else out
        info = SolveInfo()
        st = lib().amb_solve(self.h, _ptr(rhs), _ptr(out), C.byref(info))
        if not (st == OK or (allow_noconv and st == ENOCONV)):
            self._check(st)
        return out, info

    def grad(self, qoi=QOI_COMPLIANCE, dq_du=None, out=None):
        out = np.zeros(self.n_el) if out is None else out
        if dq_du is not None and not hasattr(dq_du, "data_ptr"):
            dq_du = np.ascontiguousarray(dq_du, dtype=np.float64)
        self._check(lib().amb_grad(self.h, qoi, _ptr(dq_du), _ptr(out)))
        return out

    def schur_apply(self, level, width, x, y):
        self._check(lib().amb_schur_apply(self.h, level, width, _ptr(x), _ptr(y)))

    def schur_apply_noalloc(self, level, width, x, y):
        """amb_schur_apply_noalloc: the same product without device allocation."""
        self._check(lib().amb_schur_apply_noalloc(self.h, level, width, _ptr(x), _ptr(y)))

    def level_info(self, level=1) -> LevelSizes:
        li = LevelSizes()
        self._check(lib().amb_level_info(self.h, level, C.byref(li)))
        return li

    def report(self) -> dict:
        n = C.c_size_t(0)
        self._check(lib().amb_eigen_report(self.h, None, C.byref(n)))
        buf = (C.c_char * n.value)()
        self._check(lib().amb_eigen_report(self.h, buf, C.byref(n)))
        r = Report.from_buffer(buf)
        off = Report.pairs.offset
        pairs = []
        for k in range(r.n_pairs):
            p = PairReport.from_buffer(buf, off + k * C.sizeof(PairReport))
            pairs.append(dict(level=p.level, s=p.s, t=p.t, n_computed=p.n_computed, n_selected=p.n_selected,
                              n_rows=p.n_rows, converged=p.converged, iterations=p.iterations,
                              lam=np.array(p.lambda_[:p.n_computed]), residual=p.residual))
        nl = r.n_levels
        return dict(n_levels=nl, omega_level=list(r.omega_level[:nl]), omega=r.omega,
                    n_adaptive=list(r.n_adaptive[:nl]), n_coarse=list(r.n_coarse[:nl]),
                    pcg_iterations=r.pcg_iterations, cond_estimate=r.cond_estimate, pairs=pairs)

    def export(self, what, level, index, dtype):
        n = C.c_size_t(0)
        self._check(lib().amb_export(self.h, what, level, index, None, C.byref(n)))
        buf = np.empty(n.value, dtype=np.uint8)
        self._check(lib().amb_export(self.h, what, level, index, _ptr(buf), C.byref(n)))
        return buf.view(dtype)

    def stats(self) -> dict:
        s = KernelStats()
        self._check(lib().amb_stats(self.h, C.byref(s)))
        fam = {name: dict(ms=s.ms[i], launches=s.launches[i], flops=s.flops[i], bytes=s.bytes[i])
               for i, name in enumerate(FAMILIES)}
        phases = dict(zip(("assembly", "factor", "eigen", "constraints", "coarse", "solve", "grad", "setup_total"),
                          list(s.phase_ms)))
        return dict(families=fam, phase_ms=phases, kernels_launched=s.kernels_launched,
                    tuned_shapes=s.tuned_shapes, tuning_runs=s.tuning_runs, graph_replays=s.graph_replays)
