"""The C-ABI library builds, loads and exports every entry point declared in
include/amb.h (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "amb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|void|const char\*)\s+(amb_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("amb_setup", "amb_solve", "amb_eigen_report", "amb_grad", "amb_last_error", "amb_destroy"):
        assert n in names


def test_library_builds_and_exports_every_symbol():
    from paper_1301_0191_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for n in _declared():
        assert hasattr(lib, n), n


def test_binding_structs_match_header_sizes():
    from paper_1301_0191_gb300 import binding as B
    # layouts mirror the C structs: check field order against the header text
    src = open(os.path.join(ROOT, "include", "amb.h")).read()
    assert src.index("int32_t iterations;") < src.index("double rel_residual;")
    assert ctypes.sizeof(B.PairReport) == 8 * 4 + 16 * 8 + 8
    o = B.default_options()
    assert o.precision == B.FP64 and o.max_adaptive_per_face == 10 and o.pcg_rtol == 1e-8


def test_kernel_stats_fields_follow_the_header():
    from paper_1301_0191_gb300 import binding as B
    src = open(os.path.join(ROOT, "include", "amb.h")).read()
    body = src[src.index("typedef struct {\n  double ms[AMB_FAM_N];"):src.index("} amb_kernel_stats;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = re.findall(r"(?:double|int64_t)\s+([a-z_]+)", body)
    assert names == [f[0] for f in B.KernelStats._fields_]
    assert ctypes.sizeof(B.KernelStats) == 8 * (4 * B.FAM_N + 8 + 4)
