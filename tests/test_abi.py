"""The C-ABI library builds, loads and exports every entry point declared in
include/amb.h (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import numpy as np
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


def _mesh_2x2(nx=4):
    mask = np.zeros((3, 3, nx + 1), dtype=np.uint8)
    mask[:, :, 0] = 1                      # x = 0 fixed
    return dict(nx=nx, ny=2, nz=2, h=1.0 / nx, dofs_per_node=1, dirichlet_node_mask=mask.ravel(),
                coeff=np.ones(nx * 4), poisson_ratio=0.3, tau=10.0)


@pytest.mark.parametrize("case", ["out_of_range", "not_a_box", "empty", "parent_not_a_box", "parent_out_of_range"])
def test_setup_rejects_invalid_partitions(case):
    """The decomposition is checked on the host before any device work:
    AMB_EINVAL with the violation named (no GPU needed)."""
    from paper_1301_0191_gb300 import binding as B
    m = _mesh_2x2()
    i = np.tile(np.arange(4), 4)                         # element (i, j, k) -> e = i + 4 (j + 2 k)
    e2s, n1, levels, parents, nsub, words = (i >= 2).astype(np.int32), 2, 2, (), (), ""
    if case == "out_of_range":
        e2s[5], words = 2, "out of range"
    elif case == "not_a_box":
        e2s[2], words = 0, "not a box"                   # element (2, 0, 0) joins the x < 2 box
    elif case == "empty":
        n1, words = 3, "substructure 2 is empty"
    elif case == "parent_not_a_box":
        e2s, n1, levels, parents, nsub = i.astype(np.int32), 4, 3, [np.array([0, 1, 0, 1])], [2]
        words = "level-2 substructure 0 is not a box"
    else:
        e2s, n1, levels, parents, nsub = i.astype(np.int32), 4, 3, [np.array([0, 0, 1, 2])], [2]
        words = "sub_to_parent out of range"
    with pytest.raises(B.AmbError) as ei:
        B.Context(m["nx"], m["ny"], m["nz"], m["h"], 1, m["dirichlet_node_mask"], m["coeff"], 0.3, e2s, n1,
                  levels, m["tau"], parents, nsub)
    assert ei.value.status == B.EINVAL
    assert words in str(ei.value)


def test_header_is_plain_c(tmp_path):
    """include/amb.h is a C header: it compiles as C99 with -pedantic."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "check.c"
    src.write_text('#include "amb.h"\nint main(void) { return 0; }\n')
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                        "-I", os.path.join(ROOT, "include"), str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


C_PROGRAM = r"""
#include <stdio.h>
#include <stdlib.h>
#include "amb.h"

/* 8 x 4 x 4 Poisson mesh, x = 0 clamped, 2 x 1 x 1 boxes: plan level 1 from C */
int main(void) {
  enum { NX = 8, NY = 4, NZ = 4 };
  static uint8_t mask[(NX + 1) * (NY + 1) * (NZ + 1)];
  static int32_t e2s[NX * NY * NZ];
  for (int k = 0; k <= NZ; ++k)
    for (int j = 0; j <= NY; ++j)
      for (int i = 0; i <= NX; ++i) mask[i + (NX + 1) * (j + (NY + 1) * k)] = (uint8_t)(i == 0);
  for (int k = 0; k < NZ; ++k)
    for (int j = 0; j < NY; ++j)
      for (int i = 0; i < NX; ++i) e2s[i + NX * (j + NY * k)] = i >= NX / 2;
  amb_mesh mesh = {NX, NY, NZ, 1.0 / NX, 1, mask};
  amb_partition part = {e2s, 2, NULL, NULL};
  amb_options opt;
  amb_default_options(&opt);
  amb_level_sizes info;
  int32_t sizes[8];
  int st = amb_plan(&mesh, &part, 2, opt.initial_constraints, 1, &info, sizes);
  printf("%d %d %d %lld %lld %d %d %d %d\n", st, info.n_subs, info.n_pairs, (long long)info.n_dofs,
         (long long)info.n_coarse, sizes[0], sizes[1], sizes[4], sizes[5]);
  return st;
}
"""


def test_plan_from_a_c_program(tmp_path):
    """The boundary used from plain C: a C99 program links libamb.so and plans
    a two-substructure mesh (host only, no GPU)."""
    import shutil
    import subprocess
    from paper_1301_0191_gb300 import build
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib = build.build()
    src = tmp_path / "plan.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "plan"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                        "-L", os.path.dirname(lib), "-lamb", "-Wl,-rpath," + os.path.dirname(lib), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    st, nsub, npair, ndof, ncoarse, ni0, ng0, ni1, ng1 = (int(v) for v in out.stdout.split())
    # 9 x 5 x 5 nodes, the x = 0 plane clamped; the interface is the x = 4 plane
    # (25 nodes), whose box vertices are its 4 corners; no edges; every other
    # free node is interior to one box
    assert (st, nsub, npair, ndof) == (0, 2, 1, 8 * 25)
    assert ncoarse == 4 and ng0 == ng1 == 25
    assert ni0 == 3 * 25 and ni1 == 4 * 25
