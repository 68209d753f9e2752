"""CPU checks of the C ABI: the library builds, loads and exports every
function include/pcarecon.h declares; the ctypes structs match the C layout."""

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pcarecon.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pr_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1004_0014_b300 import build, capi

    build.build()
    return capi.load_library()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("pr_create", "pr_destroy", "pr_load_model", "pr_reconstruct", "pr_forward", "pr_vjp",
              "pr_project", "pr_backproject", "pr_tumor"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1004_0014_b300 import build, capi

    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (pr_[a-z_]+)$", out, flags=re.M))
    for n in _declared():
        assert n in exported, n
        assert hasattr(lib, n)
    assert sorted(capi.EXPORTED) == _declared()


def test_struct_layout_matches_c():
    from paper_1004_0014_b300 import capi

    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "pcarecon.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(pr_volume_desc), sizeof(pr_geometry),
         sizeof(pr_solve_opts), sizeof(pr_result), offsetof(pr_solve_opts, loop_mode),
         offsetof(pr_solve_opts, tumor_max_iter), offsetof(pr_result, iters),
         offsetof(pr_result, tumor_steps));
  return 0;
}
'''
    import tempfile

    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "l.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "l")
        subprocess.check_call(["gcc", "-I" + os.path.join(ROOT, "include"), c, "-o", exe])
        got = [int(x) for x in subprocess.check_output([exe]).split()]
    want = [ctypes.sizeof(capi.VolumeDesc), ctypes.sizeof(capi.Geometry), ctypes.sizeof(capi.SolveOpts),
            ctypes.sizeof(capi.Result), capi.SolveOpts.loop_mode.offset, capi.SolveOpts.tumor_max_iter.offset,
            capi.Result.iters.offset, capi.Result.tumor_steps.offset]
    assert got == want


def test_defaults_and_version(lib):
    from paper_1004_0014_b300 import capi

    o = capi.pr_default_opts()
    assert (o.max_iters, o.c1, o.beta, o.max_backtracks, o.step0_mm) == (10, 1e-4, 0.5, 8, 1.0)
    assert (o.step_growth, o.step_growth_bt, o.warm_step, o.step_model, o.predict) == (2.0, 1.0, 1, 1, 0)
    assert "sm_103a" in capi.pr_version()


def test_oracle_is_not_imported_by_the_package():
    pkg = os.path.join(ROOT, "paper_1004_0014_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"#.*|//.*", "", text).lower().replace("oracle.", ""), f
