"""The C ABI library builds, loads and exports every symbol include/mpm.h declares
(no compute call: this runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mpm.h")).read()
    return sorted(set(re.findall(r"^\s*(?:mpm_status|const char \*)\s*\*?\s*(mpm_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2505_03067_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("mpm_box_extract", "mpm_assemble_coeffs", "mpm_solve_step", "mpm_solve_batch"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for n in _declared():
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (mpm_\w+)", out))
    assert set(_declared()) <= exported


def test_binding_covers_every_symbol():
    from paper_2505_03067_gb300 import mpm
    assert sorted(mpm.SYMBOLS) == _declared()


def test_binding_structs_match_header_sizes(libpath):
    """ctypes layouts agree with the C compiler's (offsets checked via a tiny C probe)."""
    from paper_2505_03067_gb300 import mpm
    import tempfile
    prog = r'''
#include <stdio.h>
#include <stddef.h>
#include "mpm.h"
int main(void){
 printf("%zu %zu %zu %zu %zu %zu\n", sizeof(mpm_lattice), sizeof(mpm_params), sizeof(mpm_opts),
        sizeof(mpm_report), sizeof(mpm_subgrid_desc), sizeof(mpm_box));
 printf("%zu %zu %zu %zu %zu\n", offsetof(mpm_params,k_cell), offsetof(mpm_opts,inner_rtol),
        offsetof(mpm_report,box_voxels), offsetof(mpm_subgrid_desc,stored_voxels), offsetof(mpm_report,fallback));
 return 0; }'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "p.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "p")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        out = subprocess.run([exe], capture_output=True, text=True).stdout.split()
    sizes = [int(v) for v in out]
    C = ctypes
    assert sizes[:6] == [C.sizeof(mpm.mpm_lattice), C.sizeof(mpm.mpm_params), C.sizeof(mpm.mpm_opts),
                         C.sizeof(mpm.mpm_report), C.sizeof(mpm.mpm_subgrid_desc), C.sizeof(mpm.mpm_box)]
    assert sizes[6:] == [mpm.mpm_params.k_cell.offset, mpm.mpm_opts.inner_rtol.offset,
                         mpm.mpm_report.box_voxels.offset, mpm.mpm_subgrid_desc.stored_voxels.offset,
                         mpm.mpm_report.fallback.offset]


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2505_03067_gb300")
    for dp, _, fs in os.walk(pkg):
        for f in fs:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dp, f)).read()
                assert not re.search(r"^\s*(import oracle|from oracle)", txt, re.M), f
                assert "oracle.c" not in txt and "liboracle" not in txt, f
