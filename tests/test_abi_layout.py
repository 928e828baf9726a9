"""The binding's ctypes structures against the C header's: the size of every structure of
`include/sdmhd.h` that crosses the boundary, and the offset of every field, as gcc lays them out
(plain C, the same ABI nvcc's host compiler uses)."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

from paper_2502_17805_gb300 import sdmhd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PAIRS = [("sd_mesh_desc", sdmhd.MeshDesc), ("sd_phys", sdmhd.PhysC), ("sd_init", sdmhd.InitC),
         ("sd_diag", sdmhd.DiagC), ("sd_mesh_info", sdmhd.MeshInfoC), ("sd_profile_stats", sdmhd.ProfileC),
         ("sd_step_req", sdmhd.StepReqC)]


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "sdmhd.h"', 'int main(void) {']
    for cname, py in PAIRS:
        lines.append('  printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for fname, _ in py._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, fname, cname, fname))
    lines += ['  return 0;', '}']
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    table = {}
    for line in out.splitlines():
        a, b, n = line.split()
        table[(a, b)] = int(n)
    return table


@pytest.mark.parametrize("cname,py", PAIRS, ids=[p[0] for p in PAIRS])
def test_structure_layout_matches_the_header(c_layout, cname, py):
    assert C.sizeof(py) == c_layout[(cname, "size")], cname
    for fname, _ in py._fields_:
        assert getattr(py, fname).offset == c_layout[(cname, fname)], (cname, fname)
