"""The C-ABI library builds, loads and exports every symbol include/sdmhd.h
declares; argument and topology checks that run before any device work.
No test here needs a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2502_17805_gb300 import build as libbuild
from paper_2502_17805_gb300 import inputs, sdmhd

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "sdmhd.h")


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return sdmhd.lib()


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:sd_status|const char\*)\s+(sd_\w+)\s*\(", txt, re.M)))


def test_header_declares_the_abi():
    names = _declared()
    for n in ("sd_mesh_create", "sd_state_init", "sd_residual", "sd_rk_stage", "sd_diagnostics"):
        assert n in names
    assert sorted(sdmhd.EXPORTS) == names


def test_library_exports_every_declared_symbol(lib):
    raw = C.CDLL(sdmhd.LIB_PATH)
    for n in _declared():
        assert hasattr(raw, n), n


def _desc(N, v, h, per=None, geom=0):
    v = np.ascontiguousarray(v, dtype=np.float64)
    h = np.ascontiguousarray(h, dtype=np.int64)
    d = sdmhd.MeshDesc()
    d.order, d.geom = N, geom
    d.n_vertices, d.vertices = v.shape[0], v.ctypes.data_as(C.POINTER(C.c_double))
    d.n_elements, d.hex = h.shape[0], h.ctypes.data_as(C.POINTER(C.c_int64))
    keep = [v, h]
    if per is not None:
        per = np.ascontiguousarray(per, dtype=np.float64)
        d.periodic_lengths = per.ctypes.data_as(C.POINTER(C.c_double))
        keep.append(per)
    d.bc_inner, d.bc_outer = 1, 2
    return d, keep


def test_mesh_create_rejects_bad_arguments(lib):
    out = C.c_void_p()
    assert lib.sd_mesh_create(None, None, C.byref(out)) == 1
    v, h, per = inputs.box_mesh(3)
    d, keep = _desc(9, v, h, per)
    assert lib.sd_mesh_create(C.byref(d), None, C.byref(out)) == 2  # unsupported order
    assert "order" in lib.sd_last_error().decode()
    h2 = h.copy()
    h2[0, 0] = 10 ** 6
    d, keep = _desc(4, v, h2, per)
    assert lib.sd_mesh_create(C.byref(d), None, C.byref(out)) == 1
    assert not out.value


def test_mesh_create_rejects_an_empty_mesh(lib):
    out = C.c_void_p()
    v, h, per = inputs.box_mesh(3)
    d, keep = _desc(4, v, h[:0], None)
    assert lib.sd_mesh_create(C.byref(d), None, C.byref(out)) == 1
    assert "at least one element" in lib.sd_last_error().decode()
    assert not out.value


def test_mesh_create_detects_non_conforming_topology(lib):
    out = C.c_void_p()
    v, h, per = inputs.box_mesh(3)
    # a duplicated element makes six faces shared by more than two elements
    d, keep = _desc(4, v, np.concatenate([h, h[:1]]), per)
    assert lib.sd_mesh_create(C.byref(d), None, C.byref(out)) == 3
    # an unmatched face of a periodic mesh with a periodic boundary tag
    d, keep = _desc(4, v, h[:-1], per)
    d.bc_inner = 0
    assert lib.sd_mesh_create(C.byref(d), None, C.byref(out)) == 3
    # repeated corners
    h3 = h.copy()
    h3[0, 1] = h3[0, 0]
    d, keep = _desc(4, v, h3, per)
    assert lib.sd_mesh_create(C.byref(d), None, C.byref(out)) == 3


def test_calls_reject_null_mesh(lib):
    ph = sdmhd.Phys().c()
    assert lib.sd_residual(None, C.byref(ph), 0, None, None, None, None) == 1
    assert lib.sd_rk_stage(None, C.byref(ph), 0, 0, 0.1, None, None, None, None, None) == 1
    assert lib.sd_diagnostics(None, C.byref(ph), None, None, None) == 1
    assert lib.sd_step(None, C.byref(ph), 0, 0.2, None, None, None, None, None) == 1
    assert lib.sd_advance(None, C.byref(ph), 0, 0.2, 3, None, None, None, None, None) == 1
    assert lib.sd_mesh_destroy(None) == 0
