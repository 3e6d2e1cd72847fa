"""The C-ABI library builds, loads without a GPU and exports every symbol
declared in include/ph.h (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "ph.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ph_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2509_11133_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_entry_points():
    syms = declared_symbols()
    for s in ("ph_mesh_create", "ph_assemble", "ph_recover", "ph_solve_pcg", "ph_csr_pattern", "ph_mesh_faces"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_lists_every_declared_symbol():
    import paper_2509_11133_gb300 as ph
    assert sorted(ph.EXPORTS) == declared_symbols()


def test_host_side_queries_without_gpu(lib):
    lib.ph_status_string.restype = ctypes.c_char_p
    assert lib.ph_status_string(0) == b"PH_OK"
    assert lib.ph_status_string(3) == b"PH_ERR_NONMANIFOLD"
    lib.ph_launch_count.restype = ctypes.c_int64
    assert lib.ph_launch_count() == 0
    # argument errors are returned before any CUDA call
    lib.ph_mesh_create.restype = ctypes.c_int
    out = ctypes.c_void_p()
    assert lib.ph_mesh_create(None, 0, None, -1, None, 0, None, ctypes.byref(out)) == 1
    lib.ph_assemble.restype = ctypes.c_int
    assert lib.ph_assemble(None, None, ctypes.c_double(1.0), None, None, None, None, None, None, None) == 1
