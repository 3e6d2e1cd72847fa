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
    return sorted(set(re.findall(r"\b(ph_[a-z0-9_]+)\s*\(", src)))


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


def test_size_limits_and_argument_checks_without_gpu(lib):
    """Size limits (int32 ids and CSR positions) and argument checks are
    decided on the host, before any allocation or CUDA call: oversize meshes
    give PH_ERR_OVERFLOW, bad sizes and pointers PH_ERR_ARG, empty inputs
    PH_OK.  The pointers below are never dereferenced."""
    P, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    ARG, OVERFLOW = 1, 4
    fake, odd = P(256), P(260)   # 16-byte aligned / misaligned addresses, never read
    out = ctypes.c_void_p()
    create = lib.ph_mesh_create
    create.argtypes = [P, I64, P, I64, P, I64, P, ctypes.POINTER(P)]
    create.restype = ctypes.c_int
    assert create(fake, 4, fake, 1, None, 0, None, None) == ARG            # no output handle
    assert create(fake, 4, odd, 1, None, 0, None, ctypes.byref(out)) == ARG  # tet read as int4
    assert create(fake, 4, None, 1, None, 0, None, ctypes.byref(out)) == ARG
    assert create(fake, 4, fake, 1, None, 3, None, ctypes.byref(out)) == ARG  # nN > 0 without triples
    # nnz <= 4 nE + nN + 12 nE must stay below 2^31: nE = 2^27 is one too many
    assert create(fake, 4, fake, 1 << 27, None, 0, None, ctypes.byref(out)) == OVERFLOW
    assert create(fake, (1 << 31) - 1, fake, 1, None, 0, None, ctypes.byref(out)) == OVERFLOW
    assert out.value is None
    refine = lib.ph_refine
    refine.argtypes = [P, I64, P, I64, P, I64, P, ctypes.POINTER(P)]
    refine.restype = ctypes.c_int
    assert refine(fake, 4, odd, 1, None, 0, None, ctypes.byref(out)) == ARG
    assert refine(fake, 4, fake, 1 << 28, None, 0, None, ctypes.byref(out)) == OVERFLOW  # 12 nE children
    pcg = lib.ph_solve_pcg
    pcg.argtypes = [I64, P, P, P, P, P, D, I32, ctypes.POINTER(I32), ctypes.POINTER(D), P]
    pcg.restype = ctypes.c_int
    it, rr = I32(7), D(7.0)
    assert pcg(-1, fake, fake, fake, fake, fake, 1e-10, 100, ctypes.byref(it), ctypes.byref(rr), None) == ARG
    assert pcg(10, fake, fake, fake, fake, fake, float("nan"), 100, None, None, None) == ARG
    assert pcg(10, fake, fake, fake, fake, fake, 1e-10, -1, None, None, None) == ARG
    assert pcg(10, None, fake, fake, fake, fake, 1e-10, 100, None, None, None) == ARG
    assert pcg(0, None, None, None, None, None, 1e-10, 100, ctypes.byref(it), ctypes.byref(rr), None) == 0
    assert it.value == 0 and rr.value == 0.0
    host = lib.ph_assemble_host
    host.argtypes = [P, I64, P, I64, P, I64, I64, I64, I64, P, D, P, P, P, P, P, P, P, P, P, P]
    host.restype = ctypes.c_int
    assert host(fake, 4, fake, 1, None, 0, 4, 4, -1, fake, 1.0, fake, None, None, None,
                fake, fake, fake, fake, None, None) == ARG
    assert host(fake, 4, fake, 1, None, 0, 4, 4, 16, fake, 1.0, fake, None, None, None,
                None, fake, fake, fake, None, None) == ARG                    # rowptr missing
    assert host(fake, 4, fake, 1, None, 0, 4, 4, 16, fake, 1.0, fake, None, None, None,
                fake, fake, fake, fake, fake, None) == ARG                    # U without Lambda
    for name in ("ph_rcp", "ph_half_sqrt"):
        fn = getattr(lib, name)
        fn.argtypes = [P, I64, P, P]
        fn.restype = ctypes.c_int
        assert fn(fake, -1, fake, None) == ARG
        assert fn(None, 5, fake, None) == ARG
        assert fn(None, 0, None, None) == 0
