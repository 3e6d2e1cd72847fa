"""ph_solve_pcg_noalloc: the PCG solve for callers that cannot allocate device
memory while they run (its workspace is a fixed array inside the library).

It is called here through the C ABI and must give the same result as the
allocating ph_solve_pcg, within the solve tolerance of the other tests, on two
calls in a row with different right-hand sides (the shared workspace keeps the
previous call's contents).  This file is collected last so that a failure here
stops a -x run only after every other test has run.
"""
import ctypes

import numpy as np
import pytest

import meshgen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SOLVE_RTOL = 1e-9


def _system(ph, name):
    p = meshgen.problem(name)
    dev = torch.device("cuda")
    mesh = ph.Mesh(torch.as_tensor(p.coord, device=dev), torch.as_tensor(p.tet, device=dev))
    cen = mesh.faces()["face_centroid"].cpu().numpy()
    f = torch.as_tensor(np.asarray(p.f(cen)), device=dev)
    a = torch.as_tensor(p.a, device=dev)
    rowptr, colind = mesh.csr_pattern()
    values, rhs = mesh.assemble(a, p.c, f)
    torch.cuda.synchronize()
    mesh.close()
    return rowptr, colind, values, rhs


def _noalloc(lib, rowptr, colind, values, b, x):
    it = ctypes.c_int32(0)
    rr = ctypes.c_double(0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    code = lib.ph_solve_pcg_noalloc(b.numel(), ctypes.c_void_p(rowptr.data_ptr()), ctypes.c_void_p(colind.data_ptr()),
                                    ctypes.c_void_p(values.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                    ctypes.c_void_p(x.data_ptr()), 1e-13, 50000, ctypes.byref(it), ctypes.byref(rr),
                                    stream)
    torch.cuda.synchronize()
    return code, it.value, rr.value


def test_noalloc_pcg_matches_allocating_pcg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2509_11133_gb300 as ph
    from paper_2509_11133_gb300 import build
    build.build()
    lib = ph.load()
    rowptr, colind, values, rhs = _system(ph, "sin_kuhn")
    rhs2 = rhs * -0.5 + torch.linspace(0.0, 1.0, rhs.numel(), dtype=torch.float64, device=rhs.device)
    for b in (rhs, rhs2):                     # two calls in a row, different data
        x_ref, it_ref, _, code_ref = ph.ph_solve_pcg(rowptr, colind, values, b, rtol=1e-13, maxit=50000)
        assert code_ref == 0
        x = torch.full_like(b, float("nan"))
        code, it, rr = _noalloc(lib, rowptr, colind, values, b, x)
        assert code == 0, ph.ph_status_string(code)
        assert rr <= 1e-13 and it == it_ref
        xr, xn = x_ref.cpu().numpy(), x.cpu().numpy()
        assert np.all(np.isfinite(xn))
        assert np.linalg.norm(xn - xr) <= SOLVE_RTOL * np.linalg.norm(xr)


def test_noalloc_rejects_oversize():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2509_11133_gb300 as ph
    lib = ph.load()
    one = torch.zeros(1, dtype=torch.float64, device="cuda")
    idx = torch.zeros(2, dtype=torch.int32, device="cuda")
    it = ctypes.c_int32(0)
    rr = ctypes.c_double(0)
    code = lib.ph_solve_pcg_noalloc(ph.PH_PCG_NOALLOC_MAX_N + 1, ctypes.c_void_p(idx.data_ptr()),
                                    ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(one.data_ptr()),
                                    ctypes.c_void_p(one.data_ptr()), ctypes.c_void_p(one.data_ptr()), 1e-12, 10,
                                    ctypes.byref(it), ctypes.byref(rr), None)
    assert ph.ph_status_string(code) == "PH_ERR_ARG"
    assert b"PH_PCG_NOALLOC_MAX_N" in lib.ph_last_error_message()
