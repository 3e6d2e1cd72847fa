"""GB300 (sm_103a) library for the data-parallel path of the lowest-order
primal hybrid FEM of arXiv 2509.11133: face-to-tetrahedron connectivity,
per-element local matrices, element-wise Schur condensation onto the face
multipliers, scatter into CSR, a PCG solve and element recovery.

This module is a thin ctypes binding of the C ABI in ``include/ph.h``: it
marshals torch CUDA tensors (device pointers) and the current CUDA stream into
the ``ph_*`` entry points, which do all of the work in CUDA kernels.  There is
no CPU path: if ``libph.so`` has not been built (``build.build()``), importing
the library raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB = None

PH_OK = 0
STATUS_NAMES = {0: "PH_OK", 1: "PH_ERR_ARG", 2: "PH_ERR_DEGENERATE", 3: "PH_ERR_NONMANIFOLD",
                4: "PH_ERR_OVERFLOW", 5: "PH_ERR_NOMEM", 6: "PH_ERR_CUDA", 7: "PH_ERR_NOT_CONVERGED",
                8: "PH_ERR_TIMEOUT"}

# Every symbol declared in include/ph.h.
EXPORTS = ("ph_mesh_create", "ph_mesh_destroy", "ph_mesh_info", "ph_mesh_faces", "ph_csr_pattern", "ph_assemble",
           "ph_recover", "ph_solve_pcg", "ph_mesh_check", "ph_status_string", "ph_last_error_message",
           "ph_launch_count", "ph_solve_pcg_noalloc", "ph_recover_factored", "ph_recover_factored_dw", "ph_spmv",
           "ph_misfit",
           "ph_adjoint_rhs", "ph_adjoint_grad", "ph_batch_create", "ph_batch_destroy", "ph_batch_bind",
           "ph_batch_assemble", "ph_batch_autotune", "ph_batch_set_config", "ph_batch_get_config",
           "ph_batch_graph_launch", "ph_refine", "ph_refined_info", "ph_refined_copy", "ph_refined_destroy", "ph_rcp", "ph_half_sqrt", "ph_timing_enable",
           "ph_kernel_time", "ph_assemble_host", "ph_schwarz_create", "ph_schwarz_destroy",
           "ph_solve_pcg_schwarz", "ph_fp64_peak", "ph_test_fail_alloc", "ph_test_scan_withhold",
           "ph_pool_in_use", "ph_solve_refined", "ph_mesh_create_batch", "ph_host_mesh_query",
           "ph_assemble_dw", "ph_batch_bind_recovery", "ph_mesh_create_dw")


class PHError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        self.code = code
        self.name = STATUS_NAMES.get(code, str(code))
        super().__init__(f"{where}: {self.name}" + (f" ({detail})" if detail else ""))


class ph_info(ctypes.Structure):
    _fields_ = [("nE", ctypes.c_int64), ("nC", ctypes.c_int64), ("nF", ctypes.c_int64),
                ("nF_interior", ctypes.c_int64), ("nF_dirichlet", ctypes.c_int64), ("nF_neumann", ctypes.c_int64),
                ("L", ctypes.c_int64), ("nnz", ctypes.c_int64)]


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libph.so (built in-tree); raise if it is missing."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is not built; run paper_2509_11133_gb300.build.build()")
    L = ctypes.CDLL(path)
    P, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    sig = {
        "ph_mesh_create": [P, I64, P, I64, P, I64, P, ctypes.POINTER(P)],
        "ph_mesh_create_batch": [I32, P, P, P, P, P, P, P, P],
        "ph_mesh_create_dw": [P, I64, P, I64, P, I64, P, ctypes.POINTER(P)],
        "ph_host_mesh_query": [P, I64, P, I64, P, I64, ctypes.POINTER(ph_info), P, I64, P],
        "ph_mesh_destroy": [P, P],
        "ph_mesh_info": [P, ctypes.POINTER(ph_info)],
        "ph_mesh_faces": [P, P, P, P, P, P, P, P, P],
        "ph_csr_pattern": [P, P, P, P],
        "ph_assemble": [P, P, D, P, P, P, P, P, P, P],
        "ph_assemble_dw": [P, P, D, P, P, P, P, P, P, P],
        "ph_recover_factored": [P, P, D, P, P, P, P, P],
        "ph_recover_factored_dw": [P, P, D, P, P, P, P, P],
        "ph_recover": [P, P, D, P, P, P, P, P],
        "ph_solve_pcg": [I64, P, P, P, P, P, D, I32, ctypes.POINTER(I32), ctypes.POINTER(D), P],
        "ph_solve_pcg_noalloc": [I64, P, P, P, P, P, D, I32, ctypes.POINTER(I32), ctypes.POINTER(D), P],
        "ph_mesh_check": [P, P],
        "ph_spmv": [I64, P, P, P, P, P, P],
        "ph_misfit": [P, P, P, P, P],
        "ph_adjoint_rhs": [P, P, D, P, P, P, P],
        "ph_adjoint_grad": [P, P, P, D, P, P, P, P, P],
        "ph_batch_create": [P, I32, P, ctypes.POINTER(P)],
        "ph_batch_destroy": [P, P],
        "ph_batch_bind": [P, P, P, P, P, P, P, P, P, P],
        "ph_batch_assemble": [P, P],
        "ph_batch_autotune": [P, I32, ctypes.POINTER(ctypes.c_float), P],
        "ph_batch_set_config": [P, I32, I32, I32, P],
        "ph_batch_get_config": [P, ctypes.POINTER(I32), ctypes.POINTER(I32), ctypes.POINTER(I32)],
        "ph_batch_graph_launch": [P, P],
        "ph_batch_bind_recovery": [P, P, P, P],
        "ph_refine": [P, I64, P, I64, P, I64, P, ctypes.POINTER(P)],
        "ph_refined_info": [P, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64)],
        "ph_refined_copy": [P, P, P, P, P],
        "ph_refined_destroy": [P, P],
        "ph_rcp": [P, I64, P, P],
        "ph_half_sqrt": [P, I64, P, P],
        "ph_fp64_peak": [I64, ctypes.POINTER(D), ctypes.POINTER(D), P],
        "ph_test_fail_alloc": [I64],
        "ph_test_scan_withhold": [ctypes.c_int],
        "ph_pool_in_use": [ctypes.POINTER(I64)],
        "ph_solve_refined": [P, P, P, P, P, D, D, I32, I32, ctypes.POINTER(I32), ctypes.POINTER(I32),
                             ctypes.POINTER(D), P],
        "ph_timing_enable": [ctypes.c_int],
        "ph_kernel_time": [ctypes.c_char_p, ctypes.c_int, ctypes.POINTER(D), ctypes.POINTER(I64)],
        "ph_assemble_host": [P, I64, P, I64, P, I64, I64, I64, I64, P, D, P, P, P, P, P, P, P, P, P, P],
        "ph_schwarz_create": [P, P, P, ctypes.POINTER(P)],
        "ph_schwarz_destroy": [P, P],
        "ph_solve_pcg_schwarz": [P, P, P, P, P, D, I32, ctypes.POINTER(I32), ctypes.POINTER(D), P],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.ph_status_string.argtypes = [ctypes.c_int]
    L.ph_status_string.restype = ctypes.c_char_p
    L.ph_last_error_message.argtypes = []
    L.ph_last_error_message.restype = ctypes.c_char_p
    L.ph_launch_count.argtypes = []
    L.ph_launch_count.restype = ctypes.c_int64
    _LIB = L
    return L


def _check(code: int, where: str):
    if code != PH_OK:
        detail = ""
        if code in (5, 6):
            detail = load().ph_last_error_message().decode()
        raise PHError(code, where, detail)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _need(t, dtype, n, name):
    if t is None:
        raise ValueError(f"{name} is required")
    if t.dtype != dtype or t.numel() != n:
        raise ValueError(f"{name}: expected {dtype} with {n} elements, got {t.dtype} with {t.numel()}")
    return t


def ph_launch_count() -> int:
    return int(load().ph_launch_count())


def ph_status_string(code: int) -> str:
    return load().ph_status_string(code).decode()


def ph_solve_pcg(rowptr, colind, values, rhs, x=None, rtol=1e-12, maxit=20000, stream=None, check=True):
    """Jacobi-PCG solve of H x = rhs (all CUDA tensors). Returns (x, iters, relres, status)."""
    n = rhs.numel()
    if x is None:
        x = torch.empty(n, dtype=torch.float64, device=rhs.device)
    it = ctypes.c_int32(0)
    rr = ctypes.c_double(0)
    code = load().ph_solve_pcg(n, _ptr(rowptr), _ptr(colind), _ptr(values), _ptr(rhs), _ptr(x), float(rtol),
                               int(maxit), ctypes.byref(it), ctypes.byref(rr), _stream(stream))
    if check:
        _check(code, "ph_solve_pcg")
    return x, it.value, rr.value, code


def ph_solve_pcg_noalloc(rowptr, colind, values, rhs, x=None, rtol=1e-12, maxit=20000, stream=None, check=True):
    """ph_solve_pcg without device allocation inside the library (workspace in
    a fixed device array; n <= PH_PCG_NOALLOC_MAX_N).  ``x`` is caller-owned."""
    n = rhs.numel()
    if x is None:
        x = torch.empty(n, dtype=torch.float64, device=rhs.device)
    it = ctypes.c_int32(0)
    rr = ctypes.c_double(0)
    code = load().ph_solve_pcg_noalloc(n, _ptr(rowptr), _ptr(colind), _ptr(values), _ptr(rhs), _ptr(x),
                                       float(rtol), int(maxit), ctypes.byref(it), ctypes.byref(rr), _stream(stream))
    if check:
        _check(code, "ph_solve_pcg_noalloc")
    return x, it.value, rr.value, code


PH_PCG_NOALLOC_MAX_N = 262144


class Schwarz:
    """Edge-patch additive Schwarz preconditioner of a mesh's assembled H
    (``values`` from ``Mesh.assemble``); ``solve`` runs PCG with it."""

    def __init__(self, mesh, values, stream=None):
        h = ctypes.c_void_p()
        self._h = None
        self.mesh = mesh
        _check(load().ph_schwarz_create(mesh.handle, _ptr(values.contiguous()), _stream(stream), ctypes.byref(h)),
               "ph_schwarz_create")
        self._h = h

    def solve(self, values, rhs, x=None, rtol=1e-12, maxit=20000, stream=None, check=True):
        """Returns (x, iters, relres, status) as ph_solve_pcg."""
        n = rhs.numel()
        if x is None:
            x = torch.empty(n, dtype=torch.float64, device=rhs.device)
        it = ctypes.c_int32(0)
        rr = ctypes.c_double(0)
        code = load().ph_solve_pcg_schwarz(self.mesh.handle, _ptr(values), self._h, _ptr(rhs), _ptr(x), float(rtol),
                                           int(maxit), ctypes.byref(it), ctypes.byref(rr), _stream(stream))
        if check:
            _check(code, "ph_solve_pcg_schwarz")
        return x, it.value, rr.value, code

    def close(self, stream=None):
        if self._h is not None:
            load().ph_schwarz_destroy(self._h, _stream(stream))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_refined(mesh, values, rhs, P=None, x=None, tol=1e-15, inner_rtol=1e-8, max_steps=20, maxit=100000,
                  stream=None, check=True):
    """H x = rhs to fp64 accuracy by iterative refinement (double-word
    residual) around PCG, Schwarz-preconditioned with P (a Schwarz) or Jacobi
    (P None).  Returns (x, steps, iterations, last relative correction, status)."""
    n = rhs.numel()
    if x is None:
        x = torch.empty(n, dtype=torch.float64, device=rhs.device)
    st, it, corr = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_double(0)
    code = load().ph_solve_refined(mesh.handle, _ptr(values), None if P is None else P._h, _ptr(rhs), _ptr(x),
                                   float(tol), float(inner_rtol), int(max_steps), int(maxit), ctypes.byref(st),
                                   ctypes.byref(it), ctypes.byref(corr), _stream(stream))
    if check:
        _check(code, "ph_solve_refined")
    return x, st.value, it.value, corr.value, code


def ph_spmv(rowptr, colind, values, x, y=None, stream=None):
    n = x.numel()
    y = torch.empty_like(x) if y is None else y
    _check(load().ph_spmv(n, _ptr(rowptr), _ptr(colind), _ptr(values), _ptr(x), _ptr(y), _stream(stream)),
           "ph_spmv")
    return y


class Mesh:
    """A device mesh (``ph_mesh``): connectivity, CSR pattern and geometry.

    ``coord`` (nC x 3 float64) and ``tet`` (nE x 4 int32) are CUDA tensors;
    ``neumann`` (nN x 3 int32) optional.  geometry "dw" builds with
    ph_mesh_create_dw (double-word geometry record, for ph_assemble_dw).
    Methods allocate outputs with torch and call the matching ``ph_*`` entry
    point on the current stream.
    """

    def __init__(self, coord, tet, neumann=None, stream=None, geometry="f64"):
        L = load()
        coord = coord.contiguous()
        tet = tet.contiguous()
        if coord.dtype != torch.float64 or tet.dtype != torch.int32:
            raise ValueError("coord float64, tet int32")
        nb = None if neumann is None or neumann.numel() == 0 else neumann.contiguous()
        if nb is not None and nb.dtype != torch.int32:
            raise ValueError("neumann int32")
        if geometry not in ("f64", "dw"):
            raise ValueError("geometry: 'f64' or 'dw'")
        h = ctypes.c_void_p()
        self._h = None
        fn = L.ph_mesh_create if geometry == "f64" else L.ph_mesh_create_dw
        _check(fn(_ptr(coord), coord.shape[0], _ptr(tet), tet.shape[0], _ptr(nb), 0 if nb is None else nb.shape[0],
                  _stream(stream), ctypes.byref(h)), "ph_mesh_create" if geometry == "f64" else "ph_mesh_create_dw")
        self._adopt(h, coord.device)

    @classmethod
    def _from_handle(cls, h, device):
        m = cls.__new__(cls)
        m._h = None
        m._adopt(h, device)
        return m

    def _adopt(self, h, device):
        L = load()
        self._h = h
        self.device = device
        inf = ph_info()
        _check(L.ph_mesh_info(h, ctypes.byref(inf)), "ph_mesh_info")
        self.info = {f: int(getattr(inf, f)) for f, _ in ph_info._fields_}
        self.nE, self.nC, self.nF = self.info["nE"], self.info["nC"], self.info["nF"]
        self.L, self.nnz = self.info["L"], self.info["nnz"]

    @property
    def handle(self):
        return self._h

    def close(self, stream=None):
        if self._h is not None:
            load().ph_mesh_destroy(self._h, _stream(stream))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _empty(self, n, dtype):
        return torch.empty(n, dtype=dtype, device=self.device)

    def faces(self, stream=None):
        nE, nF = self.nE, self.nF
        out = {
            "tet_face": self._empty((nE, 4), torch.int32),
            "face_tet": self._empty((nF, 2), torch.int32),
            "face_vtx": self._empty((nF, 3), torch.int32),
            "face_kind": self._empty(nF, torch.int8),
            "face_mult": self._empty(nF, torch.int32),
            "face_centroid": self._empty((nF, 3), torch.float64),
            "face_area": self._empty(nF, torch.float64),
        }
        _check(load().ph_mesh_faces(self._h, *[_ptr(out[k]) for k in ("tet_face", "face_tet", "face_vtx", "face_kind",
                                                                      "face_mult", "face_centroid", "face_area")],
                                    _stream(stream)), "ph_mesh_faces")
        return out

    def csr_pattern(self, stream=None):
        rowptr = self._empty(self.L + 1, torch.int32)
        colind = self._empty(self.nnz, torch.int32)
        _check(load().ph_csr_pattern(self._h, _ptr(rowptr), _ptr(colind), _stream(stream)), "ph_csr_pattern")
        return rowptr, colind

    def assemble(self, a, c, f_face, uD_face=None, gN_face=None, values=None, rhs=None, factor=None, stream=None,
                 variant="f64"):
        """H values and rhs; with ``factor`` (nE*10 float64, or True to
        allocate) also the element factor for recover_factored.  variant
        "dw" runs ph_assemble_dw (condensation kernel in double-word)."""
        _need(a, torch.float64, self.nE, "a")
        _need(f_face, torch.float64, self.nF, "f_face")
        if uD_face is not None:
            _need(uD_face, torch.float64, self.nF, "uD_face")
        if gN_face is not None:
            _need(gN_face, torch.float64, self.nF, "gN_face")
        values = self._empty(self.nnz, torch.float64) if values is None else _need(values, torch.float64, self.nnz,
                                                                                    "values")
        rhs = self._empty(self.L, torch.float64) if rhs is None else _need(rhs, torch.float64, self.L, "rhs")
        if factor is True:
            factor = self._empty((self.nE, 10), torch.float64)
        elif factor is not None:
            _need(factor, torch.float64, 10 * self.nE, "factor")
        if variant not in ("f64", "dw"):
            raise ValueError("variant: 'f64' or 'dw'")
        fn = load().ph_assemble if variant == "f64" else load().ph_assemble_dw
        _check(fn(self._h, _ptr(a), float(c), _ptr(f_face), _ptr(uD_face), _ptr(gN_face), _ptr(values), _ptr(rhs),
                  _ptr(factor), _stream(stream)), "ph_assemble" if variant == "f64" else "ph_assemble_dw")
        if factor is not None:
            return values, rhs, factor
        return values, rhs

    def recover(self, a, c, f_face, lam, gN_face=None, u=None, stream=None):
        _need(a, torch.float64, self.nE, "a")
        _need(f_face, torch.float64, self.nF, "f_face")
        _need(lam, torch.float64, self.L, "lambda")
        if gN_face is not None:
            _need(gN_face, torch.float64, self.nF, "gN_face")
        u = self._empty((self.nE, 4), torch.float64) if u is None else _need(u, torch.float64, 4 * self.nE, "u")
        _check(load().ph_recover(self._h, _ptr(a), float(c), _ptr(f_face), _ptr(gN_face), _ptr(lam), _ptr(u),
                                 _stream(stream)), "ph_recover")
        return u

    def recover_factored(self, factor, c, f_face, lam, gN_face=None, u=None, stream=None, variant="f64"):
        """U from the element factor of assemble(); variant "dw" computes the
        factor's product in double-word arithmetic (ph_recover_factored_dw)."""
        if variant not in ("f64", "dw"):
            raise ValueError("variant: 'f64' or 'dw'")
        name = "ph_recover_factored" if variant == "f64" else "ph_recover_factored_dw"
        _need(factor, torch.float64, 10 * self.nE, "factor")
        _need(f_face, torch.float64, self.nF, "f_face")
        _need(lam, torch.float64, self.L, "lambda")
        if gN_face is not None:
            _need(gN_face, torch.float64, self.nF, "gN_face")
        u = self._empty((self.nE, 4), torch.float64) if u is None else _need(u, torch.float64, 4 * self.nE, "u")
        _check(getattr(load(), name)(self._h, _ptr(factor), float(c), _ptr(f_face), _ptr(gN_face), _ptr(lam),
                                     _ptr(u), _stream(stream)), name)
        return u

    def misfit(self, u, u_obs, stream=None):
        """J = 1/2 sum_T e' M(T) e as a 0-dim CUDA tensor."""
        _need(u, torch.float64, 4 * self.nE, "u")
        _need(u_obs, torch.float64, 4 * self.nE, "u_obs")
        J = torch.empty((), dtype=torch.float64, device=self.device)
        _check(load().ph_misfit(self._h, _ptr(u), _ptr(u_obs), _ptr(J), _stream(stream)), "ph_misfit")
        return J

    def adjoint_rhs(self, factor, c, u, u_obs, rhs_q=None, stream=None):
        _need(factor, torch.float64, 10 * self.nE, "factor")
        rhs_q = self._empty(self.L, torch.float64) if rhs_q is None else _need(rhs_q, torch.float64, self.L, "rhs_q")
        _check(load().ph_adjoint_rhs(self._h, _ptr(factor), float(c), _ptr(u), _ptr(u_obs), _ptr(rhs_q),
                                     _stream(stream)), "ph_adjoint_rhs")
        return rhs_q

    def adjoint_grad(self, a, factor, c, u, u_obs, q, grad=None, stream=None):
        _need(a, torch.float64, self.nE, "a")
        _need(q, torch.float64, self.L, "q")
        grad = self._empty(self.nE, torch.float64) if grad is None else _need(grad, torch.float64, self.nE, "grad")
        _check(load().ph_adjoint_grad(self._h, _ptr(a), _ptr(factor), float(c), _ptr(u), _ptr(u_obs), _ptr(q),
                                      _ptr(grad), _stream(stream)), "ph_adjoint_grad")
        return grad

    def check(self, stream=None):
        _check(load().ph_mesh_check(self._h, _stream(stream)), "ph_mesh_check")


def ph_mesh_create(coord, tet, neumann=None, stream=None) -> Mesh:
    return Mesh(coord, tet, neumann, stream)


def create_meshes(coords, tets, neumanns=None, stream=None):
    """Build many meshes in one batched enqueue (ph_mesh_create_batch): lists
    of CUDA tensors (coord nC x 3 float64, tet nE x 4 int32, neumann nN x 3
    int32 or None).  Returns a list of Mesh objects sharing one allocation."""
    n = len(coords)
    coords = [c.contiguous() for c in coords]
    tets = [t.contiguous() for t in tets]
    nbs = [None if (neumanns is None or nb is None or nb.numel() == 0) else nb.contiguous()
           for nb in (neumanns or [None] * n)]
    for c, t, nb in zip(coords, tets, nbs):
        if c.dtype != torch.float64 or t.dtype != torch.int32 or (nb is not None and nb.dtype != torch.int32):
            raise ValueError("coord float64, tet and neumann int32")
    arr = lambda xs: _ptr_array(xs)
    i64 = lambda xs: (ctypes.c_int64 * max(n, 1))(*xs)
    handles = (ctypes.c_void_p * max(n, 1))()
    _check(load().ph_mesh_create_batch(n, arr(coords), i64([c.shape[0] for c in coords]), arr(tets),
                                       i64([t.shape[0] for t in tets]), arr(nbs),
                                       i64([0 if nb is None else nb.shape[0] for nb in nbs]), _stream(stream),
                                       handles), "ph_mesh_create_batch")
    dev = coords[0].device if n else torch.device("cuda")
    return [Mesh._from_handle(ctypes.c_void_p(handles[i]), dev) for i in range(n)]


def _hptr(t):
    """Address of a contiguous CPU tensor (host buffer), or None."""
    if t is None:
        return None
    if t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CPU tensor")
    return ctypes.c_void_p(t.data_ptr())


def ph_host_mesh_query(coord, tet, neumann=None, centroids=True, stream=None):
    """Counts (dict as Mesh.info) and, with centroids, the face centroids
    (nF x 3 CPU tensor) of the mesh that host tensors build."""
    nE = tet.shape[0]
    nN = 0 if neumann is None else neumann.shape[0]
    cap = 4 * nE + nN
    cen = torch.empty((max(cap, 1), 3), dtype=torch.float64) if centroids else None
    inf = ph_info()
    _check(load().ph_host_mesh_query(_hptr(coord), coord.shape[0], _hptr(tet), nE, _hptr(neumann), nN,
                                     ctypes.byref(inf), _hptr(cen), cap if centroids else 0, _stream(stream)),
           "ph_host_mesh_query")
    info = {f: int(getattr(inf, f)) for f, _ in ph_info._fields_}
    return info, (cen[:info["nF"]] if centroids else None)


def ph_assemble_host(coord, tet, a, c, f_face, counts, lam=None, uD_face=None, gN_face=None, neumann=None,
                     out=None, stream=None):
    """The whole path from and to host (CPU, ideally pinned) tensors.
    ``counts`` = (nF, L, nnz) of the mesh; returns dict(rowptr, colind,
    values, rhs[, u]) of CPU tensors (``out`` supplies them)."""
    nF, L, nnz = (int(x) for x in counts)
    nE = tet.shape[0]
    if out is None:
        out = {"rowptr": torch.empty(L + 1, dtype=torch.int32), "colind": torch.empty(nnz, dtype=torch.int32),
               "values": torch.empty(nnz, dtype=torch.float64), "rhs": torch.empty(L, dtype=torch.float64)}
        if lam is not None:
            out["u"] = torch.empty((nE, 4), dtype=torch.float64)
    _check(load().ph_assemble_host(_hptr(coord), coord.shape[0], _hptr(tet), nE, _hptr(neumann),
                                   0 if neumann is None else neumann.shape[0], nF, L, nnz, _hptr(a), float(c),
                                   _hptr(f_face), _hptr(uD_face), _hptr(gN_face), _hptr(lam), _hptr(out["rowptr"]),
                                   _hptr(out["colind"]), _hptr(out["values"]), _hptr(out["rhs"]), _hptr(out.get("u")),
                                   _stream(stream)), "ph_assemble_host")
    return out


def ph_timing_enable(on=True):
    """Switch the library's per-kernel CUDA-event timing: True or 1 for the
    element kernels, 2 for the mesh build and scans, 3 for both, False/0 off."""
    _check(load().ph_timing_enable(int(on)), "ph_timing_enable")


def ph_kernel_time(kernel: str, reset: bool = False):
    """(total device ms, launches) of the named kernel while timing was on."""
    ms, n = ctypes.c_double(), ctypes.c_int64()
    _check(load().ph_kernel_time(kernel.encode(), 1 if reset else 0, ctypes.byref(ms), ctypes.byref(n)),
           "ph_kernel_time")
    return ms.value, n.value


def ph_rcp(x, stream=None):
    """1/x with the device reciprocal of the element kernels (for testing)."""
    x = x.contiguous()
    y = torch.empty_like(x)
    _check(load().ph_rcp(_ptr(x), x.numel(), _ptr(y), _stream(stream)), "ph_rcp")
    return y


def ph_half_sqrt(x, stream=None):
    """sqrt(x)/2 with the device square root of the face areas (for testing)."""
    x = x.contiguous()
    y = torch.empty_like(x)
    _check(load().ph_half_sqrt(_ptr(x), x.numel(), _ptr(y), _stream(stream)), "ph_half_sqrt")
    return y


def ph_test_fail_alloc(after):
    """Test hook: the (after+1)-th next pool allocation fails (after < 0: off)."""
    _check(load().ph_test_fail_alloc(int(after)), "ph_test_fail_alloc")


def ph_test_scan_withhold(on):
    """Test hook: scans withhold one tile's publication (bounded waits run out)."""
    _check(load().ph_test_scan_withhold(1 if on else 0), "ph_test_scan_withhold")


def ph_pool_in_use() -> int:
    """Bytes held by live allocations of the library's pool on this device."""
    n = ctypes.c_int64()
    _check(load().ph_pool_in_use(ctypes.byref(n)), "ph_pool_in_use")
    return n.value


def ph_fp64_peak(iters=4000, stream=None):
    """(DFMA operations per second, launch ms) of the library's FP64
    throughput probe on the current device."""
    ops, ms = ctypes.c_double(), ctypes.c_double()
    _check(load().ph_fp64_peak(int(iters), ctypes.byref(ops), ctypes.byref(ms), _stream(stream)), "ph_fp64_peak")
    return ops.value, ms.value


def ph_refine(coord, tet, lists=None, stream=None):
    """One level of the 1->12 refinement on the device.  Returns (coord, tet,
    lists, nEd) as CUDA tensors (lists None if none were given) and the edge
    count of the input mesh."""
    L = load()
    coord, tet = coord.contiguous(), tet.contiguous()
    nl = 0 if lists is None else lists.shape[0]
    h = ctypes.c_void_p()
    _check(L.ph_refine(_ptr(coord), coord.shape[0], _ptr(tet), tet.shape[0],
                       _ptr(lists.contiguous()) if nl else None, nl, _stream(stream), ctypes.byref(h)), "ph_refine")
    try:
        nC, nE, nEd, nl2 = (ctypes.c_int64() for _ in range(4))
        _check(L.ph_refined_info(h, ctypes.byref(nC), ctypes.byref(nE), ctypes.byref(nEd), ctypes.byref(nl2)),
               "ph_refined_info")
        c2 = torch.empty((nC.value, 3), dtype=torch.float64, device=coord.device)
        t2 = torch.empty((nE.value, 4), dtype=torch.int32, device=coord.device)
        l2 = torch.empty((nl2.value, 3), dtype=torch.int32, device=coord.device) if nl else None
        _check(L.ph_refined_copy(h, _ptr(c2), _ptr(t2), _ptr(l2), _stream(stream)), "ph_refined_copy")
    finally:
        L.ph_refined_destroy(h, _stream(stream))
    return c2, t2, l2, nEd.value


def _ptr_array(tensors):
    arr = (ctypes.c_void_p * max(len(tensors), 1))()
    for i, t in enumerate(tensors):
        arr[i] = None if t is None else t.data_ptr()
    return arr


class Batch:
    """A batch of meshes assembled by one persistent kernel (ph_batch_*).

    bind() takes per-problem lists of CUDA tensors (outputs included); the
    lists are kept alive by the Batch while bound."""

    def __init__(self, meshes, stream=None):
        self.meshes = list(meshes)
        h = ctypes.c_void_p()
        handles = (ctypes.c_void_p * max(len(self.meshes), 1))(*[m.handle.value for m in self.meshes])
        self._h = None
        _check(load().ph_batch_create(handles, len(self.meshes), _stream(stream), ctypes.byref(h)), "ph_batch_create")
        self._h = h
        self._bound = None

    def bind(self, a, c, f_face, values, rhs, factor=None, uD_face=None, gN_face=None, stream=None):
        n = len(self.meshes)
        for m, aa, ff, vv, rr in zip(self.meshes, a, f_face, values, rhs):
            _need(aa, torch.float64, m.nE, "a")
            _need(ff, torch.float64, m.nF, "f_face")
            _need(vv, torch.float64, m.nnz, "values")
            _need(rr, torch.float64, m.L, "rhs")
        if factor is not None:
            for m, fa in zip(self.meshes, factor):
                if fa is not None:
                    _need(fa, torch.float64, 10 * m.nE, "factor")
        cs = (ctypes.c_double * max(n, 1))(*[float(x) for x in c])
        arrs = [_ptr_array(x) if x is not None else None for x in (a, f_face, uD_face, gN_face, values, rhs, factor)]
        _check(load().ph_batch_bind(self._h, arrs[0], cs, arrs[1], arrs[2], arrs[3], arrs[4], arrs[5], arrs[6],
                                    _stream(stream)), "ph_batch_bind")
        self._bound = (a, c, f_face, values, rhs, factor, uD_face, gN_face)

    def bind_recovery(self, lam, u, stream=None):
        """Recovery from the bound factors into u[i] (lists of CUDA tensors;
        lam None removes it)."""
        if lam is None:
            _check(load().ph_batch_bind_recovery(self._h, None, None, _stream(stream)), "ph_batch_bind_recovery")
            self._recovery = None
            return
        for m, l, uu in zip(self.meshes, lam, u):
            _need(l, torch.float64, m.L, "lambda")
            _need(uu, torch.float64, 4 * m.nE, "u")
        _check(load().ph_batch_bind_recovery(self._h, _ptr_array(lam), _ptr_array(u), _stream(stream)),
               "ph_batch_bind_recovery")
        self._recovery = (lam, u)

    def assemble(self, stream=None):
        _check(load().ph_batch_assemble(self._h, _stream(stream)), "ph_batch_assemble")

    def graph_launch(self, stream=None):
        _check(load().ph_batch_graph_launch(self._h, _stream(stream)), "ph_batch_graph_launch")

    def autotune(self, reps=3, stream=None):
        ms = ctypes.c_float(0)
        _check(load().ph_batch_autotune(self._h, int(reps), ctypes.byref(ms), _stream(stream)), "ph_batch_autotune")
        return ms.value

    def set_config(self, tile, threads, blocks_per_sm, stream=None):
        _check(load().ph_batch_set_config(self._h, tile, threads, blocks_per_sm, _stream(stream)),
               "ph_batch_set_config")

    def get_config(self):
        t, th, b = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(load().ph_batch_get_config(self._h, ctypes.byref(t), ctypes.byref(th), ctypes.byref(b)),
               "ph_batch_get_config")
        return {"tile": t.value, "threads": th.value, "blocks_per_sm": b.value}

    def close(self, stream=None):
        if self._h is not None:
            load().ph_batch_destroy(self._h, _stream(stream))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_system(mesh, values, rhs, rtol, maxit, precond="schwarz", P=None):
    """H Lambda = rhs on the mesh's CSR pattern: PCG with the edge-patch
    Schwarz preconditioner (P reused when given) or Jacobi.  Returns
    (Lambda, iterations, P)."""
    if precond == "schwarz":
        P = Schwarz(mesh, values) if P is None else P
        lam, it, _, _ = P.solve(values, rhs, rtol=rtol, maxit=maxit)
        return lam, it, P
    if precond != "jacobi":
        raise ValueError("precond: 'schwarz' or 'jacobi'")
    rowptr, colind = mesh.csr_pattern()
    lam, it, _, _ = ph_solve_pcg(rowptr, colind, values, rhs, rtol=rtol, maxit=maxit)
    return lam, it, None


class MisfitFunction(torch.autograd.Function):
    """J(log a) = 1/2 sum_T e_T' M(T) e_T, e = U(a) - U_obs, through assembly,
    condensation, the PCG solve and recovery; backward is the hand-written
    adjoint (ph_adjoint_rhs, a second solve with the same H -- and the same
    preconditioner -- and ph_adjoint_grad).

    apply(log_a, mesh, c, f_face, u_obs, uD_face, gN_face, rtol, maxit, precond)
    """

    @staticmethod
    def forward(ctx, log_a, mesh, c, f_face, u_obs, uD_face=None, gN_face=None, rtol=1e-12, maxit=50000,
                precond="schwarz"):
        a = torch.exp(log_a)
        values, rhs, factor = mesh.assemble(a, c, f_face, uD_face, gN_face, factor=True)
        lam, _, P = solve_system(mesh, values, rhs, rtol, maxit, precond)
        u = mesh.recover_factored(factor, c, f_face, lam, gN_face)
        J = mesh.misfit(u, u_obs)
        ctx.mesh, ctx.c, ctx.rtol, ctx.maxit, ctx.precond, ctx.P = mesh, c, rtol, maxit, precond, P
        ctx.save_for_backward(a, values, factor, u, u_obs)
        return J

    @staticmethod
    def backward(ctx, gJ):
        a, values, factor, u, u_obs = ctx.saved_tensors
        mesh = ctx.mesh
        rhs_q = mesh.adjoint_rhs(factor, ctx.c, u, u_obs)
        q, _, _ = solve_system(mesh, values, rhs_q, ctx.rtol, ctx.maxit, ctx.precond, ctx.P)
        grad = mesh.adjoint_grad(a, factor, ctx.c, u, u_obs, q)
        if ctx.P is not None:
            ctx.P.close()
            ctx.P = None
        return gJ * grad, None, None, None, None, None, None, None, None, None


def misfit(log_a, mesh, c, f_face, u_obs, uD_face=None, gN_face=None, rtol=1e-12, maxit=50000, precond="schwarz"):
    """Differentiable misfit (see MisfitFunction)."""
    return MisfitFunction.apply(log_a, mesh, c, f_face, u_obs, uD_face, gN_face, rtol, maxit, precond)
