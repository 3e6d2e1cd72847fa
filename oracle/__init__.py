"""Independent CPU oracle for the primal hybrid FEM path (arXiv 2509.11133).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run
anything here.  The CUDA library never does, and this package imports nothing
from it.  The arithmetic lives in ``ph_oracle.c`` (plain C, binary128 per
element; see its header); this module marshals arguments with ctypes and uses
library primitives only for the global solve (numpy / scipy).

Functions and the passage each one follows:
  faces              Section 3.3 (FacesUp), jump/T+ convention of Section 2.2
  multipliers        RFaces restriction, Listing SchurComplement_vectorization
  csr_pattern        sparsity of sum_T P_T' S(T) P_T (Algorithm 1, assembly)
  face_centroids     Listing StiffMassPH (Ct = (P1+P2+P3)/3)
  tet_local          Eqs. K(T), M(T), C(T); Eq. schur; Algorithm 1 first loop
  tet_recover        Algorithm 1 second loop, one element
  tet_matrices       Eqs. K(T), M(T), C(T) and the load rule of Section 4.3
  assemble           Algorithm 1 assembly + b_D (Section 4.3); its element
                     loop may run on several host threads (same bits)
  solve              Eq. schur, S Lambda = rhs (a library sparse/dense solve)
  residual, solve_refined
                     the same solve refined to fp64 accuracy (residual in
                     binary128)
  recover            Algorithm 1 second loop (host threads as assemble)
  element_blocks     Eq. VectorForm blocks (monolithic check)
  misfit, monolithic, adjoint_gradient
                     gradient of J = 1/2 sum_T e' M(T) e with respect to
                     log a_T through Eq. VectorForm (not in the paper)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ph_oracle.c")
_SO = os.path.join(_HERE, "libph_oracle.so")
_LIB = None
_LOCK = threading.Lock()

STATUS = {0: "OK", 1: "ARG", 2: "DEGENERATE", 3: "NONMANIFOLD", 4: "OVERFLOW", 5: "NOMEM"}
KIND_INTERIOR, KIND_DIRICHLET, KIND_NEUMANN = 0, 1, 2


class OracleError(RuntimeError):
    def __init__(self, code, where):
        super().__init__(f"oracle {where}: {STATUS.get(code, code)}")
        self.code = code
        self.name = STATUS.get(code, str(code))


def build(force: bool = False) -> str:
    """Compile ph_oracle.c into libph_oracle.so next to it (plain gcc)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-fopenmp", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _configure(L):
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    D = ctypes.c_double
    L.or_faces.argtypes = [I64, I64, P, I64, P, P, P, P, P, P]
    L.or_multipliers.argtypes = [I64, P, P, P]
    L.or_csr_pattern.argtypes = [I64, P, P, I64, P, P, P]
    L.or_face_centroids.argtypes = [I64, P, P, P]
    L.or_tet_local.argtypes = [P, D, D, P, P, P, P, P, P]
    L.or_tet_matrices.argtypes = [P, P, P, P, P, P, P, P, P]
    L.or_assemble.argtypes = [I64, P, P, P, I64, P, P, P, I64, P, P, P, D, P, P, P, P, P, P]
    L.or_recover.argtypes = [I64, P, P, P, P, P, P, D, P, P, P, P]
    L.or_element_blocks.argtypes = [I64, P, P, P, P, P, D, P, P, P, P, P]
    L.or_tet_recover.argtypes = [P, D, D, P, P, P, P, P, P]
    L.or_residual.argtypes = [I64, P, P, P, P, P, P]
    L.or_assemble_mt.argtypes = L.or_assemble.argtypes + [ctypes.c_int]
    L.or_recover_mt.argtypes = L.or_recover.argtypes + [ctypes.c_int]
    for f in ("or_faces", "or_multipliers", "or_csr_pattern", "or_face_centroids", "or_tet_local",
              "or_tet_matrices", "or_assemble", "or_recover", "or_element_blocks", "or_tet_recover",
              "or_assemble_mt", "or_recover_mt", "or_residual"):
        getattr(L, f).restype = ctypes.c_int
    return L


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            build()
            _LIB = _configure(ctypes.CDLL(_SO))
    return _LIB


class use_library:
    """Context manager: run the oracle functions on another build of
    ph_oracle.c (the mutation tests load deliberately broken copies)."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _LIB
        _lib()
        self.saved = _LIB
        _LIB = _configure(ctypes.CDLL(self.path))
        return self

    def __exit__(self, *exc):
        global _LIB
        _LIB = self.saved
        return False


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _check(code, where):
    if code != 0:
        raise OracleError(code, where)


def faces(tet, nC, neumann=None):
    tet = _c(tet, np.int32).reshape(-1, 4)
    nE = tet.shape[0]
    nb = _c(neumann if neumann is not None else np.zeros((0, 3)), np.int32).reshape(-1, 3)
    cap = max(4 * nE, 1)
    tet_face = np.zeros(max(4 * nE, 1), np.int32)
    face_tet = np.zeros(2 * cap, np.int32)
    face_vtx = np.zeros(3 * cap, np.int32)
    face_kind = np.zeros(cap, np.int8)
    nF = ctypes.c_int64(0)
    _check(_lib().or_faces(nE, int(nC), _p(tet), nb.shape[0], _p(nb), _p(tet_face), _p(face_tet),
                           _p(face_vtx), _p(face_kind), ctypes.byref(nF)), "faces")
    n = nF.value
    return {
        "nF": n,
        "tet_face": tet_face[:4 * nE].reshape(nE, 4),
        "face_tet": face_tet[:2 * n].reshape(n, 2),
        "face_vtx": face_vtx[:3 * n].reshape(n, 3),
        "face_kind": face_kind[:n],
    }


def multipliers(face_kind):
    fk = _c(face_kind, np.int8)
    fm = np.zeros(max(fk.size, 1), np.int32)
    L = ctypes.c_int64(0)
    _check(_lib().or_multipliers(fk.size, _p(fk), _p(fm), ctypes.byref(L)), "multipliers")
    return fm[:fk.size], L.value


def csr_pattern(tet_face, face_mult, L):
    tf = _c(tet_face, np.int32).reshape(-1, 4)
    fm = _c(face_mult, np.int32)
    nE = tf.shape[0]
    rowptr = np.zeros(L + 1, np.int32)
    colind = np.zeros(max(16 * nE, 1), np.int32)
    nnz = ctypes.c_int64(0)
    _check(_lib().or_csr_pattern(nE, _p(tf), _p(fm), int(L), _p(rowptr), _p(colind), ctypes.byref(nnz)), "csr")
    return rowptr, colind[:nnz.value].copy()


def face_centroids(coord, face_vtx):
    coord = _c(coord, np.float64)
    fv = _c(face_vtx, np.int32).reshape(-1, 3)
    out = np.zeros((fv.shape[0], 3), np.float64)
    _check(_lib().or_face_centroids(fv.shape[0], _p(fv), _p(coord), _p(out)), "centroids")
    return out


def tet_local(P, a, c, f4, sigma4, kind4=(0, 0, 0, 0), g4=(0.0, 0.0, 0.0, 0.0)):
    P = _c(P, np.float64).reshape(12)
    f4 = _c(f4, np.float64)
    s4 = _c(sigma4, np.int32)
    k4 = _c(kind4, np.int32)
    g4 = _c(g4, np.float64)
    S = np.zeros(16)
    g = np.zeros(4)
    _check(_lib().or_tet_local(_p(P), float(a), float(c), _p(f4), _p(s4), _p(k4), _p(g4), _p(S), _p(g)),
           "tet_local")
    return S.reshape(4, 4), g


def tet_recover(P, a, c, f4, sigma4, lam4, kind4=(0, 0, 0, 0), g4=(0.0, 0.0, 0.0, 0.0)):
    """U = A^-1 (B + C' lam) of one element (Algorithm 1, second loop)."""
    U = np.zeros(4)
    _check(_lib().or_tet_recover(_p(_c(P, np.float64).reshape(12)), float(a), float(c), _p(_c(f4, np.float64)),
                                 _p(_c(sigma4, np.int32)), _p(_c(kind4, np.int32)), _p(_c(g4, np.float64)),
                                 _p(_c(lam4, np.float64)), _p(U)), "tet_recover")
    return U


def tet_matrices(P, f4=(0, 0, 0, 0), sigma4=(1, 1, 1, 1)):
    P = _c(P, np.float64).reshape(12)
    f4 = _c(f4, np.float64)
    s4 = _c(sigma4, np.int32)
    K, M, C = np.zeros(16), np.zeros(16), np.zeros(16)
    area, B = np.zeros(4), np.zeros(4)
    vol = ctypes.c_double(0)
    _check(_lib().or_tet_matrices(_p(P), _p(f4), _p(s4), _p(K), _p(M), _p(C), _p(area), ctypes.byref(vol),
                                  _p(B)), "tet_matrices")
    return {"K": K.reshape(4, 4), "M": M.reshape(4, 4), "C": C.reshape(4, 4), "area": area,
            "vol": vol.value, "B": B}


def threads() -> int:
    """Host threads the element loops use by default (every core)."""
    return max(1, os.cpu_count() or 1)


def assemble(coord, tet, fc, csr, a, c, f_face, uD_face=None, gN_face=None, nthreads=None):
    """fc: output of faces(); csr: dict with face_mult, L, rowptr, colind.
    nthreads = 1 runs the plain element loop; more threads share out the
    element computations (bit-identical result, see or_assemble_mt)."""
    coord = _c(coord, np.float64)
    tet = _c(tet, np.int32)
    nE = tet.shape[0]
    rowptr, colind = csr["rowptr"], csr["colind"]
    L = csr["L"]
    values = np.zeros(max(colind.size, 1))
    rhs = np.zeros(max(L, 1))
    rhs_abs = np.zeros(max(L, 1))
    a = _c(a, np.float64)
    f_face = _c(f_face, np.float64)
    uD = None if uD_face is None else _c(uD_face, np.float64)
    gN = None if gN_face is None else _c(gN_face, np.float64)
    nt = threads() if nthreads is None else int(nthreads)
    args = [nE, _p(coord), _p(tet), _p(_c(fc["tet_face"], np.int32)), fc["nF"], _p(_c(fc["face_kind"], np.int8)),
            _p(_c(csr["face_mult"], np.int32)), _p(_c(fc["face_vtx"], np.int32)), L, _p(rowptr), _p(colind), _p(a),
            float(c), _p(f_face), _p(uD), _p(gN), _p(values), _p(rhs), _p(rhs_abs)]
    if nt <= 1:
        _check(_lib().or_assemble(*args), "assemble")
    else:
        _check(_lib().or_assemble_mt(*args, nt), "assemble")
    return values[:colind.size], rhs[:L], rhs_abs[:L]


def recover(coord, tet, fc, face_mult, a, c, f_face, lam, gN_face=None, nthreads=None):
    coord = _c(coord, np.float64)
    tet = _c(tet, np.int32)
    nE = tet.shape[0]
    U = np.zeros((max(nE, 1), 4))
    gN = None if gN_face is None else _c(gN_face, np.float64)
    lam = _c(lam if len(lam) else np.zeros(1), np.float64)
    args = [nE, _p(coord), _p(tet), _p(_c(fc["tet_face"], np.int32)), _p(_c(fc["face_kind"], np.int8)),
            _p(_c(face_mult, np.int32)), _p(_c(a, np.float64)), float(c), _p(_c(f_face, np.float64)), _p(gN),
            _p(lam), _p(U)]
    nt = threads() if nthreads is None else int(nthreads)
    if nt <= 1:
        _check(_lib().or_recover(*args), "recover")
    else:
        _check(_lib().or_recover_mt(*args, nt), "recover")
    return U[:nE]


def element_blocks(t, coord, tet, fc, a, c, f_face, gN_face=None):
    A, C, B = np.zeros(16), np.zeros(16), np.zeros(4)
    gN = None if gN_face is None else _c(gN_face, np.float64)
    _check(_lib().or_element_blocks(int(t), _p(_c(coord, np.float64)), _p(_c(tet, np.int32)),
                                    _p(_c(fc["tet_face"], np.int32)), _p(_c(fc["face_kind"], np.int8)),
                                    _p(_c(a, np.float64)), float(c), _p(_c(f_face, np.float64)), _p(gN), _p(A),
                                    _p(C), _p(B)), "element_blocks")
    return A.reshape(4, 4), C.reshape(4, 4), B


def solve(rowptr, colind, values, rhs):
    """S Lambda = rhs (Eq. schur) by a library solve: dense Cholesky for small
    systems, SuperLU otherwise."""
    L = rhs.size
    if L == 0:
        return np.zeros(0)
    if L <= 4000:
        H = np.zeros((L, L))
        for r in range(L):
            H[r, colind[rowptr[r]:rowptr[r + 1]]] = values[rowptr[r]:rowptr[r + 1]]
        import scipy.linalg as sla
        cf = sla.cho_factor(H)
        return sla.cho_solve(cf, rhs)
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    H = sp.csr_matrix((values, colind, rowptr), shape=(L, L)).tocsc()
    return spla.spsolve(H, rhs)


def residual(rowptr, colind, values, x, b):
    """b - H x with the row sums formed in binary128 (see or_residual)."""
    n = b.size
    r = np.zeros(max(n, 1))
    rp, ci = _c(rowptr, np.int32), _c(colind, np.int32)
    _check(_lib().or_residual(n, _p(rp), _p(ci), _p(_c(values, np.float64)), _p(_c(x, np.float64)),
                              _p(_c(b, np.float64)), _p(r)), "residual")
    return r[:n]


def solve_refined(rowptr, colind, values, rhs, max_steps=20):
    """S Lambda = rhs solved to fp64 accuracy: a library LU solve, then
    iterative refinement (Wilkinson) with the residual in binary128, until
    the correction is below 2^-53 of the solution.  The error of a plain fp64
    solve is ~cond(H) eps; this one is ~eps for cond(H) eps << 1.
    Returns (Lambda, refinement steps, last relative correction)."""
    L = rhs.size
    if L == 0:
        return np.zeros(0), 0, 0.0
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    H = sp.csr_matrix((values, colind, rowptr), shape=(L, L)).tocsc()
    lu = spla.splu(H)
    x = lu.solve(np.asarray(rhs, np.float64))
    corr = np.inf
    for step in range(1, max_steps + 1):
        d = lu.solve(residual(rowptr, colind, values, x, rhs))
        x = x + d
        corr = np.linalg.norm(d) / max(np.linalg.norm(x), 1e-300)
        if corr <= 2.0 ** -53:
            return x, step, corr
    return x, max_steps, corr


def ulp_sensitivity(rowptr, colind, values, rhs, trials=3, seed=0):
    """Intrinsic sensitivity of the solved face values to the last bit of the
    assembled system: the largest normwise relative change of Lambda (both
    solves refined to fp64 accuracy) when every entry of H -- keeping H
    symmetric -- and of rhs moves by one ulp in a seeded random direction.
    Two correct fp64 assemblies differ by about that much in each entry, so
    no fp64 path can promise solved values closer than this."""
    import scipy.sparse as sp
    L = rhs.size
    x, _, _ = solve_refined(rowptr, colind, values, rhs)
    H = sp.csr_matrix((values, colind, rowptr), shape=(L, L)).tocoo()
    i, j, v = H.row.astype(np.int64), H.col.astype(np.int64), H.data
    lo, hi = np.minimum(i, j), np.maximum(i, j)
    worst = 0.0
    for t in range(trials):
        rng = np.random.Generator(np.random.PCG64(seed + t))
        # direction of entry (i, j) = that of (min, max): a symmetric perturbation
        key = np.unique(lo * L + hi, return_inverse=True)[1]
        up = rng.random(key.max() + 1)[key] < 0.5
        v2 = np.where(up, np.nextafter(v, np.inf), np.nextafter(v, -np.inf))
        H2 = sp.csr_matrix((v2, (i, j)), shape=(L, L))
        H2.sort_indices()
        b2 = np.where(rng.random(L) < 0.5, np.nextafter(rhs, np.inf), np.nextafter(rhs, -np.inf))
        x2, _, _ = solve_refined(H2.indptr.astype(np.int32), H2.indices.astype(np.int32), H2.data, b2)
        worst = max(worst, float(np.linalg.norm(x2 - x) / np.linalg.norm(x)))
    return worst


def pipeline(coord, tet, a, c, f_fn, uD_fn=None, gN_fn=None, neumann=None, do_solve=True):
    """Whole path on the CPU: faces, multipliers, CSR, face data at the
    oracle's own face centroids, assembly, solve, recovery."""
    fc = faces(tet, coord.shape[0], neumann)
    fm, L = multipliers(fc["face_kind"])
    rowptr, colind = csr_pattern(fc["tet_face"], fm, L)
    cen = face_centroids(coord, fc["face_vtx"])
    f_face = np.asarray(f_fn(cen), dtype=np.float64)
    uD_face = None if uD_fn is None else np.asarray(uD_fn(cen), dtype=np.float64)
    gN_face = None if gN_fn is None else np.asarray(gN_fn(cen), dtype=np.float64)
    csr = {"face_mult": fm, "L": L, "rowptr": rowptr, "colind": colind}
    values, rhs, rhs_abs = assemble(coord, tet, fc, csr, a, c, f_face, uD_face, gN_face)
    out = dict(fc=fc, csr=csr, centroids=cen, f_face=f_face, uD_face=uD_face, gN_face=gN_face,
               values=values, rhs=rhs, rhs_abs=rhs_abs)
    if do_solve:
        lam = solve(rowptr, colind, values, rhs)
        U = recover(coord, tet, fc, fm, a, c, f_face, lam, gN_face)
        out.update(lam=lam, U=U)
    return out


# ---------------------------------------------------------------------------
# Adjoint (not in the paper): gradient of a misfit with respect to log a_T
# ---------------------------------------------------------------------------
def misfit(coord, tet, U, U_obs):
    """J = 1/2 sum_T e_T' M(T) e_T, e = U - U_obs (the L2 norm of the broken P1
    difference, M(T) of Eq. M(T))."""
    J = 0.0
    for t in range(tet.shape[0]):
        M = tet_matrices(coord[tet[t]])["M"]
        e = U[t] - U_obs[t]
        J += 0.5 * e @ M @ e
    return J


def monolithic(coord, tet, fc, face_mult, L, a, c, f_face, uD_face=None, gN_face=None):
    """The block saddle system of Eq. VectorForm, K [U; Lambda] = [B; -b_D]
    with K = [[A, -C'], [-C, 0]], as a scipy sparse matrix and right side."""
    import scipy.sparse as sp
    nE = tet.shape[0]
    N = 4 * nE
    rows, cols, vals = [], [], []
    rhs = np.zeros(N + L)
    for t in range(nE):
        A, C, B = element_blocks(t, coord, tet, fc, a, c, f_face, gN_face)
        idx = 4 * t + np.arange(4)
        rows.append(np.repeat(idx, 4)); cols.append(np.tile(idx, 4)); vals.append(A.ravel())
        rhs[idx] = B
        for k in range(4):
            l = face_mult[fc["tet_face"][t, k] & 0x7FFFFFFF]
            if l < 0:
                continue
            rows.append(np.full(4, N + l)); cols.append(idx); vals.append(-C[k])
            rows.append(idx); cols.append(np.full(4, N + l)); vals.append(-C[k])
    if uD_face is not None:
        dir_ = np.where(fc["face_kind"] == KIND_DIRICHLET)[0]
        fv = fc["face_vtx"][dir_]
        x, y, z = coord[fv[:, 0]], coord[fv[:, 1]], coord[fv[:, 2]]
        area = 0.5 * np.linalg.norm(np.cross(z - x, y - x), axis=1)
        rhs[N + face_mult[dir_]] = -area * uD_face[dir_]
    K = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N + L, N + L))
    return K, rhs


def adjoint_gradient(coord, tet, a, c, f_fn, U_obs, uD_fn=None, gN_fn=None, neumann=None):
    """dJ/d(log a_T) by the adjoint of Eq. VectorForm.

    Forward: K [U; Lambda] = [B; -b_D].  J = 1/2 sum_T e_T' M(T) e_T.
    Adjoint: K' [p; q] = [dJ/dU; 0] = [M e; 0] (K is symmetric).
    Since only A(T) = a_T K(T) + c M(T) depends on theta_T = log a_T, with
    dA(T)/dtheta_T = a_T K(T):   dJ/dtheta_T = -a_T p_T' K(T) U_T.
    Solved with a sparse direct solver on the whole saddle system (small
    meshes only).  Returns (J, grad, U, Lambda)."""
    import scipy.sparse.linalg as spla
    fc = faces(tet, coord.shape[0], neumann)
    fm, L = multipliers(fc["face_kind"])
    cen = face_centroids(coord, fc["face_vtx"])
    f_face = np.asarray(f_fn(cen), np.float64)
    uD_face = None if uD_fn is None else np.asarray(uD_fn(cen), np.float64)
    gN_face = None if gN_fn is None else np.asarray(gN_fn(cen), np.float64)
    K, rhs = monolithic(coord, tet, fc, fm, L, a, c, f_face, uD_face, gN_face)
    K = K.tocsc()
    lu = spla.splu(K)
    sol = lu.solve(rhs)
    nE = tet.shape[0]
    U = sol[:4 * nE].reshape(nE, 4)
    lam = sol[4 * nE:]
    e = U - U_obs
    J = 0.0
    src = np.zeros(4 * nE + L)
    Ks = []
    for t in range(nE):
        m = tet_matrices(coord[tet[t]])
        J += 0.5 * e[t] @ m["M"] @ e[t]
        src[4 * t:4 * t + 4] = m["M"] @ e[t]
        Ks.append(m["K"])
    adj = lu.solve(src, trans="T")
    p = adj[:4 * nE].reshape(nE, 4)
    grad = np.array([-a[t] * p[t] @ Ks[t] @ U[t] for t in range(nE)])
    return J, grad, U, lam
