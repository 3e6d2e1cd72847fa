"""System-level pins of the oracle: the condensed solve equals the monolithic
saddle-point solve of Eq. VectorForm, a constant patch test, CSR structure and
the convergence rates of Table 4."""
import numpy as np
import pytest

import meshgen
import oracle
from tests.quadrature import tet_rule, tri_rule

LFACE = [(0, 1, 2), (0, 2, 3), (0, 3, 1), (3, 2, 1)]
OPP = [3, 1, 2, 0]


def _area(coord, fv):
    x, y, z = coord[fv[:, 0]], coord[fv[:, 1]], coord[fv[:, 2]]
    return 0.5 * np.linalg.norm(np.cross(z - x, y - x), axis=1)


@pytest.mark.parametrize("case", ["mixed1", "mixed2", "kuhn_lognormal"])
def test_condensed_equals_monolithic(case):
    if case.startswith("mixed"):
        p = meshgen.problem("paper_mixed", int(case[-1]))
        a = p.a
    else:
        p = meshgen.problem("kuhn_m1_k1")
        a = meshgen.lognormal_field(p.nE, 17)
    r = oracle.pipeline(p.coord, p.tet, a, p.c, p.f, p.uD, p.gN, p.neumann)
    fc, fm, L = r["fc"], r["csr"]["face_mult"], r["csr"]["L"]
    nE = p.nE
    N = 4 * nE
    Mtx = np.zeros((N + L, N + L))
    rhs = np.zeros(N + L)
    for t in range(nE):
        A, C, B = oracle.element_blocks(t, p.coord, p.tet, fc, a, p.c, r["f_face"], r["gN_face"])
        Mtx[4 * t:4 * t + 4, 4 * t:4 * t + 4] = A
        rhs[4 * t:4 * t + 4] = B
        for k in range(4):
            l = fm[fc["tet_face"][t, k] & 0x7FFFFFFF]
            if l < 0:
                continue
            Mtx[N + l, 4 * t:4 * t + 4] -= C[k]
            Mtx[4 * t:4 * t + 4, N + l] -= C[k]
    if r["uD_face"] is not None:
        dir_ = np.where(fc["face_kind"] == oracle.KIND_DIRICHLET)[0]
        rhs[N + fm[dir_]] = -_area(p.coord, fc["face_vtx"][dir_]) * r["uD_face"][dir_]
    sol = np.linalg.solve(Mtx, rhs)
    U_mono, lam_mono = sol[:N].reshape(nE, 4), sol[N:]
    assert np.linalg.norm(r["lam"] - lam_mono) <= 1e-10 * np.linalg.norm(lam_mono)
    assert np.linalg.norm(r["U"] - U_mono) <= 1e-10 * np.linalg.norm(U_mono)


def test_patch_constant():
    """f = f0, u_D = f0/c on the whole boundary: U = f0/c, Lambda = 0."""
    p = meshgen.problem("kuhn_m2_k1")
    a = meshgen.lognormal_field(p.nE, 4)
    f0, c = 1.7, 0.4
    r = oracle.pipeline(p.coord, p.tet, a, c, lambda x: np.full(x.shape[0], f0),
                        lambda x: np.full(x.shape[0], f0 / c))
    assert np.abs(r["rhs"]).max() <= 1e-13 * r["rhs_abs"].max()
    assert np.abs(r["lam"]).max() <= 1e-11
    assert np.allclose(r["U"], f0 / c, rtol=1e-12, atol=0)


def test_csr_structure():
    p = meshgen.problem("kuhn_m2_k1")
    r = oracle.pipeline(p.coord, p.tet, p.a, p.c, p.f, do_solve=False)
    fc, csr = r["fc"], r["csr"]
    rowptr, colind, vals = csr["rowptr"], csr["colind"], r["values"]
    nF, nE = fc["nF"], p.nE
    assert csr["L"] == nF                                     # all faces Dirichlet or interior
    assert rowptr[-1] == nF + 12 * nE
    deg = 1 + (fc["face_tet"][:, 1] >= 0)
    assert np.array_equal(np.diff(rowptr), 1 + 3 * deg)
    import scipy.sparse as sp
    H = sp.csr_matrix((vals, colind, rowptr), shape=(nF, nF))
    assert abs(H - H.T).max() <= 1e-15 * abs(H).max()
    assert np.all(H.diagonal() > 0)
    for r_ in range(nF):
        cols = colind[rowptr[r_]:rowptr[r_ + 1]]
        assert np.all(np.diff(cols) > 0)


def test_csr_with_neumann_rows():
    p = meshgen.problem("paper_mixed", 2)
    r = oracle.pipeline(p.coord, p.tet, p.a, p.c, p.f, p.uD, p.gN, p.neumann, do_solve=False)
    fc, csr = r["fc"], r["csr"]
    fm = csr["face_mult"]
    # nnz = L + sum_T m_T (m_T - 1), m_T = number of non-Neumann faces of T
    mT = (fm[fc["tet_face"] & 0x7FFFFFFF] >= 0).sum(axis=1)
    assert csr["rowptr"][-1] == csr["L"] + int((mT * (mT - 1)).sum())


# --------------------------------------------------------------------------
# Table 4: a priori error rates for u = x^2 y^2 z^2 with mixed conditions
# --------------------------------------------------------------------------
def error_norms(p, r):
    """||u - u_h||_Y (mesh-dependent norm of Section 4) and ||kappa - kappa_h||_h
    (Eq. eMnorm), kappa = grad u . nu_T and kappa_h = sigma_k lambda_F on faces
    outside Gamma_N."""
    coord, tet = p.coord, p.tet.astype(np.int64)
    P = coord[tet]                                               # (nE, 4, 3)
    E = P[:, 1:] - P[:, :1]                                      # rows e1, e2, e3
    Einv = np.linalg.inv(E)                                      # columns: grad lambda_1..3
    G = np.empty((tet.shape[0], 4, 3))
    G[:, 1:] = np.transpose(Einv, (0, 2, 1))
    G[:, 0] = -G[:, 1:].sum(axis=1)
    vol = np.abs(np.linalg.det(E)) / 6
    edges = np.array([[0, 1], [0, 2], [0, 3], [1, 2], [1, 3], [2, 3]])
    h = np.linalg.norm(P[:, edges[:, 0]] - P[:, edges[:, 1]], axis=2).max()
    U = r["U"]
    bary, w = tet_rule(8)
    X = np.einsum("qi,tid->tqd", bary, P)
    e = meshgen.x2y2z2_solution(X) - np.einsum("qi,ti->tq", bary, U)
    ge = meshgen.x2y2z2_grad(X) - np.einsum("ti,tid->td", U, G)[:, None, :]
    l2 = (vol[:, None] * w[None, :] * e * e).sum()
    h1 = (vol[:, None] * w[None, :] * (ge * ge).sum(axis=2)).sum()
    errY = np.sqrt(h1 + l2 / h ** 2)
    fc, fm = r["fc"], r["csr"]["face_mult"]
    tb, tw = tri_rule(6)
    acc = 0.0
    for k in range(4):
        F = fc["tet_face"][:, k] & 0x7FFFFFFF
        sig = np.where(fc["tet_face"][:, k] < 0, -1.0, 1.0)
        l = fm[F]
        keep = l >= 0
        nu = -G[:, OPP[k]] / np.linalg.norm(G[:, OPP[k]], axis=1, keepdims=True)
        V = P[:, list(LFACE[k])]                                  # (nE, 3, 3)
        Xf = np.einsum("qi,tid->tqd", tb, V)
        kap = np.einsum("tqd,td->tq", meshgen.x2y2z2_grad(Xf), nu)
        kh = np.where(keep, sig * r["lam"][np.where(keep, l, 0)], 0.0)
        area = 0.5 * np.linalg.norm(np.cross(V[:, 2] - V[:, 0], V[:, 1] - V[:, 0]), axis=1)
        d = (kap - kh[:, None]) ** 2
        acc += (keep * area * (d * tw[None, :]).sum(axis=1)).sum()
    errh = np.sqrt(h * acc)
    return errY, errh


def _rates(levels):
    eY, eh = [], []
    for lv in levels:
        p = meshgen.problem("paper_mixed", lv)
        r = oracle.pipeline(p.coord, p.tet, p.a, p.c, p.f, p.uD, p.gN, p.neumann)
        y, hh = error_norms(p, r)
        eY.append(y)
        eh.append(hh)
    eY, eh = np.array(eY), np.array(eh)
    return eY, eh, np.log2(eY[:-1] / eY[1:]), np.log2(eh[:-1] / eh[1:])


def _check_rates(golden_dir, levels, eY, eh, rY, rh):
    tab = np.loadtxt(f"{golden_dir}/table4_errors.txt")
    # first order in both norms (Table 4: 0.97-1.00 and 0.93-0.95); the
    # pre-asymptotic Y-rate approaches 1 from above, the h-rate from below
    assert np.all((rY > 0.95) & (rY < 1.15)), rY
    assert np.all(np.diff(rY) < 0), rY
    assert np.all((rh > 0.8) & (rh < 1.05)), rh
    assert np.all(np.diff(rh) > 0), rh
    # magnitudes: within a factor 4 of the paper's values (its norm quadrature
    # and its h are not stated)
    idx = [lv - 1 for lv in levels]
    assert np.all(np.abs(np.log(eY / tab[idx, 1])) < np.log(4.0))
    assert np.all(np.abs(np.log(eh / tab[idx, 3])) < np.log(4.0))


def test_table4_rates(golden_dir):
    levels = (1, 2, 3)
    _check_rates(golden_dir, levels, *_rates(levels))


@pytest.mark.slow
def test_table4_rates_level4(golden_dir):
    levels = (1, 2, 3, 4)
    _check_rates(golden_dir, levels, *_rates(levels))
