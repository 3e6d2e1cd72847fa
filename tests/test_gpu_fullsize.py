"""Parity at the full workload sizes, in the launch configuration bench.py
times (the same entry points and kernels, grids sized by the element count).

- lognormal_3m (3,359,232 tets) and jitter_checker_18m (17,915,904 tets):
  connectivity and CSR pattern compared bit-exactly with the oracle over the
  whole mesh;
- H rows and rhs entries of 2000 sampled faces, and the recovery of 2000
  sampled elements, compared with the oracle's per-element evaluation;
- properties that hold at any size: H symmetric with a positive diagonal,
  nnz = nF + 12 nE for an all-Dirichlet mesh, 12 m^2 4^k boundary faces.
"""
import numpy as np
import pytest

import meshgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

VAL_RTOL = 1e-12
NSAMPLE = 2000


@pytest.fixture(scope="module")
def ph():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2509_11133_gb300 as ph
    from paper_2509_11133_gb300 import build
    build.build()
    ph.load()
    return ph


def _host(t):
    return t.cpu().numpy()


def run_full(ph, p):
    dev = torch.device("cuda")
    mesh = ph.Mesh(torch.as_tensor(p.coord, device=dev), torch.as_tensor(p.tet, device=dev))
    fc = {k: _host(v) for k, v in mesh.faces().items()}
    f = np.asarray(p.f(fc["face_centroid"]), np.float64)
    rowptr, colind = mesh.csr_pattern()
    a_d, f_d = torch.as_tensor(p.a, device=dev), torch.as_tensor(f, device=dev)
    values, rhs, factor = mesh.assemble(a_d, p.c, f_d, factor=True)
    lam = np.random.default_rng(3).standard_normal(mesh.L)
    lam_d = torch.as_tensor(lam, device=dev)
    u = mesh.recover(a_d, p.c, f_d, lam_d)
    uf = mesh.recover_factored(factor, p.c, f_d, lam_d)
    mesh.check()
    out = dict(info=dict(mesh.info), fc=fc, f=f, lam=lam, rowptr=_host(rowptr), colind=_host(colind),
               values=_host(values), rhs=_host(rhs), U=_host(u), U_factored=_host(uf))
    mesh.close()
    return out


def check_connectivity(p, g):
    o = oracle.faces(p.tet, p.nC)
    for k in ("tet_face", "face_tet", "face_vtx", "face_kind"):
        assert np.array_equal(g["fc"][k], o[k]), k
    fm, L = oracle.multipliers(o["face_kind"])
    assert np.array_equal(g["fc"]["face_mult"], fm)
    rowptr, colind = oracle.csr_pattern(o["tet_face"], fm, L)
    assert np.array_equal(g["rowptr"], rowptr)
    assert np.array_equal(g["colind"], colind)


def element_inputs(p, g, t):
    tf = g["fc"]["tet_face"][t]
    F = tf & 0x7FFFFFFF
    sig = np.where(tf < 0, -1, 1)
    return p.coord[p.tet[t]], g["f"][F], sig, F


def check_sampled_rows(p, g, rng):
    """Rows of H and rhs entries of sampled faces, rebuilt from the oracle's
    element blocks of the face's one or two tets."""
    fc, rowptr, colind = g["fc"], g["rowptr"], g["colind"]
    faces = rng.choice(g["info"]["nF"], NSAMPLE, replace=False)
    fm = fc["face_mult"]
    for F in faces:
        l = fm[F]
        row = {}
        rhs, rhs_abs = 0.0, 0.0
        for T in fc["face_tet"][F]:
            if T < 0:
                continue
            P, f4, sig, Fk = element_inputs(p, g, T)
            S, gv = oracle.tet_local(P, p.a[T], p.c, f4, sig)
            k = int(np.nonzero(Fk == F)[0][0])
            for m in range(4):
                row[fm[Fk[m]]] = row.get(fm[Fk[m]], 0.0) + S[k, m]
            rhs += gv[k]
            rhs_abs += abs(gv[k])
        lo, hi = rowptr[l], rowptr[l + 1]
        assert sorted(row) == list(colind[lo:hi])
        want = np.array([row[c] for c in colind[lo:hi]])
        got = g["values"][lo:hi]
        assert np.all(np.abs(got - want) <= VAL_RTOL * np.abs(want)), (F, got, want)
        assert abs(g["rhs"][l] - rhs) <= 1e-12 * rhs_abs + 1e-300


def check_sampled_recovery(p, g, rng):
    tets = rng.choice(p.nE, NSAMPLE, replace=False)
    fm = g["fc"]["face_mult"]
    for t in tets:
        P, f4, sig, Fk = element_inputs(p, g, t)
        U = oracle.tet_recover(P, p.a[t], p.c, f4, sig, g["lam"][fm[Fk]])
        assert np.all(np.abs(g["U"][t] - U) <= 1e-12 * np.abs(U).max())
        assert np.all(np.abs(g["U_factored"][t] - U) <= 1e-12 * np.abs(U).max())


def check_properties(p, g, m, k):
    import scipy.sparse as sp
    info = g["info"]
    nF, nE = info["nF"], info["nE"]
    assert info["L"] == nF and info["nnz"] == nF + 12 * nE
    assert info["nF_dirichlet"] == 12 * m * m * 4 ** k
    H = sp.csr_matrix((g["values"], g["colind"], g["rowptr"]), shape=(nF, nF))
    D = H - H.T
    assert abs(D).max() <= 1e-12 * abs(H).max()
    assert np.all(H.diagonal() > 0)


@pytest.fixture(scope="module")
def lognormal(ph):
    p = meshgen.problem("lognormal_3m")
    return p, run_full(ph, p)


@pytest.fixture(scope="module")
def jitter(ph):
    p = meshgen.problem("jitter_checker_18m")
    return p, run_full(ph, p)


def test_lognormal_3m_connectivity(lognormal):
    check_connectivity(*lognormal)


def test_lognormal_3m_sampled_rows_and_recovery(lognormal):
    p, g = lognormal
    rng = np.random.default_rng(11)
    check_sampled_rows(p, g, rng)
    check_sampled_recovery(p, g, rng)


def test_lognormal_3m_properties(lognormal):
    check_properties(*lognormal, m=3, k=4)


def test_jitter_checker_18m_connectivity(jitter):
    check_connectivity(*jitter)


def test_jitter_checker_18m_sampled_rows_and_recovery(jitter):
    p, g = jitter
    rng = np.random.default_rng(12)
    check_sampled_rows(p, g, rng)
    check_sampled_recovery(p, g, rng)


def test_jitter_checker_18m_properties(jitter):
    check_properties(*jitter, m=1, k=6)
