"""Parity at the full workload sizes, in the launch configuration bench.py
times (the same entry points and kernels, grids sized by the element count).

- lognormal_3m (3,359,232 tets) and jitter_checker_18m (17,915,904 tets):
  connectivity, CSR pattern and face centroids compared bit-exactly with the
  oracle over the whole mesh;
- every H value, rhs entry and recovered element value compared with the
  oracle's assembly and recovery of the whole mesh (its element loops on all
  host cores, bit-identical to one thread), for the fp64 path and for the
  double-word variant;
- H rows and rhs entries of 2000 sampled faces, and the recovery of 2000
  sampled elements, also compared with the oracle's per-element entry points;
- properties that hold at any size: H symmetric with a positive diagonal,
  nnz = nF + 12 nE for an all-Dirichlet mesh, 12 m^2 4^k boundary faces.

Every oracle input comes from the workload generator, a seeded generator or
the oracle itself (its own faces and face centroids); the GPU side evaluates
f at the centroids the library exports.
"""
import numpy as np
import pytest

import meshgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

VAL_RTOL = 1e-12
NSAMPLE = 2000
LAM_SEED = 3


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


_ORACLE = {}


def oracle_data(p):
    """The oracle's faces, multipliers, CSR pattern, face centroids and f, and
    its assembly and recovery (seeded random Lambda) of the whole mesh; kept
    for the module's next test on the same workload."""
    if p.name not in _ORACLE:
        _ORACLE.clear()
        fc = oracle.faces(p.tet, p.nC)
        fm, L = oracle.multipliers(fc["face_kind"])
        rowptr, colind = oracle.csr_pattern(fc["tet_face"], fm, L)
        csr = dict(face_mult=fm, L=L, rowptr=rowptr, colind=colind)
        cen = oracle.face_centroids(p.coord, fc["face_vtx"])
        f = np.asarray(p.f(cen), np.float64)
        values, rhs, rhs_abs = oracle.assemble(p.coord, p.tet, fc, csr, p.a, p.c, f)
        lam = np.random.default_rng(LAM_SEED).standard_normal(L)
        U = oracle.recover(p.coord, p.tet, fc, fm, p.a, p.c, f, lam)
        _ORACLE[p.name] = dict(fc=fc, csr=csr, cen=cen, f=f, values=values, rhs=rhs, rhs_abs=rhs_abs, lam=lam,
                               U=U)
    return _ORACLE[p.name]


def run_full(ph, p, geometry="f64", variant="f64"):
    """The full-size path on the GPU: mesh build, assembly with the element
    factor, recovery with and (fp64 record) without the factor; variant "dw"
    assembles with ph_assemble_dw and recovers with ph_recover_factored_dw."""
    dev = torch.device("cuda")
    mesh = ph.Mesh(torch.as_tensor(p.coord, device=dev), torch.as_tensor(p.tet, device=dev), geometry=geometry)
    fc = {k: _host(v) for k, v in mesh.faces().items()}
    f = np.asarray(p.f(fc["face_centroid"]), np.float64)
    rowptr, colind = mesh.csr_pattern()
    a_d, f_d = torch.as_tensor(p.a, device=dev), torch.as_tensor(f, device=dev)
    values, rhs, factor = mesh.assemble(a_d, p.c, f_d, factor=True, variant=variant)
    lam = np.random.default_rng(LAM_SEED).standard_normal(mesh.L)
    lam_d = torch.as_tensor(lam, device=dev)
    u = mesh.recover(a_d, p.c, f_d, lam_d) if geometry == "f64" else None
    uf = mesh.recover_factored(factor, p.c, f_d, lam_d, variant=variant)
    mesh.check()
    out = dict(info=dict(mesh.info), fc=fc, rowptr=_host(rowptr), colind=_host(colind), values=_host(values),
               rhs=_host(rhs), U=None if u is None else _host(u), U_factored=_host(uf))
    mesh.close()
    return out


def check_connectivity(p, g):
    o = oracle_data(p)
    for k in ("tet_face", "face_tet", "face_vtx", "face_kind"):
        assert np.array_equal(g["fc"][k], o["fc"][k]), k
    assert np.array_equal(g["fc"]["face_mult"], o["csr"]["face_mult"])
    assert np.array_equal(g["rowptr"], o["csr"]["rowptr"])
    assert np.array_equal(g["colind"], o["csr"]["colind"])
    assert np.array_equal(g["fc"]["face_centroid"], o["cen"])


def recovery_terms(p, o):
    """Per element, the magnitude of the terms the recovery sums,
    (1/(c|T|)) sum_m (|T|/4 |f_m| + |F_m| |Lambda_m or g_N,m|): the scale of
    the rounding in U = z'sum/(c|T|) - 3 (Qf/9) z' (numpy, from the mesh; o
    holds the oracle's faces, face data, multipliers and Lambda, and g_N when
    the mesh has Neumann faces)."""
    P = p.coord[p.tet]
    vol = np.abs(np.linalg.det(P[:, 1:] - P[:, :1])) / 6.0
    x = p.coord[o["fc"]["face_vtx"]]
    area = 0.5 * np.linalg.norm(np.cross(x[:, 1] - x[:, 0], x[:, 2] - x[:, 0]), axis=1)
    F = o["fc"]["tet_face"] & 0x7FFFFFFF
    l = o["csr"]["face_mult"][F]
    side = np.abs(o["lam"][np.maximum(l, 0)])
    if o.get("gN") is not None:
        side = np.where(l >= 0, side, np.abs(o["gN"][F]))
    z = vol[:, None] / 4 * np.abs(o["f"][F]) + area[F] * side
    return z.sum(axis=1) / (p.c * vol)


U_TERM_ULPS = 8
EPS64 = 2.0 ** -53


def check_all_values(p, g, what):
    """Every H value (1e-12 of itself: an off-diagonal entry has one addend,
    the diagonal's two addends are positive), every rhs entry (1e-12 of the
    sum of its addends' magnitudes) and every recovered value, against the
    oracle's whole-mesh assembly and recovery.

    The recovery U = z'sum/(c|T|) - 3 (Qf/9) z' with a random Lambda (not a
    solution of the system) cancels: at some elements its terms are 1e6-1e7
    times the largest |U| (on the 17.9M-tet mesh, 7e7).  An fp64 evaluation
    is then exact only to the rounding of the terms, so the bar is 1e-12 of
    the element's largest |U| plus 8 ulp of the terms' magnitudes
    (recovery_terms); the worst error measured is under one ulp of the terms,
    for the fp64 path and the double-word variant alike (both printed)."""
    o = oracle_data(p)
    err = np.abs(g["values"] - o["values"])
    ratio = float((err / np.abs(o["values"])).max())
    bad = int(np.count_nonzero(err > VAL_RTOL * np.abs(o["values"])))
    rerr = float((np.abs(g["rhs"] - o["rhs"]) / np.maximum(o["rhs_abs"], 1e-300)).max())
    scale = np.abs(o["U"]).max(axis=1)
    terms = recovery_terms(p, o)
    bar = VAL_RTOL * scale + U_TERM_ULPS * EPS64 * terms
    over = {}
    for k in ("U", "U_factored"):
        if g[k] is None:
            continue
        e = np.abs(g[k] - o["U"]).max(axis=1)
        t = int(np.argmax(e / scale))
        over[k] = int(np.count_nonzero(e > bar))
        big = e > VAL_RTOL * scale  # the cancelling elements
        ulps = float((e[big] / (EPS64 * terms[big])).max()) if big.any() else 0.0
        print(f"{p.name} {what} {k}: worst {e[t] / scale[t]:.3g} of max|U| at element {t}, whose terms are "
              f"{terms[t] / scale[t]:.3g} x max|U|; {int(big.sum())} of {e.size} elements above 1e-12 max|U|, "
              f"at most {ulps:.3g} ulp of their terms; {over[k]} above the bar")
    print(f"{p.name} {what}: {o['values'].size} H values, worst relative error {ratio:.3g} ({bad} above "
          f"{VAL_RTOL:g}); rhs worst {rerr:.3g} of the addends' magnitudes")
    assert bad == 0, (bad, ratio)
    assert rerr <= 1e-12
    assert all(n == 0 for n in over.values()), over


def element_inputs(p, o, t):
    tf = o["fc"]["tet_face"][t]
    F = tf & 0x7FFFFFFF
    sig = np.where(tf < 0, -1, 1)
    return p.coord[p.tet[t]], o["f"][F], sig, F


def check_sampled_rows(p, g, rng):
    """Rows of H and rhs entries of sampled faces, rebuilt from the oracle's
    element blocks of the face's one or two tets."""
    o = oracle_data(p)
    fc, fm = o["fc"], o["csr"]["face_mult"]
    rowptr, colind = g["rowptr"], g["colind"]
    for F in rng.choice(g["info"]["nF"], NSAMPLE, replace=False):
        l = fm[F]
        row = {}
        rhs, rhs_abs = 0.0, 0.0
        for T in fc["face_tet"][F]:
            if T < 0:
                continue
            P, f4, sig, Fk = element_inputs(p, o, T)
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


def check_sampled_recovery(p, g, rng, u_rtol=1e-12):
    o = oracle_data(p)
    fm = o["csr"]["face_mult"]
    for t in rng.choice(p.nE, NSAMPLE, replace=False):
        P, f4, sig, Fk = element_inputs(p, o, t)
        U = oracle.tet_recover(P, p.a[t], p.c, f4, sig, o["lam"][fm[Fk]])
        for k in ("U", "U_factored"):
            if g[k] is not None:
                assert np.all(np.abs(g[k][t] - U) <= u_rtol * np.abs(U).max()), (k, t)


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


def test_lognormal_3m_all_values(lognormal):
    check_all_values(*lognormal, "f64")


def test_lognormal_3m_sampled_rows_and_recovery(lognormal):
    p, g = lognormal
    rng = np.random.default_rng(11)
    check_sampled_rows(p, g, rng)
    check_sampled_recovery(p, g, rng)


def test_lognormal_3m_properties(lognormal):
    check_properties(*lognormal, m=3, k=4)


def test_lognormal_3m_double_word_variant(ph, lognormal):
    """ph_assemble_dw on the fp64 record of the 3.36M-tet mesh: every H value,
    rhs entry and value recovered from its element factor by
    ph_recover_factored_dw, at the fp64 path's bars."""
    p, _ = lognormal
    g = run_full(ph, p, "f64", "dw")
    g["U"] = None
    check_all_values(p, g, "dw")


def test_jitter_checker_18m_connectivity(jitter):
    check_connectivity(*jitter)


def test_jitter_checker_18m_all_values(jitter):
    check_all_values(*jitter, "f64")


def test_jitter_checker_18m_sampled_rows_and_recovery(jitter):
    p, g = jitter
    rng = np.random.default_rng(12)
    check_sampled_rows(p, g, rng)
    check_sampled_recovery(p, g, rng)


def test_jitter_checker_18m_properties(jitter):
    check_properties(*jitter, m=1, k=6)


def test_jitter_checker_18m_double_word_mesh(ph, jitter):
    """ph_mesh_create_dw + ph_assemble_dw + ph_recover_factored_dw on the
    17.9M-tet jittered mesh, the variant bench.py times: connectivity
    bit-exact, every H value, rhs entry and recovered value at the fp64
    path's bars."""
    p, _ = jitter
    g = run_full(ph, p, "dw", "dw")
    check_connectivity(p, g)
    check_all_values(p, g, "dw mesh")
