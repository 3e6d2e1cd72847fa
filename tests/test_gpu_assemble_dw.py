"""The double-word assembly variant (ph_assemble_dw) against the oracle, at the
tolerances of the fp64 path: H entrywise relative 1e-12, rhs within 1e-12 of
the sum of its addends' magnitudes, connectivity untouched.  Also: the element
factor and H agree with the fp64 path to ~1e-13 (both approximate the same
exact values), recovery from the variant's factor matches the oracle, and
elements outside the double-word range (a reaction term that dominates, tiny
coefficients) take the fp64 fallback and still match.

Cases: every mesh of the fp64 parity tests (Listing 1 with and without mixed
boundary data, Kuhn cubes, shuffled and degree-sorted meshes, the lognormal
and jittered checkerboard workloads at small size), a soup of random
isolated elements of graded flatness (slivers included) with diffusion- and
reaction-dominated coefficients.  The full-size workloads (every value of the
3.36M- and 17.9M-tet meshes) are checked in test_gpu_fullsize.py."""
import numpy as np
import pytest

import meshgen
import oracle
from tests.test_gpu_parity import CASES, assert_values_close, cu, host, make_case, oracle_face_data, run_oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ph():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2509_11133_gb300 as ph
    from paper_2509_11133_gb300 import build
    build.build()
    ph.load()
    return ph


def run_both(ph, p, a=None, c=None):
    """fp64 and double-word assembly of problem p on one mesh."""
    a = p.a if a is None else a
    c = p.c if c is None else c
    mesh = ph.Mesh(cu(p.coord, torch.float64), cu(p.tet, torch.int32),
                   cu(p.neumann, torch.int32) if p.neumann.size else None)
    fc = {k: host(v) for k, v in mesh.faces().items()}
    cen = fc["face_centroid"]
    f = np.asarray(p.f(cen), np.float64)
    uD = None if p.uD is None else np.asarray(p.uD(cen), np.float64)
    gN = None if p.gN is None else np.asarray(p.gN(cen), np.float64)
    opt = lambda x: None if x is None else cu(x, torch.float64)
    out = {"mesh": mesh, "fc": fc, "f": f, "uD": uD, "gN": gN}
    for variant in ("f64", "dw"):
        v, r, fa = mesh.assemble(cu(a, torch.float64), c, cu(f, torch.float64), opt(uD), opt(gN), factor=True,
                                 variant=variant)
        out[variant] = {"values": host(v), "rhs": host(r), "factor": host(fa), "factor_d": fa}
    mesh.check()
    return out


def assert_close_to_f64(g):
    v64, vdw = g["f64"]["values"], g["dw"]["values"]
    assert np.all(np.abs(vdw - v64) <= 1e-13 * np.abs(v64))
    f64, fdw = g["f64"]["factor"], g["dw"]["factor"]
    scale = np.abs(f64).max(axis=1, keepdims=True)
    assert np.all(np.abs(fdw - f64) <= 1e-13 * scale)


@pytest.mark.parametrize("name", CASES)
def test_dw_assembly_parity(ph, name):
    p = make_case(name)
    g = run_both(ph, p)
    o = run_oracle(p)
    assert_values_close({"values": g["dw"]["values"], "rhs": g["dw"]["rhs"]}, o)
    assert_close_to_f64(g)
    g["mesh"].close()


@pytest.mark.parametrize("name", ["sin_kuhn", "mixed_l2", "lognormal_small", "jitter_checker_small"])
def test_dw_factor_recovery_parity(ph, name):
    p = make_case(name)
    g = run_both(ph, p)
    fc = oracle.faces(p.tet, p.nC, p.neumann)
    fm, L = oracle.multipliers(fc["face_kind"])
    lam = np.random.default_rng(2).standard_normal(L)
    u = g["mesh"].recover_factored(g["dw"]["factor_d"], p.c, cu(g["f"], torch.float64), cu(lam, torch.float64),
                                   None if g["gN"] is None else cu(g["gN"], torch.float64))
    fo, _, gNo = oracle_face_data(p, fc)
    Uo = oracle.recover(p.coord, p.tet, fc, fm, p.a, p.c, fo, lam, gNo)
    scale = np.abs(Uo).max(axis=1, keepdims=True)
    assert np.all(np.abs(host(u) - Uo) <= 1e-12 * scale)
    g["mesh"].close()


def element_soup(n, seed, flat=(1e-3, 1.0)):
    """n isolated elements (4 own vertices each, every face a boundary face):
    regular tetrahedra, randomly rotated and jittered by 15% of their size,
    whose vertex 3 is then pulled towards the plane of the other three,
    leaving a height ratio log-uniform in `flat` (slivers at the low end:
    |det E|^2 / (g00 g11 g22) ~ 0.5 ratio^2), sizes over three decades."""
    rng = np.random.default_rng(seed)
    base = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], float)
    Qr, _ = np.linalg.qr(rng.standard_normal((n, 3, 3)))
    P = np.einsum("vj,nij->nvi", base, Qr) + 0.15 * rng.standard_normal((n, 4, 3))
    c3 = (P[:, 0] + P[:, 1] + P[:, 2]) / 3
    nrm = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    off = np.einsum("ij,ij->i", P[:, 3] - c3, nrm)
    keep = 10.0 ** rng.uniform(np.log10(flat[0]), np.log10(flat[1]), n)
    P[:, 3] = P[:, 3] - (off * (1 - keep))[:, None] * nrm
    P *= (10.0 ** rng.uniform(-2, 1, n))[:, None, None]
    P += rng.uniform(-1, 1, (n, 1, 3))
    coord = P.reshape(-1, 3)
    tet = np.arange(4 * n, dtype=np.int32).reshape(n, 4)
    return coord, tet


def assert_soup_close(p, g, o, which):
    """assert_values_close with a report of the worst element on failure
    (in a soup, element t owns H entries 16t..16t+15)."""
    v, w = g[which]["values"], o["values"]
    err = np.abs(v - w) / np.abs(w)
    if not np.all(err <= 1e-12):
        t = int(np.argmax(err)) // 16
        P = p.coord[p.tet[t]]
        E = P[1:] - P[0]
        det = abs(np.linalg.det(E))
        ge = np.einsum("ij,ij->i", E, E)
        print(f"{which}: worst error {err.max():.3e} at element {t}: a={p.a[t]:.3e} c={p.c} "
              f"flatness det^2/prod(g)={det ** 2 / ge.prod():.3e} c h^2/a={p.c * ge.max() / p.a[t]:.3e}")
    assert_values_close({"values": v, "rhs": g[which]["rhs"]}, o)


@pytest.mark.parametrize("c", [1e-2, 1.0])
def test_dw_element_soup_against_oracle(ph, c):
    """Diffusion-dominated elements (a >= 1, sizes up to ~10, c <= 1) of any
    shape, slivers included: both assemblies within 1e-12 of the oracle (the
    flat ones take the fp64 path in the variant)."""
    coord, tet = element_soup(4000, 11 + int(c * 100))
    a = 10.0 ** np.random.default_rng(5).uniform(0, 4, tet.shape[0])
    p = meshgen.Problem("soup", coord, tet, a, c, lambda x: meshgen.sin_source(x))
    g = run_both(ph, p)
    o = run_oracle(p)
    assert_soup_close(p, g, o, "f64")
    assert_soup_close(p, g, o, "dw")
    g["mesh"].close()


def test_dw_fallback_elements(ph):
    """A reaction term that dominates the element (c h^2 >> a) takes the fp64
    path: every element of this soup (well shaped: the fp64 split form itself
    needs G_e well conditioned when c h^2 >> a) does, so the result is the
    fp64 path's bit for bit, and it matches the oracle."""
    coord, tet = element_soup(2000, 3, flat=(0.3, 1.0))
    P = coord[tet]
    h2 = np.max(np.sum((P[:, 1:] - P[:, :1]) ** 2, axis=2), axis=1)
    # c h^2 / a in [5, 10]: past the double-word rule, and short of the regime
    # (c h^2 >> a) where the fp64 split form itself loses the rhs's last digits
    a = 5.0 * h2 / np.random.default_rng(9).uniform(5, 10, tet.shape[0])
    p = meshgen.Problem("fallback", coord, tet, a, 5.0, lambda x: meshgen.sin_source(x))
    g = run_both(ph, p)
    o = run_oracle(p)
    assert_soup_close(p, g, o, "dw")
    for k in ("values", "rhs", "factor"):
        assert np.array_equal(g["dw"][k].view(np.uint64), g["f64"][k].view(np.uint64)), k
    g["mesh"].close()


def test_dw_large_coefficients(ph):
    """a in [1e8, 1e14] (the oracle's binary128 local solve stays accurate up
    to a/(c h^2) ~ 1e20): the condensation kernel's scale 1/a travels as a
    separate power of two; the double-word path matches the oracle."""
    coord, tet = element_soup(1000, 4, flat=(1e-2, 1.0))  # the flattest take the fp64 path
    a = 10.0 ** np.random.default_rng(10).uniform(8, 14, tet.shape[0])
    p = meshgen.Problem("large", coord, tet, a, 0.5, lambda x: meshgen.sin_source(x))
    g = run_both(ph, p)
    o = run_oracle(p)
    assert_soup_close(p, g, o, "f64")
    assert_soup_close(p, g, o, "dw")
    assert_close_to_f64(g)
    g["mesh"].close()


def dw_mesh_run(ph, p, lam_seed=2):
    """A mesh from ph_mesh_create_dw: its connectivity, areas, ph_assemble_dw
    output and recovery from its factor."""
    neu = cu(p.neumann, torch.int32) if p.neumann.size else None
    mesh = ph.Mesh(cu(p.coord, torch.float64), cu(p.tet, torch.int32), neu, geometry="dw")
    fc = {k: host(v) for k, v in mesh.faces().items()}
    cen = fc["face_centroid"]
    f = np.asarray(p.f(cen), np.float64)
    uD = None if p.uD is None else np.asarray(p.uD(cen), np.float64)
    gN = None if p.gN is None else np.asarray(p.gN(cen), np.float64)
    opt = lambda x: None if x is None else cu(x, torch.float64)
    v, r, fa = mesh.assemble(cu(p.a, torch.float64), p.c, cu(f, torch.float64), opt(uD), opt(gN), factor=True,
                             variant="dw")
    lam = np.random.default_rng(lam_seed).standard_normal(mesh.L)
    u = mesh.recover_factored(fa, p.c, cu(f, torch.float64), cu(lam, torch.float64), opt(gN))
    rowptr, colind = mesh.csr_pattern()
    mesh.check()
    out = dict(mesh=mesh, fc=fc, f=f, uD=uD, gN=gN, values=host(v), rhs=host(r), U=host(u), lam=lam,
               rowptr=host(rowptr), colind=host(colind))
    return out


@pytest.mark.parametrize("name", CASES)
def test_dw_mesh_parity(ph, name):
    """ph_mesh_create_dw + ph_assemble_dw + ph_recover_factored against the
    oracle: connectivity and CSR pattern bit-exact, H and rhs at 1e-12,
    recovery at 1e-12; face areas equal to the fp64 build's."""
    from tests.test_gpu_parity import assert_connectivity_equal
    p = make_case(name)
    g = dw_mesh_run(ph, p)
    o = run_oracle(p)
    assert_connectivity_equal(g, o)
    assert_values_close(g, o)
    Uo = oracle.recover(p.coord, p.tet, o["fc"], o["csr"]["face_mult"], p.a, p.c, o["f"], g["lam"], o["gN"])
    assert np.all(np.abs(g["U"] - Uo) <= 1e-12 * np.abs(Uo).max(axis=1, keepdims=True))
    q = ph.Mesh(cu(p.coord, torch.float64), cu(p.tet, torch.int32),
                cu(p.neumann, torch.int32) if p.neumann.size else None)
    a64 = host(q.faces()["face_area"])
    assert np.array_equal(g["fc"]["face_area"], a64)
    q.close()
    g["mesh"].close()


def test_dw_mesh_flat_elements_fall_back(ph):
    """Flat elements of a double-word mesh get their fp64 geometry recomputed
    from the vertices for the fp64 condensation kernel: still the oracle's
    values."""
    coord, tet = element_soup(3000, 8, flat=(1e-3, 1.0))
    a = 10.0 ** np.random.default_rng(12).uniform(0, 4, tet.shape[0])
    p = meshgen.Problem("soup", coord, tet, a, 0.3, lambda x: meshgen.sin_source(x))
    g = dw_mesh_run(ph, p)
    o = run_oracle(p)
    assert_soup_close(p, {"dw": g}, o, "dw")
    g["mesh"].close()


def test_dw_mesh_refuses_fp64_record_entry_points(ph):
    p = make_case("sin_kuhn")
    m = ph.Mesh(cu(p.coord, torch.float64), cu(p.tet, torch.int32), geometry="dw")
    a = cu(p.a, torch.float64)
    f = cu(np.ones(m.nF), torch.float64)
    for call in (lambda: m.assemble(a, 1.0, f), lambda: m.recover(a, 1.0, f, cu(np.zeros(m.L), torch.float64)),
                 lambda: ph.Batch([m])):
        with pytest.raises(ph.PHError) as e:
            call()
        assert e.value.name == "PH_ERR_ARG"
    m.close()


@pytest.mark.parametrize("name", ["sin_kuhn", "mixed_l2", "lognormal_small", "jitter_checker_small", "shuffled"])
def test_dw_recovery_parity(ph, name):
    """ph_recover_factored_dw, from the fp64 factor and from the double-word
    factor, against the oracle's recovery with a random Lambda: within 1e-12
    of each element's largest |U| plus 8 ulp of the magnitude of the terms the
    recovery sums (z' and its sum stay fp64; the pairs carry the smaller
    (Qf z')/3); the fp64 path's factor recovery printed beside it."""
    from tests.test_gpu_fullsize import EPS64, U_TERM_ULPS, recovery_terms
    p = make_case(name)
    g = run_both(ph, p)
    fc = oracle.faces(p.tet, p.nC, p.neumann)
    fm, L = oracle.multipliers(fc["face_kind"])
    lam = np.random.default_rng(2).standard_normal(L)
    fo, _, gNo = oracle_face_data(p, fc)
    Uo = oracle.recover(p.coord, p.tet, fc, fm, p.a, p.c, fo, lam, gNo)
    gN = None if g["gN"] is None else cu(g["gN"], torch.float64)
    args = (p.c, cu(g["f"], torch.float64), cu(lam, torch.float64), gN)
    scale = np.abs(Uo).max(axis=1)
    terms = recovery_terms(p, {"fc": fc, "f": fo, "gN": gNo, "lam": lam, "csr": {"face_mult": fm}})
    bar = 1e-12 * scale + U_TERM_ULPS * EPS64 * terms
    for fac in ("f64", "dw"):
        for variant in ("f64", "dw"):
            u = host(g["mesh"].recover_factored(g[fac]["factor_d"], *args, variant=variant))
            e = np.abs(u - Uo).max(axis=1)
            print(f"{name}: factor {fac}, recovery {variant}: worst {float((e / scale).max()):.3g} of max|U|")
            assert np.all(e <= bar), (fac, variant)
    g["mesh"].close()
