"""Parity of the CUDA library (through its C ABI) with the CPU oracle.

Connectivity and CSR pattern: bit-exact.  H values: entrywise relative 1e-12.
rhs: |gpu - oracle| <= 1e-12 * (sum of |addends|) (interior contributions of
the two tets cancel).  Recovery with a given Lambda: 1e-12 relative to the
element's largest value.  Solved Lambda and U: 2-norm relative 1e-9.
"""
import numpy as np
import pytest

import meshgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

VAL_RTOL = 1e-12
RHS_RTOL = 1e-12
SOLVE_RTOL = 1e-9


@pytest.fixture(scope="module")
def ph():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2509_11133_gb300 as ph
    from paper_2509_11133_gb300 import build
    build.build()
    ph.load()
    return ph


def cu(x, dtype):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def gpu_face_data(mesh, p):
    """Face data evaluated at the GPU-exported face centroids."""
    fc = {k: host(v) for k, v in mesh.faces().items()}
    cen = fc["face_centroid"]
    f = np.asarray(p.f(cen), np.float64)
    uD = None if p.uD is None else np.asarray(p.uD(cen), np.float64)
    gN = None if p.gN is None else np.asarray(p.gN(cen), np.float64)
    return fc, f, uD, gN


def run_gpu(ph, p, a=None, lam=None, solve=False):
    a = p.a if a is None else a
    mesh = ph.Mesh(cu(p.coord, torch.float64), cu(p.tet, torch.int32),
                   cu(p.neumann, torch.int32) if p.neumann.size else None)
    fc, f, uD, gN = gpu_face_data(mesh, p)
    rowptr, colind = mesh.csr_pattern()
    a_d, f_d = cu(a, torch.float64), cu(f, torch.float64)
    uD_d = None if uD is None else cu(uD, torch.float64)
    gN_d = None if gN is None else cu(gN, torch.float64)
    values, rhs, factor = mesh.assemble(a_d, p.c, f_d, uD_d, gN_d, factor=True)
    out = dict(mesh=mesh, fc=fc, f=f, uD=uD, gN=gN, rowptr=host(rowptr), colind=host(colind), values=host(values),
               rhs=host(rhs))
    if solve:
        x, it, rr, _ = ph.ph_solve_pcg(rowptr, colind, values, rhs, rtol=1e-13, maxit=50000)
        out.update(lam=host(x), iters=it, relres=rr)
        lam = out["lam"]
    if lam is not None:
        lam_d = cu(lam, torch.float64)
        u = mesh.recover(a_d, p.c, f_d, lam_d, gN_d)
        out["U"] = host(u)
        out["U_factored"] = host(mesh.recover_factored(factor, p.c, f_d, lam_d, gN_d))
    mesh.check()
    return out


def oracle_face_data(p, fc):
    """f, u_D and g_N at the oracle's own face centroids.  The GPU side
    evaluates them at the centroids the library exports, so each side derives
    its inputs on its own (a test checks the two sets of centroids bit for
    bit)."""
    cen = oracle.face_centroids(p.coord, fc["face_vtx"])
    f = np.asarray(p.f(cen), np.float64)
    uD = None if p.uD is None else np.asarray(p.uD(cen), np.float64)
    gN = None if p.gN is None else np.asarray(p.gN(cen), np.float64)
    return f, uD, gN


def run_oracle(p, a=None, solve=False):
    a = p.a if a is None else a
    fc = oracle.faces(p.tet, p.nC, p.neumann)
    fm, L = oracle.multipliers(fc["face_kind"])
    rowptr, colind = oracle.csr_pattern(fc["tet_face"], fm, L)
    csr = {"face_mult": fm, "L": L, "rowptr": rowptr, "colind": colind}
    f, uD, gN = oracle_face_data(p, fc)
    values, rhs, rhs_abs = oracle.assemble(p.coord, p.tet, fc, csr, a, p.c, f, uD, gN)
    out = dict(fc=fc, csr=csr, f=f, uD=uD, gN=gN, values=values, rhs=rhs, rhs_abs=rhs_abs)
    if solve:
        lam = oracle.solve(rowptr, colind, values, rhs)
        out.update(lam=lam, U=oracle.recover(p.coord, p.tet, fc, fm, a, p.c, f, lam, gN))
    return out


def assert_connectivity_equal(g, o):
    fc = g["fc"]
    assert fc["tet_face"].shape == o["fc"]["tet_face"].shape
    assert np.array_equal(fc["tet_face"], o["fc"]["tet_face"])
    assert np.array_equal(fc["face_tet"], o["fc"]["face_tet"])
    assert np.array_equal(fc["face_vtx"], o["fc"]["face_vtx"])
    assert np.array_equal(fc["face_kind"], o["fc"]["face_kind"])
    assert np.array_equal(fc["face_mult"], o["csr"]["face_mult"])
    assert np.array_equal(g["rowptr"], o["csr"]["rowptr"])
    assert np.array_equal(g["colind"], o["csr"]["colind"])


def assert_values_close(g, o):
    v, w = g["values"], o["values"]
    assert v.shape == w.shape
    err = np.abs(v - w) / np.abs(w)
    assert np.all(err <= VAL_RTOL), (err.max(), int(np.argmax(err)))
    d = np.abs(g["rhs"] - o["rhs"])
    tol = RHS_RTOL * o["rhs_abs"] + 1e-300
    assert np.all(d <= tol), float((d / tol).max())


CASES = ["listing1", "listing1_mixed", "sin_kuhn", "kuhn_m2_k1", "shuffled", "mixed_l2", "lognormal_small",
         "jitter_checker_small", "degree_sorted", "mixed_degree_sorted"]


def renumber_by_degree(coord, tet, lists=()):
    """Vertices renumbered by ascending number of incident tets, so that the
    busiest vertices are the largest ids of most of their faces: face-key
    buckets of up to 108 entries (tet and Neumann keys mixed)."""
    deg = np.bincount(tet.ravel(), minlength=coord.shape[0])
    order = np.argsort(deg, kind="stable")
    inv = np.empty_like(order)
    inv[order] = np.arange(order.size)
    return coord[order], inv[tet].astype(np.int32), [inv[l].astype(np.int32) for l in lists]


def make_case(name):
    if name == "listing1":
        coord, tet, _, _ = meshgen.listing1_mesh()
        return meshgen.Problem(name, coord, tet, np.ones(5), 1.0, lambda x: meshgen.sin_source(x))
    if name == "listing1_mixed":
        return meshgen.problem("paper_mixed", 0)
    if name == "sin_kuhn":
        return meshgen.problem("sin_kuhn")
    if name == "kuhn_m2_k1":
        return meshgen.problem("kuhn_m2_k1")
    if name == "shuffled":
        p = meshgen.problem("kuhn_m2_k1")
        coord, tet = meshgen.shuffled(p.coord, p.tet, 5)
        return meshgen.Problem(name, coord, tet, meshgen.lognormal_field(tet.shape[0], 9), 0.3, p.f)
    if name == "mixed_l2":
        return meshgen.problem("paper_mixed", 2)
    if name == "degree_sorted":
        p = meshgen.problem("kuhn_m2_k1")
        coord, tet, _ = renumber_by_degree(p.coord, p.tet)
        return meshgen.Problem(name, coord, tet, meshgen.lognormal_field(tet.shape[0], 3), 0.5, p.f)
    if name == "mixed_degree_sorted":
        p = meshgen.problem("paper_mixed", 2)
        coord, tet, (neu,) = renumber_by_degree(p.coord, p.tet, [p.neumann])
        p.coord, p.tet, p.neumann = coord, tet, neu
        return p
    if name == "lognormal_small":
        # the lognormal workload's recipe on a 3^3 cube refined twice (23,328 tets:
        # many blocks and a ragged tail)
        coord, tet = meshgen.kuhn_cube(3)
        coord, tet, _ = meshgen.refined(coord, tet, 2)
        return meshgen.Problem(name, coord, tet, meshgen.lognormal_field(tet.shape[0], 2), 0.1,
                               lambda x: meshgen.sin_source(x))
    if name == "jitter_checker_small":
        coord, tet = meshgen.kuhn_cube(1)
        coord, tet, _ = meshgen.refined(coord, tet, 3)
        coord, _ = meshgen.jitter_interior(coord, tet, 0.2, seed=3)
        return meshgen.Problem(name, coord, tet, meshgen.checkerboard_field(coord, tet), 1.0,
                               lambda x: meshgen.sin_source(x))
    raise KeyError(name)


@pytest.mark.parametrize("name", CASES)
def test_assembly_parity(ph, name):
    p = make_case(name)
    g = run_gpu(ph, p)
    o = run_oracle(p)
    # the GPU's face centroids are the oracle's (same face tuples, same formula)
    cen_o = oracle.face_centroids(p.coord, o["fc"]["face_vtx"])
    assert np.array_equal(g["fc"]["face_centroid"], cen_o)
    assert_connectivity_equal(g, o)
    assert_values_close(g, o)
    g["mesh"].close()


@pytest.mark.parametrize("name", ["sin_kuhn", "mixed_l2", "lognormal_small", "jitter_checker_small"])
def test_recovery_parity_given_lambda(ph, name):
    p = make_case(name)
    fc = oracle.faces(p.tet, p.nC, p.neumann)
    fm, L = oracle.multipliers(fc["face_kind"])
    lam = np.random.default_rng(1).standard_normal(L)
    g = run_gpu(ph, p, lam=lam)
    fo, _, gNo = oracle_face_data(p, fc)
    Uo = oracle.recover(p.coord, p.tet, fc, fm, p.a, p.c, fo, lam, gNo)
    scale = np.abs(Uo).max(axis=1, keepdims=True)
    assert np.all(np.abs(g["U"] - Uo) <= 1e-12 * scale)
    assert np.all(np.abs(g["U_factored"] - Uo) <= 1e-12 * scale)
    g["mesh"].close()


@pytest.mark.parametrize("name", ["sin_kuhn", "listing1_mixed", "mixed_l2"])
def test_solve_and_recover_parity(ph, name):
    p = make_case(name)
    g = run_gpu(ph, p, solve=True)
    o = run_oracle(p, solve=True)
    assert g["relres"] <= 1e-13
    assert np.linalg.norm(g["lam"] - o["lam"]) <= SOLVE_RTOL * np.linalg.norm(o["lam"])
    assert np.linalg.norm(g["U"] - o["U"]) <= SOLVE_RTOL * np.linalg.norm(o["U"])
    assert np.linalg.norm(g["U_factored"] - o["U"]) <= SOLVE_RTOL * np.linalg.norm(o["U"])
    g["mesh"].close()


@pytest.mark.parametrize("name", ["jitter_checker_small", "lognormal_small"])
def test_refined_solve_parity(ph, name):
    """The whole path with solves refined to fp64 accuracy on both sides:
    GPU assembly + ph_solve_refined against oracle assembly + the oracle's
    refined direct solve.  The two assemblies differ in the last bits of H and
    rhs, so the bar is 1e-9, or 10x the system's measured intrinsic
    sensitivity (one-ulp perturbations, oracle) where that is above 1e-9;
    both numbers are printed."""
    p = make_case(name)
    g = run_gpu(ph, p)
    o = run_oracle(p)
    rowptr, colind = o["csr"]["rowptr"], o["csr"]["colind"]
    lam_o, _, _ = oracle.solve_refined(rowptr, colind, o["values"], o["rhs"])
    mesh = g["mesh"]
    P = ph.Schwarz(mesh, cu(g["values"], torch.float64))
    lam_g, steps, it, corr, _ = ph.solve_refined(mesh, cu(g["values"], torch.float64), cu(g["rhs"], torch.float64),
                                                 P, tol=1e-15)
    P.close()
    err = np.linalg.norm(lam_g.cpu().numpy() - lam_o) / np.linalg.norm(lam_o)
    sens = oracle.ulp_sensitivity(rowptr, colind, o["values"], o["rhs"], trials=2)
    tol = SOLVE_RTOL if sens <= SOLVE_RTOL else 10 * sens
    print(f"{name}: Lambda error {err:.3e}, intrinsic sensitivity {sens:.3e}, bar {tol:.3e}")
    assert err <= tol
    mesh.close()


def test_table4_rates_from_gpu(ph):
    """The GPU pipeline reproduces the oracle's convergence behaviour (Table 4)."""
    from tests.test_oracle_system import error_norms
    eY = []
    for lv in (1, 2, 3):
        p = meshgen.problem("paper_mixed", lv)
        g = run_gpu(ph, p, solve=True)
        r = {"U": g["U"], "lam": g["lam"], "fc": {"tet_face": g["fc"]["tet_face"]},
             "csr": {"face_mult": g["fc"]["face_mult"]}}
        eY.append(error_norms(p, r)[0])
        g["mesh"].close()
    rY = np.log2(np.array(eY[:-1]) / np.array(eY[1:]))
    assert np.all((rY > 0.95) & (rY < 1.15))


def test_determinism(ph):
    p = make_case("lognormal_small")
    g1 = run_gpu(ph, p)
    g2 = run_gpu(ph, p)
    assert np.array_equal(g1["values"].view(np.uint64), g2["values"].view(np.uint64))
    assert np.array_equal(g1["rhs"].view(np.uint64), g2["rhs"].view(np.uint64))
    g1["mesh"].close()
    g2["mesh"].close()


def test_patch_constant(ph):
    p = meshgen.problem("kuhn_m2_k1")
    f0, c = 1.7, 0.4
    p = meshgen.Problem("patch", p.coord, p.tet, meshgen.lognormal_field(p.nE, 4), c,
                        lambda x: np.full(x.shape[0], f0), uD=lambda x: np.full(x.shape[0], f0 / c))
    g = run_gpu(ph, p, solve=True)
    assert np.abs(g["lam"]).max() <= 1e-10
    assert np.allclose(g["U"], f0 / c, rtol=1e-10, atol=0)
    g["mesh"].close()


# ---------------------------------------------------------------------------
# edge cases and errors
# ---------------------------------------------------------------------------
def test_single_tet_and_empty(ph):
    p = meshgen.Problem("one", np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float),
                        np.array([[0, 1, 2, 3]], np.int32), np.array([2.0]), 0.5, lambda x: meshgen.sin_source(x))
    g = run_gpu(ph, p)
    o = run_oracle(p)
    assert_connectivity_equal(g, o)
    assert_values_close(g, o)
    g["mesh"].close()
    m = ph.Mesh(torch.zeros((0, 3), dtype=torch.float64, device="cuda"),
                torch.zeros((0, 4), dtype=torch.int32, device="cuda"))
    assert m.nF == 0 and m.L == 0 and m.nnz == 0
    v, r = m.assemble(torch.zeros(0, dtype=torch.float64, device="cuda"), 1.0,
                      torch.zeros(0, dtype=torch.float64, device="cuda"))
    assert v.numel() == 0 and r.numel() == 0
    m.close()


def test_all_neumann_single_tet(ph):
    """Every face Neumann: no multipliers (L = 0, empty H)."""
    coord = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    tet = np.array([[0, 1, 2, 3]], np.int32)
    nb = np.array([[0, 1, 2], [0, 2, 3], [0, 3, 1], [3, 2, 1]], np.int32)
    m = ph.Mesh(cu(coord, torch.float64), cu(tet, torch.int32), cu(nb, torch.int32))
    assert m.L == 0 and m.nnz == 0 and m.nF == 4 and m.info["nF_neumann"] == 4
    m.close()


def _expect(ph, code_name, coord, tet, nb=None):
    with pytest.raises(ph.PHError) as e:
        ph.Mesh(cu(coord, torch.float64), cu(tet, torch.int32), None if nb is None else cu(nb, torch.int32))
    assert e.value.name == code_name


def test_errors(ph):
    coord, tet = meshgen.kuhn_cube(1)
    _expect(ph, "PH_ERR_NONMANIFOLD", coord, np.vstack([tet, tet[:1]]))
    _expect(ph, "PH_ERR_ARG", coord, np.array([[0, 1, 2, 99]], np.int32))
    _expect(ph, "PH_ERR_ARG", coord, np.array([[0, 1, 1, 2]], np.int32))
    flat = coord.copy()
    flat[:, 2] = 0.0
    _expect(ph, "PH_ERR_DEGENERATE", flat, tet)
    fc = oracle.faces(tet, 8)
    inner = fc["face_vtx"][np.where(fc["face_tet"][:, 1] >= 0)[0][:1]]
    _expect(ph, "PH_ERR_ARG", coord, tet, inner)
    _expect(ph, "PH_ERR_ARG", coord, tet, np.array([[0, 1, 6]], np.int32))
    # invalid coefficient: flagged on the device, reported by ph_mesh_check
    m = ph.Mesh(cu(coord, torch.float64), cu(tet, torch.int32))
    a = torch.ones(m.nE, dtype=torch.float64, device="cuda")
    a[3] = -1.0
    f = torch.ones(m.nF, dtype=torch.float64, device="cuda")
    m.assemble(a, 1.0, f)
    with pytest.raises(ph.PHError) as e:
        m.check()
    assert e.value.name == "PH_ERR_ARG"
    m.check()  # cleared
    with pytest.raises(ph.PHError):
        m.assemble(torch.ones(m.nE, dtype=torch.float64, device="cuda"), 0.0, f)
    m.close()


def test_launch_counter(ph):
    n0 = ph.ph_launch_count()
    p = make_case("sin_kuhn")
    g = run_gpu(ph, p)
    assert ph.ph_launch_count() > n0
    g["mesh"].close()
