"""ph_assemble_host (the whole path from and to host buffers, copies
overlapped with the kernels) against the same steps through the device entry
points: bit-identical outputs, pinned and pageable buffers, with and without
Neumann and Dirichlet data, and the count check; and the cold host path: the
counts and face centroids from ph_host_mesh_query alone, with no device
tensor in the caller's hands."""
import numpy as np
import pytest

import meshgen

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


def device_path(ph, p):
    cu = lambda x: torch.as_tensor(np.ascontiguousarray(x), device="cuda")
    neu = cu(p.neumann.astype(np.int32)) if p.neumann.size else None
    m = ph.Mesh(cu(p.coord), cu(p.tet.astype(np.int32)), neu)
    cen = m.faces()["face_centroid"].cpu().numpy()
    data = {"f": np.asarray(p.f(cen), np.float64),
            "uD": None if p.uD is None else np.asarray(p.uD(cen), np.float64),
            "gN": None if p.gN is None else np.asarray(p.gN(cen), np.float64),
            "lam": np.random.default_rng(4).standard_normal(m.L)}
    opt = lambda k: None if data[k] is None else cu(data[k])
    rowptr, colind = m.csr_pattern()
    values, rhs, factor = m.assemble(cu(p.a), p.c, cu(data["f"]), opt("uD"), opt("gN"), factor=True)
    u = m.recover_factored(factor, p.c, cu(data["f"]), cu(data["lam"]), opt("gN"))
    ref = {"rowptr": rowptr.cpu(), "colind": colind.cpu(), "values": values.cpu(), "rhs": rhs.cpu(), "u": u.cpu()}
    counts = (m.nF, m.L, m.nnz)
    m.close()
    return data, ref, counts


@pytest.mark.parametrize("case", ["lognormal_small", "paper_mixed2"])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_path_matches_device_path(ph, case, pinned):
    if case == "paper_mixed2":
        p = meshgen.problem("paper_mixed", 2)
    else:
        coord, tet = meshgen.kuhn_cube(3)
        coord, tet, _ = meshgen.refined(coord, tet, 2)
        p = meshgen.Problem(case, coord, tet, meshgen.lognormal_field(tet.shape[0], 2), 0.1,
                            lambda x: meshgen.sin_source(x))
    data, ref, counts = device_path(ph, p)
    host = lambda x: None if x is None else (torch.from_numpy(np.ascontiguousarray(x)).pin_memory() if pinned
                                              else torch.from_numpy(np.ascontiguousarray(x)))
    out = ph.ph_assemble_host(host(p.coord), host(p.tet.astype(np.int32)), host(p.a), p.c, host(data["f"]), counts,
                              lam=host(data["lam"]), uD_face=host(data["uD"]), gN_face=host(data["gN"]),
                              neumann=host(p.neumann.astype(np.int32)) if p.neumann.size else None)
    for k in ("rowptr", "colind", "values", "rhs", "u"):
        assert torch.equal(out[k], ref[k]), k


def test_host_path_checks_counts(ph):
    coord, tet = meshgen.kuhn_cube(2)
    p = meshgen.Problem("k2", coord, tet, np.ones(tet.shape[0]), 1.0, lambda x: meshgen.sin_source(x))
    data, ref, (nF, L, nnz) = device_path(ph, p)
    with pytest.raises(ph.PHError) as e:
        ph.ph_assemble_host(torch.from_numpy(coord), torch.from_numpy(tet.astype(np.int32)),
                            torch.from_numpy(p.a), 1.0, torch.from_numpy(data["f"]), (nF, L, nnz + 1))
    assert e.value.name == "PH_ERR_ARG"


def test_host_path_full_size(ph):
    """The bench's end-to-end configuration: the lognormal workload (3,359,232
    tets), pinned buffers, outputs bit-identical to the device entry points."""
    p = meshgen.problem("lognormal_3m")
    data, ref, counts = device_path(ph, p)
    pin = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
    out = ph.ph_assemble_host(pin(p.coord), pin(p.tet.astype(np.int32)), pin(p.a), p.c, pin(data["f"]), counts,
                              lam=pin(data["lam"]))
    for k in ("rowptr", "colind", "values", "rhs", "u"):
        assert torch.equal(out[k], ref[k]), k


@pytest.mark.parametrize("case", ["lognormal_small", "paper_mixed2"])
def test_cold_host_path(ph, case):
    if case == "paper_mixed2":
        p = meshgen.problem("paper_mixed", 2)
    else:
        coord, tet = meshgen.kuhn_cube(3)
        coord, tet, _ = meshgen.refined(coord, tet, 2)
        p = meshgen.Problem(case, coord, tet, meshgen.lognormal_field(tet.shape[0], 2), 0.1,
                            lambda x: meshgen.sin_source(x))
    data, ref, counts = device_path(ph, p)
    h = lambda x: None if x is None else torch.from_numpy(np.ascontiguousarray(x))
    neu = h(p.neumann.astype(np.int32)) if p.neumann.size else None
    info, cen = ph.ph_host_mesh_query(h(p.coord), h(p.tet.astype(np.int32)), neu)
    assert (info["nF"], info["L"], info["nnz"]) == counts
    cen = cen.numpy()
    f = np.asarray(p.f(cen), np.float64)
    assert np.array_equal(f, data["f"])  # the same centroids as the device build's
    uD = None if p.uD is None else np.asarray(p.uD(cen), np.float64)
    gN = None if p.gN is None else np.asarray(p.gN(cen), np.float64)
    out = ph.ph_assemble_host(h(p.coord), h(p.tet.astype(np.int32)), h(p.a), p.c, h(f),
                              (info["nF"], info["L"], info["nnz"]), lam=h(data["lam"]), uD_face=h(uD), gN_face=h(gN),
                              neumann=neu)
    for k in ("rowptr", "colind", "values", "rhs", "u"):
        assert torch.equal(out[k], ref[k]), k
    # counts only, and a centroid buffer that is too small
    info2, none = ph.ph_host_mesh_query(h(p.coord), h(p.tet.astype(np.int32)), neu, centroids=False)
    assert info2 == info and none is None
