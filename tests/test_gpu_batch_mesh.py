"""The batched mesh build (ph_mesh_create_batch): many meshes of uneven size,
with and without Neumann faces, from one enqueued build and one host
synchronisation.  Every problem's connectivity and CSR pattern must be
bit-identical to the oracle's and to a plain ph_mesh_create of that problem;
geometry-derived arrays (face areas, centroids) and assembly on the returned
meshes must equal the plain ones bit for bit; the meshes may be destroyed in
any order; an invalid problem fails the whole call."""
import numpy as np
import pytest

import meshgen
import oracle

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


def cu(x):
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


def problems():
    out = []
    for i, (m, k) in enumerate([(1, 0), (2, 1), (1, 2), (3, 1), (6, 1), (2, 2)]):
        coord, tet = meshgen.kuhn_cube(m)
        coord, tet, _ = meshgen.refined(coord, tet, k)
        out.append(meshgen.Problem(f"k{m}_{k}", coord, tet, meshgen.lognormal_field(tet.shape[0], 50 + i), 0.2,
                                   lambda x: meshgen.sin_source(x)))
    out.insert(2, meshgen.problem("paper_mixed", 2))        # Neumann faces
    coord, tet = meshgen.shuffled(out[1].coord, out[1].tet, 7)
    out.append(meshgen.Problem("shuffled", coord, tet, meshgen.lognormal_field(tet.shape[0], 9), 0.7, out[1].f))
    out.append(meshgen.problem("paper_mixed", 1))
    return out


def build(ph, probs):
    return ph.create_meshes([cu(p.coord) for p in probs], [cu(p.tet.astype(np.int32)) for p in probs],
                            [cu(p.neumann.astype(np.int32)) if p.neumann.size else None for p in probs])


def test_batched_build_matches_oracle_and_plain(ph):
    probs = problems()
    meshes = build(ph, probs)
    for p, m in zip(probs, meshes):
        nb = p.neumann if p.neumann.size else None
        o = oracle.faces(p.tet, p.nC, nb)
        fm, L = oracle.multipliers(o["face_kind"])
        rowptr, colind = oracle.csr_pattern(o["tet_face"], fm, L)
        g = {k: v.cpu().numpy() for k, v in m.faces().items()}
        for k in ("tet_face", "face_tet", "face_vtx", "face_kind"):
            assert np.array_equal(g[k], o[k]), (p.name, k)
        assert np.array_equal(g["face_mult"], fm)
        rp, ci = m.csr_pattern()
        assert np.array_equal(rp.cpu().numpy(), rowptr) and np.array_equal(ci.cpu().numpy(), colind), p.name
        assert (m.nE, m.nC, m.nF, m.L, m.nnz) == (p.nE, p.nC, o["nF"], L, colind.size)
        # every array equal to a plain build of the same problem
        q = ph.Mesh(cu(p.coord), cu(p.tet.astype(np.int32)), cu(p.neumann.astype(np.int32)) if nb is not None else None)
        assert m.info == q.info
        h = {k: v.cpu().numpy() for k, v in q.faces().items()}
        for k in g:
            assert np.array_equal(g[k].view(np.uint8), h[k].view(np.uint8)), (p.name, k)
        f = cu(np.asarray(p.f(g["face_centroid"]), np.float64))
        uD = None if p.uD is None else cu(np.asarray(p.uD(g["face_centroid"]), np.float64))
        gN = None if p.gN is None else cu(np.asarray(p.gN(g["face_centroid"]), np.float64))
        v1, r1, f1 = m.assemble(cu(p.a), p.c, f, uD, gN, factor=True)
        v2, r2, f2 = q.assemble(cu(p.a), p.c, f, uD, gN, factor=True)
        assert torch.equal(v1, v2) and torch.equal(r1, r2) and torch.equal(f1, f2), p.name
        lam = cu(np.random.default_rng(3).standard_normal(m.L))
        assert torch.equal(m.recover_factored(f1, p.c, f, lam, gN), q.recover_factored(f2, p.c, f, lam, gN))
        m.check()
        q.close()
    for i in np.random.default_rng(0).permutation(len(meshes)):  # any order
        meshes[i].close()
    torch.cuda.synchronize()


def test_batched_build_feeds_the_batched_assembly(ph):
    probs = problems()[:6]
    meshes = build(ph, probs)
    fs = [cu(np.asarray(p.f(m.faces()["face_centroid"].cpu().numpy()), np.float64)) for p, m in zip(probs, meshes)]
    outs = [(torch.empty(m.nnz, dtype=torch.float64, device="cuda"), torch.empty(m.L, dtype=torch.float64,
                                                                                  device="cuda")) for m in meshes]
    b = ph.Batch(meshes)
    b.bind([cu(p.a) for p in probs], [p.c for p in probs], fs, [o[0] for o in outs], [o[1] for o in outs])
    b.graph_launch()
    torch.cuda.synchronize()
    for p, m, f, (v, r) in zip(probs, meshes, fs, outs):
        v2, r2 = m.assemble(cu(p.a), p.c, f)
        assert torch.equal(v, v2) and torch.equal(r, r2)
    b.close()
    for m in meshes:
        m.close()


def test_batched_build_rejects_an_invalid_problem(ph):
    probs = problems()[:4]
    tets = [cu(p.tet.astype(np.int32)) for p in probs]
    bad = probs[2].tet.astype(np.int32).copy()
    bad[5, 1] = probs[2].nC + 3  # id out of range in one problem
    tets[2] = cu(bad)
    with pytest.raises(ph.PHError) as e:
        ph.create_meshes([cu(p.coord) for p in probs], tets)
    assert e.value.name == "PH_ERR_ARG"


def test_batched_build_of_empty_problems(ph):
    probs = [problems()[i] for i in (0, 1, 3)]  # no Neumann faces
    coords = [cu(p.coord) for p in probs]
    tets = [cu(p.tet.astype(np.int32)) for p in probs]
    coords.insert(1, torch.zeros((0, 3), dtype=torch.float64, device="cuda"))
    tets.insert(1, torch.zeros((0, 4), dtype=torch.int32, device="cuda"))
    meshes = ph.create_meshes(coords, tets)
    assert meshes[1].nE == 0 and meshes[1].nF == 0 and meshes[1].L == 0
    for p, m in zip(probs, [meshes[0], meshes[2], meshes[3]]):
        o = oracle.faces(p.tet, p.nC)
        assert np.array_equal(m.faces()["tet_face"].cpu().numpy(), o["tet_face"])
    for m in meshes:
        m.close()
