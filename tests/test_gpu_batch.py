"""Batched assembly (one persistent launch over many meshes of uneven size,
each with its own coefficient field) against plain per-problem ph_assemble
calls: values, rhs and element factor must be bit-identical, under every
configuration the autotuner tries, and through the captured CUDA graph.
Problems of the batch are also checked against the oracle directly."""
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
    for i, (m, k) in enumerate([(1, 0), (2, 1), (1, 2), (3, 1), (6, 1), (2, 2), (5, 1)]):
        coord, tet = meshgen.kuhn_cube(m)
        coord, tet, _ = meshgen.refined(coord, tet, k)
        out.append(meshgen.Problem(f"k{m}_{k}", coord, tet, meshgen.lognormal_field(tet.shape[0], 4000 + i),
                                   0.1 + 0.05 * i, lambda x: meshgen.sin_source(x)))
    out.append(meshgen.problem("paper_mixed", 2))          # Neumann faces and Dirichlet data
    coord, tet = meshgen.shuffled(out[1].coord, out[1].tet, 3)
    out.append(meshgen.Problem("shuffled", coord, tet, meshgen.lognormal_field(tet.shape[0], 9), 0.7, out[1].f))
    return out


class Case:
    def __init__(self, ph, p):
        neu = cu(p.neumann.astype(np.int32)) if p.neumann.size else None
        self.mesh = ph.Mesh(cu(p.coord), cu(p.tet.astype(np.int32)), neu)
        cen = self.mesh.faces()["face_centroid"].cpu().numpy()
        self.f = cu(np.asarray(p.f(cen), np.float64))
        self.uD = None if p.uD is None else cu(np.asarray(p.uD(cen), np.float64))
        self.gN = None if p.gN is None else cu(np.asarray(p.gN(cen), np.float64))
        self.a = cu(p.a)
        self.c = p.c
        m = self.mesh
        self.values = torch.full((m.nnz,), np.nan, dtype=torch.float64, device="cuda")
        self.rhs = torch.full((m.L,), np.nan, dtype=torch.float64, device="cuda")
        self.factor = torch.full((m.nE, 10), np.nan, dtype=torch.float64, device="cuda")
        self.ref = m.assemble(self.a, self.c, self.f, self.uD, self.gN, factor=True)


@pytest.fixture(scope="module")
def batch(ph):
    cases = [Case(ph, p) for p in problems()]
    b = ph.Batch([c.mesh for c in cases])
    b.bind([c.a for c in cases], [c.c for c in cases], [c.f for c in cases], [c.values for c in cases],
           [c.rhs for c in cases], factor=[c.factor for c in cases], uD_face=[c.uD for c in cases],
           gN_face=[c.gN for c in cases])
    return b, cases


def assert_identical(cases):
    torch.cuda.synchronize()
    for c in cases:
        v, r, f = c.ref
        assert torch.equal(c.values, v)
        assert torch.equal(c.rhs, r)
        assert torch.equal(c.factor, f)
        c.mesh.check()


def _reset(cases):
    for c in cases:
        c.values.fill_(np.nan)
        c.rhs.fill_(np.nan)
        c.factor.fill_(np.nan)


def test_batched_equals_plain(batch):
    b, cases = batch
    _reset(cases)
    b.assemble()
    assert_identical(cases)


@pytest.mark.parametrize("i", [0, 2, 4, 7, 8])
def test_batched_against_oracle(batch, i):
    """Problem i of the uneven batch against the oracle (Kuhn 1^3 cube, 1^3
    refined twice, 6^3 refined once, the paper's mixed example with Neumann
    and Dirichlet data, and the shuffled mesh): CSR pattern bit-exact, H
    entrywise to 1e-12, rhs to 1e-12 of the sum of its addends' magnitudes."""
    b, cases = batch
    _reset(cases)
    b.assemble()
    torch.cuda.synchronize()
    p, c = problems()[i], cases[i]
    ref = oracle.pipeline(p.coord, p.tet, p.a, p.c, p.f, p.uD, p.gN, p.neumann if p.neumann.size else None,
                          do_solve=False)
    rowptr, colind = c.mesh.csr_pattern()
    assert np.array_equal(rowptr.cpu().numpy(), ref["csr"]["rowptr"])
    assert np.array_equal(colind.cpu().numpy(), ref["csr"]["colind"])
    v = c.values.cpu().numpy()
    assert np.all(np.abs(v - ref["values"]) <= 1e-12 * np.abs(ref["values"]))
    r = c.rhs.cpu().numpy()
    assert np.all(np.abs(r - ref["rhs"]) <= 1e-12 * ref["rhs_abs"] + 1e-300)
    c.mesh.check()


@pytest.mark.parametrize("cfg", [(256, 64, 2), (1024, 128, 4), (4096, 256, 8), (16384, 128, 1), (32, 32, 32)])
def test_every_configuration(batch, cfg):
    b, cases = batch
    b.set_config(*cfg)
    assert tuple(b.get_config().values()) == cfg
    _reset(cases)
    b.assemble()
    assert_identical(cases)


def test_autotune_and_graph(batch):
    b, cases = batch
    ms = b.autotune(reps=2)
    assert ms > 0
    cfg = b.get_config()
    assert cfg["tile"] in (256, 1024, 4096, 16384)
    for _ in range(2):
        _reset(cases)
        b.graph_launch()
        assert_identical(cases)
    # rebinding new coefficients keeps the graph valid and changes the result
    for c in cases:
        c.a.mul_(1.5)
        c.ref = c.mesh.assemble(c.a, c.c, c.f, c.uD, c.gN, factor=True)
    _reset(cases)
    b.graph_launch()
    assert_identical(cases)


def test_config4_recipe_subset(ph):
    """16 problems drawn like the batched workload (sizes log-uniform in
    [1e4, 5e5] elements, each its own lognormal field)."""
    rng = np.random.Generator(np.random.PCG64(4))
    sizes = np.exp(rng.uniform(np.log(1e4), np.log(5e5), 16))
    cases = []
    for i, s in enumerate(sizes):
        m = int(np.clip(round((s / 72) ** (1 / 3)), 6, 19))
        coord, tet = meshgen.kuhn_cube(m)
        coord, tet, _ = meshgen.refined(coord, tet, 1)
        p = meshgen.Problem("b", coord, tet, meshgen.lognormal_field(tet.shape[0], 4000 + i), 0.1,
                            lambda x: meshgen.sin_source(x))
        cases.append(Case(ph, p))
    b = ph.Batch([c.mesh for c in cases])
    b.bind([c.a for c in cases], [c.c for c in cases], [c.f for c in cases], [c.values for c in cases],
           [c.rhs for c in cases], factor=[c.factor for c in cases])
    b.autotune(reps=1)
    b.graph_launch()
    assert_identical(cases)
    b.close()


def test_batched_recovery_in_the_graph(ph):
    """Assembly and recovery of an uneven batch in one captured graph (three
    launches): every problem's u bit-identical to ph_recover_factored on its
    own factor, and the oracle's recovery within 1e-12."""
    probs = problems()
    cases = [Case(ph, p) for p in probs]
    b = ph.Batch([c.mesh for c in cases])
    b.bind([c.a for c in cases], [c.c for c in cases], [c.f for c in cases], [c.values for c in cases],
           [c.rhs for c in cases], factor=[c.factor for c in cases], uD_face=[c.uD for c in cases],
           gN_face=[c.gN for c in cases])
    rng = np.random.default_rng(21)
    lam_h = [rng.standard_normal(c.mesh.L) for c in cases]
    lam = [cu(x) for x in lam_h]
    us = [torch.full((c.mesh.nE, 4), np.nan, dtype=torch.float64, device="cuda") for c in cases]
    b.bind_recovery(lam, us)
    n0 = ph.ph_launch_count()
    b.graph_launch()
    torch.cuda.synchronize()
    assert ph.ph_launch_count() - n0 == 3
    for p, c, l, lh, u in zip(probs, cases, lam, lam_h, us):
        v, r, fa = c.ref
        ref = c.mesh.recover_factored(fa, c.c, c.f, l, c.gN)
        assert torch.equal(u, ref), p.name
        # the oracle on its own faces, face data and the host copy of Lambda
        fc = oracle.faces(p.tet, p.nC, p.neumann if p.neumann.size else None)
        fm, _ = oracle.multipliers(fc["face_kind"])
        cen = oracle.face_centroids(p.coord, fc["face_vtx"])
        gN = None if p.gN is None else np.asarray(p.gN(cen), np.float64)
        Uo = oracle.recover(p.coord, p.tet, fc, fm, p.a, c.c, np.asarray(p.f(cen), np.float64), lh, gN)
        scale = np.abs(Uo).max(axis=1, keepdims=True)
        assert np.all(np.abs(u.cpu().numpy() - Uo) <= 1e-12 * scale), p.name
    b.bind_recovery(None, None)  # back to two launches
    n0 = ph.ph_launch_count()
    b.graph_launch()
    torch.cuda.synchronize()
    assert ph.ph_launch_count() - n0 == 2
    b.close()
