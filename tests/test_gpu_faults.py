"""Error paths of the library, exercised without faulting or hanging the GPU
(the failures are made on the host or by bounded device waits):

- a device allocation that fails (test hook) returns PH_ERR_NOMEM and the
  failed call leaves nothing allocated in the library's pool;
- a scan whose look-back wait runs out (test hook: one tile never publishes,
  with a short poll limit) makes ph_mesh_create return PH_ERR_TIMEOUT, and
  the next build on the same context is correct;
- an iteration cap gives PH_ERR_NOT_CONVERGED;
- a NaN or negative coefficient, a NaN reaction constant and a NaN vertex
  give PH_ERR_ARG / PH_ERR_DEGENERATE.
"""
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
    yield ph
    ph.ph_test_fail_alloc(-1)
    ph.ph_test_scan_withhold(False)


def cu(x):
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


def kuhn(m, k=0):
    coord, tet = meshgen.kuhn_cube(m)
    if k:
        coord, tet, _ = meshgen.refined(coord, tet, k)
    return coord, tet


def test_allocation_failure_returns_nomem_without_leak(ph):
    coord, tet = kuhn(3, 1)
    c_d, t_d = cu(coord), cu(tet)
    torch.cuda.synchronize()
    before = ph.ph_pool_in_use()
    for after in (0, 1):  # the mesh arrays, then the build's scratch
        ph.ph_test_fail_alloc(after)
        with pytest.raises(ph.PHError) as e:
            ph.Mesh(c_d, t_d)
        assert e.value.name == "PH_ERR_NOMEM"
        torch.cuda.synchronize()
        assert ph.ph_pool_in_use() == before
    ph.ph_test_fail_alloc(-1)
    m = ph.Mesh(c_d, t_d)
    values, rhs = m.assemble(cu(np.ones(m.nE)), 1.0, cu(np.ones(m.nF)))
    rowptr, colind = m.csr_pattern()
    ph.ph_test_fail_alloc(0)  # the solver's workspace
    x, it, rr, code = ph.ph_solve_pcg(rowptr, colind, values, rhs, check=False)
    ph.ph_test_fail_alloc(-1)
    assert ph.ph_status_string(code) == "PH_ERR_NOMEM"
    m.check()
    m.close()
    torch.cuda.synchronize()
    assert ph.ph_pool_in_use() == before


def test_scan_lookback_timeout(ph):
    coord, tet = kuhn(16)  # 4913 vertices: the bucket scan spans 5 tiles of 4096
    c_d, t_d = cu(coord), cu(tet)
    ph.ph_test_scan_withhold(True)
    try:
        with pytest.raises(ph.PHError) as e:
            ph.Mesh(c_d, t_d)
    finally:
        ph.ph_test_scan_withhold(False)
    assert e.value.name == "PH_ERR_TIMEOUT"
    # the context is intact: the same build now matches the oracle
    m = ph.Mesh(c_d, t_d)
    o = oracle.faces(tet, coord.shape[0])
    assert np.array_equal(m.faces()["tet_face"].cpu().numpy(), o["tet_face"])
    m.close()


def test_iteration_cap_not_converged(ph):
    p = meshgen.problem("sin_kuhn")
    m = ph.Mesh(cu(p.coord), cu(p.tet))
    f = cu(np.asarray(p.f(m.faces()["face_centroid"].cpu().numpy()), np.float64))
    values, rhs = m.assemble(cu(p.a), p.c, f)
    rowptr, colind = m.csr_pattern()
    _, it, rr, code = ph.ph_solve_pcg(rowptr, colind, values, rhs, rtol=1e-12, maxit=3, check=False)
    assert ph.ph_status_string(code) == "PH_ERR_NOT_CONVERGED" and it == 3 and rr > 1e-12
    P = ph.Schwarz(m, values)
    _, it, rr, code = P.solve(values, rhs, rtol=1e-12, maxit=3, check=False)
    assert ph.ph_status_string(code) == "PH_ERR_NOT_CONVERGED" and it == 3 and rr > 1e-12
    with pytest.raises(ph.PHError) as e:
        P.solve(values, rhs, rtol=1e-12, maxit=3)
    assert e.value.name == "PH_ERR_NOT_CONVERGED"
    P.close()
    m.close()


@pytest.mark.parametrize("bad", [np.nan, -1.0, np.inf, 0.0])
def test_invalid_coefficient_flags_arg(ph, bad):
    coord, tet = kuhn(2, 1)
    m = ph.Mesh(cu(coord), cu(tet))
    a = np.ones(m.nE)
    a[17] = bad
    m.assemble(cu(a), 1.0, cu(np.ones(m.nF)))
    with pytest.raises(ph.PHError) as e:
        m.check()
    assert e.value.name == "PH_ERR_ARG"
    m.check()  # cleared by the previous check
    with pytest.raises(ph.PHError) as e:
        m.assemble(cu(np.ones(m.nE)), float("nan"), cu(np.ones(m.nF)))
    assert e.value.name == "PH_ERR_ARG"
    m.close()


def test_nan_vertex_is_degenerate(ph):
    coord, tet = kuhn(2)
    coord = coord.copy()
    coord[13] = np.nan
    with pytest.raises(ph.PHError) as e:
        ph.Mesh(cu(coord), cu(tet))
    assert e.value.name == "PH_ERR_DEGENERATE"
