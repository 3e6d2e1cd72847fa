"""The oracle's multi-threaded element loops (or_assemble_mt, or_recover_mt)
give the same bits as its plain loops, and report the same first error."""
import numpy as np
import pytest

import meshgen
import oracle


def _system(p):
    fc = oracle.faces(p.tet, p.nC, p.neumann if p.neumann.size else None)
    fm, L = oracle.multipliers(fc["face_kind"])
    rowptr, colind = oracle.csr_pattern(fc["tet_face"], fm, L)
    cen = oracle.face_centroids(p.coord, fc["face_vtx"])
    data = {k: (None if fn is None else np.asarray(fn(cen), np.float64)) for k, fn in
            (("f", p.f), ("uD", p.uD), ("gN", p.gN))}
    return fc, {"face_mult": fm, "L": L, "rowptr": rowptr, "colind": colind}, data


@pytest.mark.parametrize("name", ["paper_mixed", "lognormal"])
def test_threaded_loops_are_bit_identical(name):
    if name == "paper_mixed":
        p = meshgen.problem("paper_mixed", 2)
    else:
        coord, tet = meshgen.kuhn_cube(2)
        coord, tet, _ = meshgen.refined(coord, tet, 2)
        coord, tet = meshgen.shuffled(coord, tet, 5)
        p = meshgen.Problem(name, coord, tet, meshgen.lognormal_field(tet.shape[0], 8), 0.3,
                            lambda x: meshgen.sin_source(x))
    fc, csr, d = _system(p)
    ref = oracle.assemble(p.coord, p.tet, fc, csr, p.a, p.c, d["f"], d["uD"], d["gN"], nthreads=1)
    for nt in (2, 5):
        got = oracle.assemble(p.coord, p.tet, fc, csr, p.a, p.c, d["f"], d["uD"], d["gN"], nthreads=nt)
        for r, g in zip(ref, got):
            assert np.array_equal(r.view(np.int64), g.view(np.int64))
    lam = np.random.default_rng(1).standard_normal(csr["L"])
    U1 = oracle.recover(p.coord, p.tet, fc, csr["face_mult"], p.a, p.c, d["f"], lam, d["gN"], nthreads=1)
    U4 = oracle.recover(p.coord, p.tet, fc, csr["face_mult"], p.a, p.c, d["f"], lam, d["gN"], nthreads=4)
    assert np.array_equal(U1.view(np.int64), U4.view(np.int64))


def test_threaded_loops_report_the_first_error():
    coord, tet = meshgen.kuhn_cube(2)
    p = meshgen.Problem("k", coord, tet, np.ones(tet.shape[0]), 1.0, lambda x: meshgen.sin_source(x))
    fc, csr, d = _system(p)
    a = p.a.copy()
    a[7] = np.nan
    a[30] = -1.0
    for nt in (1, 3):
        with pytest.raises(oracle.OracleError) as e:
            oracle.assemble(p.coord, p.tet, fc, csr, a, p.c, d["f"], nthreads=nt)
        assert e.value.name == "ARG"
        with pytest.raises(oracle.OracleError) as e:
            oracle.recover(p.coord, p.tet, fc, csr["face_mult"], a, p.c, d["f"], np.zeros(csr["L"]), nthreads=nt)
        assert e.value.name == "ARG"
