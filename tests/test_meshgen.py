"""Pins of the seeded input generator (the paper's refinement and counts)."""
import numpy as np
import pytest

import meshgen
import oracle


def _read_refine(golden_dir):
    T, C, cur = [], [], None
    for line in open(f"{golden_dir}/refine_example.txt"):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line in ("T", "C"):
            cur = line
            continue
        (T if cur == "T" else C).append([float(v) for v in line.split()])
    return np.array(T, dtype=np.int64), np.array(C)


def test_refine_example(golden_dir):
    """Section 3.4 Example: [1 3 2 4] on the unit reference tet -> 12 tets, 11 nodes."""
    T_ref, C_ref = _read_refine(golden_dir)
    coord = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    tet = np.array([[1, 3, 2, 4]], np.int32) - 1
    c2, t2, _ = meshgen.red_refine(coord, tet)
    assert np.array_equal(t2 + 1, T_ref)
    assert np.array_equal(c2, C_ref)


def _counts(level):
    coord, tet, _, _ = meshgen.listing1_mesh()
    coord, tet, _ = meshgen.refined(coord, tet, level)
    U, _ = meshgen.number_edges(tet, coord.shape[0])
    fc = oracle.faces(tet, coord.shape[0])
    return tet.shape[0], coord.shape[0], U.shape[0], fc["nF"]


@pytest.mark.parametrize("level", [1, 2, 3, 4])
def test_table1_counts(golden_dir, level):
    """Table 1: (nE, nC, nEd, nF) per level; nF comes from the oracle's faces."""
    rows = np.loadtxt(f"{golden_dir}/table1_counts.txt", dtype=np.int64)
    want = rows[rows[:, 0] == level][0, 1:]
    assert tuple(_counts(level)) == tuple(want)


@pytest.mark.slow
def test_table1_counts_level5(golden_dir):
    rows = np.loadtxt(f"{golden_dir}/table1_counts.txt", dtype=np.int64)
    assert tuple(_counts(5)) == tuple(rows[rows[:, 0] == 5][0, 1:])


def _vol6(coord, tet):
    P = [coord[tet[:, i]] for i in range(4)]
    return np.einsum("ij,ij->i", P[1] - P[0], np.cross(P[2] - P[0], P[3] - P[0]))


def test_children_volumes():
    """Corner children have 1/8 of the parent volume, octahedron children 1/16,
    and all keep the parent's orientation."""
    coord, tet = meshgen.kuhn_cube(1)
    v0 = _vol6(coord, tet)
    c2, t2, _ = meshgen.red_refine(coord, tet)
    v1 = _vol6(c2, t2)
    nE = tet.shape[0]
    assert np.allclose(v1[:nE], v0 / 8, rtol=1e-14, atol=0)
    kids = v1[nE:].reshape(nE, 11)
    assert np.allclose(kids[:, :3], (v0 / 8)[:, None], rtol=1e-14, atol=0)
    assert np.allclose(kids[:, 3:], (v0 / 16)[:, None], rtol=1e-14, atol=0)


@pytest.mark.parametrize("m,k", [(1, 0), (2, 1), (1, 2), (3, 1)])
def test_kuhn_euler_and_boundary(m, k):
    """V - E + F - T = 1 for the cube, and 12 m^2 4^k boundary faces."""
    coord, tet = meshgen.kuhn_cube(m)
    coord, tet, _ = meshgen.refined(coord, tet, k)
    U, _ = meshgen.number_edges(tet, coord.shape[0])
    fc = oracle.faces(tet, coord.shape[0])
    assert coord.shape[0] - U.shape[0] + fc["nF"] - tet.shape[0] == 1
    assert int((fc["face_kind"] == oracle.KIND_DIRICHLET).sum()) == 12 * m * m * 4 ** k
    assert np.isclose(np.abs(_vol6(coord, tet)).sum() / 6, 1.0, rtol=1e-13)


def test_jitter_valid():
    coord, tet = meshgen.kuhn_cube(1)
    coord, tet, _ = meshgen.refined(coord, tet, 3)
    c2, _ = meshgen.jitter_interior(coord, tet, 0.2, seed=3)
    v0, v1 = _vol6(coord, tet), _vol6(c2, tet)
    assert np.all(v1 / v0 >= 0.1)
    bnd = np.any((coord == 0) | (coord == 1), axis=1)
    assert np.array_equal(c2[bnd], coord[bnd])
    assert np.abs(c2[~bnd] - coord[~bnd]).max() > 0
    assert np.isclose(np.abs(v1).sum() / 6, 1.0, rtol=1e-12)
