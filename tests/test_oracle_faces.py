"""Pins of the oracle's face connectivity (Section 3.3) against the paper's
printed example, a brute-force definition on tiny meshes and invariants."""
import numpy as np
import pytest

import meshgen
import oracle

LFACE = [(0, 1, 2), (0, 2, 3), (0, 3, 1), (3, 2, 1)]


def test_listing1_faces_example(golden_dir):
    coord, tet, _, _ = meshgen.listing1_mesh()
    fc = oracle.faces(tet, 8)
    lines = [l.split() for l in open(f"{golden_dir}/listing1_faces.txt") if l.strip() and not l.startswith("#")]
    g = {l[0]: [int(v) for v in l[1:]] for l in lines}
    assert fc["nF"] == g["nF"][0]
    # rows 4t+1..4t+4 are tet t's local faces in local order (t = 1..4)
    for t in range(4):
        for k in range(4):
            assert list(fc["face_vtx"][4 * t + k]) == [tet[t][j] for j in LFACE[k]]
            assert fc["tet_face"][t][k] == 4 * t + k
    ids = [(int(x) & 0x7FFFFFFF) + 1 for x in fc["tet_face"][4]]
    assert ids == g["tet5_rows"]
    assert all(int(x) < 0 for x in fc["tet_face"][4])      # tet 5 is T- of all its faces


def brute_faces(tet):
    """The definition on a dict: first sighting of a vertex set numbers it."""
    ids, tf, ftet, fvtx = {}, [], [], []
    for t, T in enumerate(tet):
        row = []
        for k in range(4):
            tup = tuple(int(T[j]) for j in LFACE[k])
            key = frozenset(tup)
            if key not in ids:
                ids[key] = len(ftet)
                ftet.append([t, -1])
                fvtx.append(list(tup))
                row.append(ids[key])
            else:
                F = ids[key]
                assert ftet[F][1] == -1
                ftet[F][1] = t
                row.append(F | -0x80000000)
        tf.append(row)
    return np.array(tf, np.int32), np.array(ftet, np.int32), np.array(fvtx, np.int32)


@pytest.mark.parametrize("case", ["kuhn2", "kuhn1k1", "shuffled", "listing1k1"])
def test_faces_match_bruteforce(case):
    if case == "kuhn2":
        coord, tet = meshgen.kuhn_cube(2)
    elif case == "kuhn1k1":
        coord, tet = meshgen.kuhn_cube(1)
        coord, tet, _ = meshgen.refined(coord, tet, 1)
    elif case == "shuffled":
        coord, tet = meshgen.kuhn_cube(2)
        coord, tet, _ = meshgen.refined(coord, tet, 1)
        coord, tet = meshgen.shuffled(coord, tet, 7)
    else:
        coord, tet, _, _ = meshgen.listing1_mesh()
        coord, tet, _ = meshgen.refined(coord, tet, 1)
    fc = oracle.faces(tet, coord.shape[0])
    tf, ft, fv = brute_faces(tet)
    assert np.array_equal(fc["tet_face"], tf)
    assert np.array_equal(fc["face_tet"], ft)
    assert np.array_equal(fc["face_vtx"], fv)


def test_face_invariants():
    coord, tet = meshgen.kuhn_cube(2)
    coord, tet, _ = meshgen.refined(coord, tet, 2)
    fc = oracle.faces(tet, coord.shape[0])
    nE, nF = tet.shape[0], fc["nF"]
    ft = fc["face_tet"]
    deg = 1 + (ft[:, 1] >= 0)
    assert deg.sum() == 4 * nE                                  # every slot is one face occurrence
    assert np.all(ft[:, 0] < np.where(ft[:, 1] >= 0, ft[:, 1], nE))   # T+ is the lower tet
    ids = fc["tet_face"] & 0x7FFFFFFF
    assert np.bincount(ids.ravel(), minlength=nF).tolist() == deg.tolist()
    # face ids follow first occurrence in (t, k) order
    first = np.where(fc["tet_face"].ravel() >= 0)[0]
    assert np.array_equal(fc["tet_face"].ravel()[first], np.arange(nF))


def test_neumann_marking_table2(golden_dir):
    """Table 2: L = interior + Dirichlet faces of the mixed problem."""
    rows = np.loadtxt(f"{golden_dir}/table2_sizes.txt", dtype=np.int64)
    for level in (1, 2, 3):
        p = meshgen.problem("paper_mixed", level)
        fc = oracle.faces(p.tet, p.nC, p.neumann)
        fm, L = oracle.multipliers(fc["face_kind"])
        r = rows[rows[:, 0] == level][0]
        assert (p.nE, fc["nF"], 4 * p.nE, L) == tuple(r[1:])


def test_faces_errors():
    coord, tet = meshgen.kuhn_cube(1)
    with pytest.raises(oracle.OracleError) as e:       # a face in three tets
        bad = np.vstack([tet, tet[:1]])
        oracle.faces(bad, coord.shape[0])
    assert e.value.name == "NONMANIFOLD"
    with pytest.raises(oracle.OracleError) as e:
        oracle.faces(np.array([[0, 1, 2, 9]]), 8)
    assert e.value.name == "ARG"
    with pytest.raises(oracle.OracleError) as e:
        oracle.faces(np.array([[0, 1, 1, 2]]), 8)
    assert e.value.name == "ARG"
    with pytest.raises(oracle.OracleError) as e:       # Neumann triple on an interior face
        fc = oracle.faces(tet, 8)
        inner = fc["face_vtx"][np.where(fc["face_tet"][:, 1] >= 0)[0][0]]
        oracle.faces(tet, 8, inner[None, :])
    assert e.value.name == "ARG"
    with pytest.raises(oracle.OracleError) as e:       # Neumann triple not in the mesh
        oracle.faces(tet, 8, np.array([[0, 1, 6]]))
    assert e.value.name == "ARG"
    fc = oracle.faces(np.zeros((0, 4), np.int32), 0)
    assert fc["nF"] == 0


def test_face_centroids_reference():
    """Ct = (P_x + P_y + P_z)/3 of each face tuple (Listing StiffMassPH)."""
    coord = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    fc = oracle.faces(np.array([[0, 1, 2, 3]]), 4)
    cen = oracle.face_centroids(coord, fc["face_vtx"])
    want = np.array([[1, 1, 0], [0, 1, 1], [1, 0, 1], [1, 1, 1]]) / 3.0
    assert np.array_equal(cen, want)
