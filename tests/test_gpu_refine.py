"""Device refinement (ph_refine) against the host generator, which follows
Listing RedRefine / refineFaces and is pinned by the refinement example of
Section 3.4 and Table 1: coordinates, tets and boundary lists bit-identical."""
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


def cu(x):
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


def check(ph, coord, tet, lists=()):
    """The device takes one list of triples: the concatenation of `lists`,
    refined as one list (refineFaces applied to it)."""
    L = np.vstack(lists).astype(np.int32) if lists else None
    c_ref, t_ref, l_ref = meshgen.red_refine(coord, tet, [L] if lists else [])
    c, t, l, nEd = ph.ph_refine(cu(coord), cu(tet.astype(np.int32)), None if L is None else cu(L))
    torch.cuda.synchronize()
    assert np.array_equal(t.cpu().numpy(), t_ref)
    assert np.array_equal(c.cpu().numpy().view(np.uint64), c_ref.view(np.uint64))
    assert nEd == meshgen.number_edges(tet, coord.shape[0])[0].shape[0]
    if lists:
        assert np.array_equal(l.cpu().numpy(), np.vstack(l_ref))
    return c, t, l


def test_paper_example(ph, golden_dir):
    coord = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    tet = np.array([[1, 3, 2, 4]], np.int32) - 1
    c, t, _ = check(ph, coord, tet)
    T = [l.split() for l in open(f"{golden_dir}/refine_example.txt") if l[:1].isdigit()]
    assert np.array_equal(t.cpu().numpy() + 1, np.array([list(map(int, r)) for r in T[:12]]))


def test_listing1_levels_with_boundary_lists(ph):
    coord, tet, Db, Nb = meshgen.listing1_mesh()
    lists = (Db, Nb)
    for _ in range(3):
        check(ph, coord, tet, lists)
        coord, tet, lists = meshgen.red_refine(coord, tet, list(lists))
        lists = tuple(lists)


@pytest.mark.parametrize("m,k", [(1, 0), (2, 1), (3, 2)])
def test_kuhn_and_shuffled(ph, m, k):
    coord, tet = meshgen.kuhn_cube(m)
    coord, tet, _ = meshgen.refined(coord, tet, k)
    check(ph, coord, tet)
    c2, t2 = meshgen.shuffled(coord, tet, 11)
    check(ph, c2, t2)


def test_chained_on_device_equals_host(ph):
    """Six levels chained on the device (the 17.9M-tet cube) equal the host
    generator's mesh."""
    coord, tet = meshgen.kuhn_cube(1)
    c, t = cu(coord), cu(tet)
    for _ in range(6):
        c, t, _, _ = ph.ph_refine(c, t)
    hc, ht, _ = meshgen.refined(coord, tet, 6)
    assert t.shape[0] == 17915904
    assert np.array_equal(t.cpu().numpy(), ht)
    assert np.array_equal(c.cpu().numpy().view(np.uint64), hc.view(np.uint64))


def test_bad_list_triple(ph):
    coord, tet = meshgen.kuhn_cube(1)
    with pytest.raises(ph.PHError) as e:
        ph.ph_refine(cu(coord), cu(tet), cu(np.array([[0, 1, 2]], np.int32)))   # 1-2 is not an edge
    assert e.value.name == "PH_ERR_ARG"
    bad = tet.copy()
    bad[3, 2] = bad[3, 1]                              # repeated vertex
    with pytest.raises(ph.PHError) as e:
        ph.ph_refine(cu(coord), cu(bad))
    assert e.value.name == "PH_ERR_ARG"
    c, t, l, nEd = ph.ph_refine(cu(coord), cu(tet[:0]))  # empty mesh: coordinates pass through
    assert t.shape[0] == 0 and nEd == 0 and torch.equal(c, cu(coord))
