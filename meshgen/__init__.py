"""Seeded synthetic inputs for the primal hybrid FEM path.

This module produces the *inputs* of the method and nothing else: tetrahedral
meshes of the unit cube (the paper's 5-tet cube of Listing 1 and Kuhn m^3
cubes), the paper's 1->12 red refinement (Section 3.4, Listing "RedRefine")
used to grow them, seeded vertex jitter, per-element coefficient fields, and the
analytic problem data f, u_D, g as plain functions of position.  It holds none
of the method's arithmetic (no face connectivity, no local matrices, no
condensation), so both the oracle and the CUDA path may take their inputs from
here.

Conventions: vertex ids are 0-based int32; ``tet`` is (nE, 4) int32; ``coord``
is (nC, 3) float64.  Local edges of a tet [I J K L] are taken in the paper's
order IJ, IK, IL, JK, JL, KL (Listing "NumEdges").
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Local edge order of a tet [I J K L]: IJ, IK, IL, JK, JL, KL (Listing NumEdges).
LOCAL_EDGES = np.array([[0, 1], [0, 2], [0, 3], [1, 2], [1, 3], [2, 3]], dtype=np.int64)


# --------------------------------------------------------------------------
# Base meshes
# --------------------------------------------------------------------------
def listing1_mesh():
    """The 5-tet unit cube of Listing 1 (Section 2.3), converted to 0-based ids.

    Returns (coord, tet, Db, Nb): Db holds the 2 Dirichlet faces (the z=1 side),
    Nb the 10 Neumann faces, each a vertex triple.
    """
    coord = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0],
                      [0, 0, 1], [1, 0, 1], [0, 1, 1], [1, 1, 1]], dtype=np.float64)
    tet = np.array([[1, 2, 3, 5], [5, 8, 6, 2], [7, 3, 8, 5], [4, 8, 3, 2], [8, 3, 2, 5]],
                   dtype=np.int32) - 1
    Db = np.array([[7, 8, 5], [5, 8, 6]], dtype=np.int32) - 1
    Nb = np.array([[1, 5, 2], [5, 6, 2], [1, 3, 5], [7, 5, 3], [7, 3, 8], [4, 8, 3],
                   [2, 6, 8], [4, 2, 8], [4, 3, 2], [1, 2, 3]], dtype=np.int32) - 1
    return coord, tet, Db, Nb


def kuhn_cube(m: int):
    """Unit cube split into m^3 subcubes, each into the 6 Kuhn tets.

    Subcube with corner v: tets [v, v+e_p1, v+e_p1+e_p2, v+(1,1,1)] over the 6
    permutations p of the axes.  All 6 share the main diagonal, so the
    triangulation is conforming across subcubes.
    """
    if m < 1:
        raise ValueError("m >= 1")
    n = m + 1
    g = np.arange(n, dtype=np.float64) / m
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    # vertex id = i + n*(j + n*k)
    coord = np.stack([X.transpose(2, 1, 0).ravel(), Y.transpose(2, 1, 0).ravel(),
                      Z.transpose(2, 1, 0).ravel()], axis=1)
    ii, jj, kk = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    base = (ii + n * (jj + n * kk)).transpose(2, 1, 0).ravel().astype(np.int64)
    step = np.array([1, n, n * n], dtype=np.int64)
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    tets = []
    for p in perms:
        v0 = base
        v1 = v0 + step[p[0]]
        v2 = v1 + step[p[1]]
        v3 = v0 + step.sum()
        tets.append(np.stack([v0, v1, v2, v3], axis=1))
    # subcube-major order: the 6 tets of one subcube are consecutive
    tet = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)
    return coord, tet


# --------------------------------------------------------------------------
# Red refinement (Section 3.4, Listing RedRefine) and boundary-face refinement
# --------------------------------------------------------------------------
def number_edges(tet: np.ndarray, nC: int):
    """Edge numbering of Listing NumEdges: edges of all tets, tet-major, local
    order IJ..KL, numbered by first occurrence ('stable' unique).

    Returns (U, edge_of) with U (nEd, 2) sorted vertex pairs in first-occurrence
    order and edge_of (nE, 6) the edge id of each local edge.
    """
    nE = tet.shape[0]
    e = tet.astype(np.int64)[:, LOCAL_EDGES]              # (nE, 6, 2)
    lo = np.minimum(e[..., 0], e[..., 1]).ravel()
    hi = np.maximum(e[..., 0], e[..., 1]).ravel()
    key = lo * np.int64(nC) + hi
    _, first, inv = np.unique(key, return_index=True, return_inverse=True)
    order = np.argsort(first, kind="stable")               # unique ids -> first-occurrence rank
    rank = np.empty_like(order)
    rank[order] = np.arange(order.size)
    edge_of = rank[inv].reshape(nE, 6)
    U = np.stack([lo[first[order]], hi[first[order]]], axis=1)
    return U, edge_of


def red_refine(coord: np.ndarray, tet: np.ndarray, faces_lists=()):
    """One level of the paper's 1->12 refinement (Listing RedRefine).

    New nodes: walking the tets in order, each tet contributes its centroid and
    then the midpoints of its not-yet-seen edges (IJ, IK, IL, JK, JL, KL), which
    is the node order that the listing's stable unique of [Ct M1..M6] gives.
    Child 1 replaces the parent; children 2..12 of parent t sit at
    nE + 11 t + (0..10) (0-based), as in the listing.  Each array in
    ``faces_lists`` (vertex triples, e.g. Db, Nb) is split 1->4 at edge
    midpoints (refineFaces).
    """
    coord = np.asarray(coord, dtype=np.float64)
    tet = np.asarray(tet)
    nC = coord.shape[0]
    nE = tet.shape[0]
    U, edge_of = number_edges(tet, nC)
    nEd = U.shape[0]
    T = tet.astype(np.int64)
    # first-occurrence flags of edge slots, tet-major
    flat = edge_of.ravel()
    seen_first = np.zeros(flat.size, dtype=bool)
    firstpos = np.full(nEd, -1, dtype=np.int64)
    # position of the first occurrence of each edge id
    order = np.argsort(flat, kind="stable")
    fo = order[np.r_[True, flat[order][1:] != flat[order][:-1]]]
    firstpos[flat[fo]] = fo
    seen_first[fo] = True
    cnt_before = np.cumsum(seen_first) - seen_first       # edges first seen strictly before slot
    tt = np.arange(nE, dtype=np.int64)
    cent_id = nC + tt + cnt_before[6 * tt]
    mid_id = np.empty(nEd, dtype=np.int64)
    mid_id[flat[fo]] = nC + fo // 6 + 1 + cnt_before[fo]
    nC_new = nC + nE + nEd
    new_coord = np.empty((nC_new, 3), dtype=np.float64)
    new_coord[:nC] = coord
    P = [coord[T[:, i]] for i in range(4)]
    new_coord[cent_id] = (P[0] + P[1] + P[2] + P[3]) / 4.0
    a = T[np.arange(nE)[:, None], LOCAL_EDGES[:, 0][None, :]].ravel()[fo]
    b = T[np.arange(nE)[:, None], LOCAL_EDGES[:, 1][None, :]].ravel()[fo]
    new_coord[mid_id[flat[fo]]] = (coord[a] + coord[b]) / 2.0

    A = mid_id[edge_of]          # (nE, 6): midpoint node of IJ, IK, IL, JK, JL, KL
    IJ, IK, IL, JK, JL, KL = (A[:, i] for i in range(6))
    I, J, K, L = (T[:, i] for i in range(4))
    C = cent_id
    kids = [
        (I, IJ, IK, IL),
        (J, JK, IJ, JL),
        (K, IK, JK, KL),
        (L, KL, JL, IL),
        (IJ, IK, IL, C),
        (JK, IJ, JL, C),
        (IK, JK, KL, C),
        (KL, JL, IL, C),
        (IJ, JK, IK, C),
        (IK, KL, IL, C),
        (IJ, IL, JL, C),
        (KL, JK, JL, C),
    ]
    out = np.empty((12 * nE, 4), dtype=np.int64)
    out[:nE] = np.stack(kids[0], axis=1)
    rest = np.stack([np.stack(k, axis=1) for k in kids[1:]], axis=1)   # (nE, 11, 4)
    out[nE:] = rest.reshape(-1, 4)
    new_lists = []
    if faces_lists:
        # edge lookup for boundary triples: midpoint id of the undirected edge (x, y)
        keyU = U[:, 0] * np.int64(nC) + U[:, 1]
        srt = np.argsort(keyU)
        keyS = keyU[srt]

        def mid(x, y):
            lo = np.minimum(x, y)
            hi = np.maximum(x, y)
            k = lo * np.int64(nC) + hi
            pos = np.searchsorted(keyS, k)
            if np.any(pos >= keyS.size) or np.any(keyS[np.minimum(pos, keyS.size - 1)] != k):
                raise ValueError("boundary face edge not in mesh")
            return mid_id[srt[pos]]

        for Fl in faces_lists:
            Fl = np.asarray(Fl, dtype=np.int64)
            if Fl.size == 0:
                new_lists.append(Fl.reshape(0, 3).astype(np.int32))
                continue
            n1, n2, n3 = Fl[:, 0], Fl[:, 1], Fl[:, 2]
            m12, m13, m23 = mid(n1, n2), mid(n1, n3), mid(n2, n3)
            nF = Fl.shape[0]
            o = np.empty((4 * nF, 3), dtype=np.int64)
            o[:nF] = np.stack([n1, m12, m13], axis=1)
            r = np.stack([np.stack([n2, m23, m12], axis=1),
                          np.stack([n3, m13, m23], axis=1),
                          np.stack([m12, m23, m13], axis=1)], axis=1)
            o[nF:] = r.reshape(-1, 3)
            new_lists.append(o.astype(np.int32))
    if nC_new >= 2 ** 31:
        raise OverflowError("vertex ids exceed int32")
    return new_coord, out.astype(np.int32), new_lists


def refined(coord, tet, levels: int, faces_lists=()):
    lists = list(faces_lists)
    for _ in range(levels):
        coord, tet, lists = red_refine(coord, tet, lists)
    return coord, tet, lists


# --------------------------------------------------------------------------
# Jitter and coefficient fields
# --------------------------------------------------------------------------
def _signed_vol6(coord, tet):
    P0, P1, P2, P3 = (coord[tet[:, i]] for i in range(4))
    return np.einsum("ij,ij->i", P1 - P0, np.cross(P2 - P0, P3 - P0))


def jitter_interior(coord, tet, frac=0.2, seed=3, min_ratio=0.1, max_rounds=12):
    """Move every interior vertex by a vector uniform in a ball of radius
    frac * (its shortest incident edge), seeded.  Tets whose signed volume
    changes sign or drops below ``min_ratio`` of its unjittered value get their
    vertices redrawn with the radius halved; after ``max_rounds`` the remaining
    offenders are left unmoved.  Returns (new_coord, n_redrawn_vertices).
    """
    coord = np.asarray(coord, dtype=np.float64)
    nC = coord.shape[0]
    rng = np.random.Generator(np.random.PCG64(seed))
    on_bnd = np.any((coord == 0.0) | (coord == 1.0), axis=1)
    e = tet.astype(np.int64)[:, LOCAL_EDGES].reshape(-1, 2)
    lens = np.linalg.norm(coord[e[:, 0]] - coord[e[:, 1]], axis=1)
    hv = np.full(nC, np.inf)
    np.minimum.at(hv, e[:, 0], lens)
    np.minimum.at(hv, e[:, 1], lens)
    radius = np.where(on_bnd, 0.0, frac * hv)

    def draw(idx, rad):
        d = rng.standard_normal((idx.size, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        r = rad * rng.random(idx.size) ** (1.0 / 3.0)
        return d * r[:, None]

    vol0 = _signed_vol6(coord, tet)
    disp = np.zeros_like(coord)
    idx = np.nonzero(radius > 0)[0]
    disp[idx] = draw(idx, radius[idx])
    newc = coord + disp
    v = _signed_vol6(newc, tet)
    redrawn = 0
    for rnd in range(max_rounds + 1):
        bad = ~(v / vol0 >= min_ratio)
        if not bad.any():
            return newc, redrawn
        verts = np.unique(tet[bad].ravel())
        verts = verts[radius[verts] > 0]
        redrawn += verts.size
        radius[verts] *= 0.5
        if rnd == max_rounds:
            disp[verts] = 0.0
        else:
            disp[verts] = draw(verts, radius[verts])
        newc[verts] = coord[verts] + disp[verts]
        # only tets touching a moved vertex change volume
        moved = np.zeros(nC, dtype=bool)
        moved[verts] = True
        touched = np.nonzero(moved[tet].any(axis=1))[0]
        v[touched] = _signed_vol6(newc, tet[touched])
    return newc, redrawn


def lognormal_field(nE: int, seed: int, sigma: float = 1.0):
    """a_K = exp(g_K), g_K iid N(0, sigma^2) from numpy PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.exp(sigma * rng.standard_normal(nE))


def checkerboard_field(coord, tet, blocks=8, lo=1.0, hi=1e4):
    """a_K in {lo, hi} on a blocks^3 checkerboard of the unit cube, chosen by
    the element centroid: block index floor(blocks * centroid) clamped to
    [0, blocks-1]; hi where i+j+k is odd."""
    cen = coord[tet.astype(np.int64)].mean(axis=1)
    b = np.clip(np.floor(blocks * cen).astype(np.int64), 0, blocks - 1)
    odd = (b.sum(axis=1) % 2) == 1
    return np.where(odd, hi, lo).astype(np.float64)


# --------------------------------------------------------------------------
# Analytic problem data (functions of position only)
# --------------------------------------------------------------------------
def sin_source(x, a=1.0, c=1.0):
    """f for u = sin(pi x) sin(pi y) sin(pi z) with constant a:
    -div(a grad u) + c u = (3 pi^2 a + c) u."""
    x = np.asarray(x, dtype=np.float64)
    u = np.sin(math.pi * x[..., 0]) * np.sin(math.pi * x[..., 1]) * np.sin(math.pi * x[..., 2])
    return (3.0 * math.pi ** 2 * a + c) * u


def sin_solution(x):
    x = np.asarray(x, dtype=np.float64)
    return np.sin(math.pi * x[..., 0]) * np.sin(math.pi * x[..., 1]) * np.sin(math.pi * x[..., 2])


def x2y2z2_solution(x):
    """The paper's manufactured solution u = x^2 y^2 z^2 (Section 4, Example)."""
    x = np.asarray(x, dtype=np.float64)
    return x[..., 0] ** 2 * x[..., 1] ** 2 * x[..., 2] ** 2


def x2y2z2_grad(x):
    x = np.asarray(x, dtype=np.float64)
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    return np.stack([2 * X * Y ** 2 * Z ** 2, 2 * X ** 2 * Y * Z ** 2, 2 * X ** 2 * Y ** 2 * Z], axis=-1)


def x2y2z2_source(x):
    """f = -Laplace(u) + u for u = x^2 y^2 z^2 (a = c = 1)."""
    x = np.asarray(x, dtype=np.float64)
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    return -2.0 * (Y ** 2 * Z ** 2 + X ** 2 * Z ** 2 + X ** 2 * Y ** 2) + X ** 2 * Y ** 2 * Z ** 2


def cube_outward_normal(x, tol=1e-12):
    """Outward unit normal of the unit cube at boundary points x (..., 3),
    chosen by the side the point lies on."""
    x = np.asarray(x, dtype=np.float64)
    n = np.zeros(x.shape)
    for d in range(3):
        n[..., d] = np.where(np.abs(x[..., d]) <= tol, -1.0, n[..., d])
        n[..., d] = np.where(np.abs(x[..., d] - 1.0) <= tol, 1.0, n[..., d])
    return n


# --------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------
@dataclass
class Problem:
    name: str
    coord: np.ndarray
    tet: np.ndarray
    a: np.ndarray                   # per-element coefficient (nE,)
    c: float
    f: object                       # callable f(x) -> values
    uD: object = None               # callable or None (zero Dirichlet)
    gN: object = None               # callable or None
    neumann: np.ndarray = field(default_factory=lambda: np.zeros((0, 3), np.int32))
    info: dict = field(default_factory=dict)

    @property
    def nE(self):
        return int(self.tet.shape[0])

    @property
    def nC(self):
        return int(self.coord.shape[0])


def problem(name: str, levels: int | None = None) -> Problem:
    """The synthetic workloads.

    - ``sin_kuhn``: Kuhn 1^3 cube refined 2 levels (864 tets), a=1, c=1,
      f from u=sin(pi x)sin(pi y)sin(pi z), zero Dirichlet on the whole boundary.
    - ``lognormal_3m``: Kuhn 3^3 cube refined 4 levels (3,359,232 tets),
      a_K = exp(N(0,1)) with seed 2, c=0.1, same f, zero Dirichlet.
    - ``jitter_checker_18m``: Kuhn 1^3 cube refined 6 levels (17,915,904 tets),
      interior vertices jittered by up to 0.2 h (seed 3), a_K in {1, 1e4} on an
      8^3 checkerboard, c=1, same f, zero Dirichlet.
    - ``paper_mixed``: the Listing-1 cube refined ``levels`` times with the
      paper's mixed boundary conditions (Dirichlet on z=1, Neumann elsewhere)
      and u = x^2 y^2 z^2 (Section 4, Example), a=c=1.
    - ``kuhn(m,k)`` style names ``kuhn_m{m}_k{k}``: a=1, c=1, sin data.
    """
    if name == "sin_kuhn":
        coord, tet = kuhn_cube(1)
        coord, tet, _ = refined(coord, tet, 2 if levels is None else levels)
        return Problem(name, coord, tet, np.ones(tet.shape[0]), 1.0,
                       lambda x: sin_source(x, 1.0, 1.0), info={"m": 1, "k": 2})
    if name == "lognormal_3m":
        coord, tet = kuhn_cube(3)
        coord, tet, _ = refined(coord, tet, 4 if levels is None else levels)
        return Problem(name, coord, tet, lognormal_field(tet.shape[0], 2), 0.1,
                       lambda x: sin_source(x, 1.0, 1.0), info={"m": 3, "k": 4, "seed": 2})
    if name == "jitter_checker_18m":
        coord, tet = kuhn_cube(1)
        coord, tet, _ = refined(coord, tet, 6 if levels is None else levels)
        coord, nred = jitter_interior(coord, tet, 0.2, seed=3)
        return Problem(name, coord, tet, checkerboard_field(coord, tet), 1.0,
                       lambda x: sin_source(x, 1.0, 1.0),
                       info={"m": 1, "k": 6, "seed": 3, "jitter_redrawn": int(nred)})
    if name == "paper_mixed":
        lv = 1 if levels is None else levels
        coord, tet, Db, Nb = listing1_mesh()
        coord, tet, (Db, Nb) = refined(coord, tet, lv, (Db, Nb))

        def g(x):
            return np.einsum("...i,...i->...", x2y2z2_grad(x), cube_outward_normal(x))

        return Problem(name, coord, tet, np.ones(tet.shape[0]), 1.0, x2y2z2_source,
                       uD=x2y2z2_solution, gN=g, neumann=Nb, info={"level": lv, "Db": Db})
    if name.startswith("kuhn_m"):
        m, k = name[len("kuhn_m"):].split("_k")
        coord, tet = kuhn_cube(int(m))
        coord, tet, _ = refined(coord, tet, int(k))
        return Problem(name, coord, tet, np.ones(tet.shape[0]), 1.0,
                       lambda x: sin_source(x, 1.0, 1.0), info={"m": int(m), "k": int(k)})
    raise KeyError(name)


def shuffled(coord, tet, seed: int):
    """Same mesh with vertices renumbered and tets reordered by a seeded
    permutation, and each tet's vertex tuple rotated by a seeded even/odd
    permutation: a stress input for connectivity (no refinement locality)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nC, nE = coord.shape[0], tet.shape[0]
    pv = rng.permutation(nC)
    inv = np.empty(nC, dtype=np.int64)
    inv[pv] = np.arange(nC)
    coord2 = coord[pv]
    tet2 = inv[tet.astype(np.int64)]
    tet2 = tet2[rng.permutation(nE)]
    perms = np.array([[0, 1, 2, 3], [1, 0, 2, 3], [2, 3, 0, 1], [3, 1, 2, 0], [0, 2, 3, 1], [1, 2, 0, 3]])
    choice = rng.integers(0, perms.shape[0], nE)
    tet2 = np.take_along_axis(tet2, perms[choice], axis=1)
    return coord2, tet2.astype(np.int32)
