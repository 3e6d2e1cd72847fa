"""Pins of the oracle's per-element matrices and condensation (Section 4.2,
Eq. schur) against closed forms, invariances and exact identities."""
import math

import numpy as np
import pytest

import oracle

REF = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
LFACE = [(0, 1, 2), (0, 2, 3), (0, 3, 1), (3, 2, 1)]
OPP = [3, 1, 2, 0]          # local vertex opposite local face k


def test_reference_tet_matrices():
    m = oracle.tet_matrices(REF)
    K = np.array([[3, -1, -1, -1], [-1, 1, 0, 0], [-1, 0, 1, 0], [-1, 0, 0, 1]]) / 6
    M = (np.eye(4) + np.ones((4, 4))) / 120
    assert np.allclose(m["K"], K, rtol=0, atol=1e-16)
    assert np.allclose(m["M"], M, rtol=0, atol=1e-18)
    assert np.allclose(m["area"], [0.5, 0.5, 0.5, math.sqrt(3) / 2], rtol=1e-16, atol=0)
    assert m["vol"] == pytest.approx(1 / 6, rel=1e-16)
    # C(T) rows: sigma_k |F_k| r_k, r_k = 1/3 on the face's vertices (Eq. C(T))
    for k in range(4):
        for j in range(4):
            want = m["area"][k] / 3 if j in LFACE[k] else 0.0
            assert m["C"][k, j] == pytest.approx(want, rel=1e-16, abs=0)


@pytest.mark.parametrize("a,c", [(1.0, 1.0), (3.0, 0.25), (1e4, 1.0), (0.01, 5.0)])
def test_reference_tet_condensed_closed_form(a, c):
    S, _ = oracle.tet_local(REF, a, c, [0, 0, 0, 0], [1, 1, 1, 1])
    D = 1600 * a * a + 100 * a * c + c * c
    s00 = 4 * (1800 * a * a + 250 * a * c + 3 * c * c) / (3 * c * D)
    s01 = 2 * (3600 * a * a + 100 * a * c + c * c) / (3 * c * D)
    s03 = 2 * math.sqrt(3) * (180 * a + c) / (3 * c * (80 * a + c))
    s33 = 12 * (30 * a + c) / (c * (80 * a + c))
    want = np.array([[s00, s01, s01, s03], [s01, s00, s01, s03], [s01, s01, s00, s03], [s03, s03, s03, s33]])
    assert np.allclose(S, want, rtol=4e-16 * 8, atol=0)


def test_reference_tet_rational_values(golden_dir):
    S, _ = oracle.tet_local(REF, 1.0, 1.0, [0, 0, 0, 0], [1, 1, 1, 1])
    assert S[0, 0] == pytest.approx(8212 / 5103, rel=2e-16)
    assert S[0, 1] == pytest.approx(7402 / 5103, rel=2e-16)
    assert S[0, 3] == pytest.approx(362 * math.sqrt(3) / 243, rel=4e-16)
    assert S[3, 3] == pytest.approx(124 / 27, rel=2e-16)


def rand_tet(rng, h=1.0):
    while True:
        P = rng.standard_normal((4, 3)) * h
        v = np.dot(P[1] - P[0], np.cross(P[2] - P[0], P[3] - P[0]))
        if abs(v) > 0.05 * h ** 3:
            return P


def test_vertex_permutation_covariance():
    """Relabelling the vertices relabels the faces; S and g follow."""
    rng = np.random.default_rng(11)
    perms = [[1, 0, 2, 3], [2, 3, 0, 1], [3, 1, 2, 0], [1, 2, 3, 0], [0, 3, 1, 2]]
    for _ in range(10):
        P = rand_tet(rng)
        sig = rng.choice([-1, 1], 4)
        f = rng.standard_normal(4)
        a, c = float(rng.uniform(0.1, 10)), float(rng.uniform(0.1, 10))
        S, g = oracle.tet_local(P, a, c, f, sig)
        for p in perms:
            P2 = P[p]
            # face k of the relabelled tet is opposite vertex p[OPP[k]] of the original
            src = [OPP.index(p[OPP[k]]) for k in range(4)]
            S2, g2 = oracle.tet_local(P2, a, c, f[src], sig[src])
            assert np.allclose(S2, S[np.ix_(src, src)], rtol=1e-14, atol=0)
            assert np.allclose(g2, g[src], rtol=1e-13, atol=1e-15 * np.abs(g).max())


def test_rigid_motion_and_scaling():
    """S is invariant under rotation + translation, and S(lam P; a, c) =
    lam S(P; a/lam^2, c) (K ~ lam, M ~ lam^3, C ~ lam^2)."""
    rng = np.random.default_rng(5)
    for _ in range(5):
        P = rand_tet(rng)
        sig = rng.choice([-1, 1], 4)
        a, c = 2.0, 0.7
        S, _ = oracle.tet_local(P, a, c, np.zeros(4), sig)
        Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
        S2, _ = oracle.tet_local(P @ Q.T + rng.standard_normal(3), a, c, np.zeros(4), sig)
        assert np.allclose(S2, S, rtol=1e-13, atol=0)
        lam = 0.125
        S3, _ = oracle.tet_local(lam * P, a, c, np.zeros(4), sig)
        S4, _ = oracle.tet_local(P, a / lam ** 2, c, np.zeros(4), sig)
        assert np.allclose(S3, lam * S4, rtol=1e-14, atol=0)


def test_constant_load_identity():
    """f = f0 gives A (f0/c) 1 = B (K 1 = 0, M 1 = |T|/4 1), hence
    g = -C A^-1 B = -(f0/c) sigma |F|."""
    rng = np.random.default_rng(3)
    for _ in range(10):
        P = rand_tet(rng, h=rng.uniform(1e-3, 1))
        sig = rng.choice([-1, 1], 4)
        f0, a, c = 2.5, float(rng.uniform(0.01, 1e3)), float(rng.uniform(0.01, 10))
        _, g = oracle.tet_local(P, a, c, [f0] * 4, sig)
        area = oracle.tet_matrices(P)["area"]
        assert np.allclose(g, -(f0 / c) * sig * area, rtol=1e-14, atol=0)


def test_symmetric_positive_definite():
    rng = np.random.default_rng(9)
    for _ in range(20):
        P = rand_tet(rng)
        S, _ = oracle.tet_local(P, float(rng.uniform(0.1, 10)), 0.3, np.zeros(4), rng.choice([-1, 1], 4))
        assert np.array_equal(S, S.T) or np.allclose(S, S.T, rtol=1e-15, atol=0)
        assert np.linalg.eigvalsh(S).min() > 0


def test_neumann_rows_and_load():
    """A Neumann face has no multiplier (zero row/column) and adds
    |F| g phi_j(Ct) to B (Section 4.3, LN)."""
    P = REF
    S, g = oracle.tet_local(P, 1.0, 1.0, np.zeros(4), [1, 1, 1, 1], kind4=[0, 2, 0, 0], g4=[0, 3.0, 0, 0])
    assert np.all(S[1, :] == 0) and np.all(S[:, 1] == 0) and g[1] == 0
    # compare with the Dirichlet version driven by an equivalent load
    m = oracle.tet_matrices(P)
    B = np.array([m["area"][1] * 3.0 / 3 if j in LFACE[1] else 0.0 for j in range(4)])
    A = m["K"] + m["M"]
    C = m["C"].copy()
    C[1] = 0
    want = -C @ np.linalg.solve(A, B)
    assert np.allclose(g, want, rtol=1e-13, atol=1e-15)


def test_quad_accuracy_against_mpmath():
    """Precision check: on badly conditioned elements (a/(c h^2) ~ 1e9) the
    quad evaluation matches a 50-digit evaluation of C A^-1 C' to ~1 ulp."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    rng = np.random.default_rng(1)
    for _ in range(4):
        P = rand_tet(rng, h=3e-3)
        sig = rng.choice([-1, 1], 4)
        a, c = 1e4, 1.0
        S, _ = oracle.tet_local(P, a, c, np.zeros(4), sig)
        Pm = [[mp.mpf(float(x)) for x in row] for row in P]
        Gm = mp.matrix(4, 4)
        for j in range(4):
            Gm[0, j] = 1
            for d in range(3):
                Gm[d + 1, j] = Pm[j][d]
        vol = abs(mp.det(Gm)) / 6
        Gi = Gm ** -1
        G = [[Gi[i, d + 1] for d in range(3)] for i in range(4)]
        A = mp.matrix(4, 4)
        for i in range(4):
            for j in range(4):
                A[i, j] = a * vol * sum(G[i][d] * G[j][d] for d in range(3)) + c * vol / 20 * (2 if i == j else 1)
        C = mp.matrix(4, 4)
        for k in range(4):
            x, y, z = (Pm[i] for i in LFACE[k])
            u = [z[d] - x[d] for d in range(3)]
            v = [y[d] - x[d] for d in range(3)]
            cr = [u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]]
            ar = mp.sqrt(sum(q * q for q in cr)) / 2
            for j in range(4):
                C[k, j] = int(sig[k]) * ar / 3 if j in LFACE[k] else 0
        Sm = C * (A ** -1) * C.T
        for k in range(4):
            for m_ in range(4):
                ref = float(Sm[k, m_])
                assert abs(S[k, m_] - ref) <= 2.3e-16 * abs(ref)


def test_tet_recover_inverts_the_local_system():
    """U = A^-1 (B + C' lam) satisfies A U = B + C' lam (checked with the
    separately exported A, C, B of the same element)."""
    rng = np.random.default_rng(21)
    for _ in range(10):
        P = rand_tet(rng)
        sig = rng.choice([-1, 1], 4)
        f, lam = rng.standard_normal(4), rng.standard_normal(4)
        U = oracle.tet_recover(P, 1.0, 1.0, f, sig, lam)
        m = oracle.tet_matrices(P, f, sig)
        A = m["K"] + m["M"]
        assert np.allclose(A @ U, m["B"] + m["C"].T @ lam, rtol=1e-12, atol=1e-14 * np.abs(A @ U).max())
