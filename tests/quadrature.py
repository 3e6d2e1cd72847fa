"""Quadrature rules for error norms in the convergence checks (test utility).

Collapsed-coordinate (Duffy / Stroud conical product) rules built from
Gauss-Legendre points on [0, 1]:
  tetrahedron  x = u, y = v (1-u), z = w (1-u)(1-v),  Jacobian (1-u)^2 (1-v)
  triangle     x = u, y = v (1-u),                    Jacobian (1-u)
An n-point Gauss-Legendre factor integrates degree 2n-1 exactly, so the tet
rule is exact for polynomials of degree <= 2n-3 and the triangle rule for
degree <= 2n-2 (A. H. Stroud, Approximate Calculation of Multiple Integrals,
1971, Section 2.5).
"""
import numpy as np


def _gl01(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return (x + 1) / 2, w / 2


def tet_rule(n=8):
    """Barycentric points (q, 4) and weights (q,) summing to 1 (= |T| scale)."""
    x, w = _gl01(n)
    U, V, W = np.meshgrid(x, x, x, indexing="ij")
    WU, WV, WW = np.meshgrid(w, w, w, indexing="ij")
    px = U
    py = V * (1 - U)
    pz = W * (1 - U) * (1 - V)
    wt = WU * WV * WW * (1 - U) ** 2 * (1 - V) * 6.0     # reference volume 1/6 -> weights sum to 1
    px, py, pz, wt = px.ravel(), py.ravel(), pz.ravel(), wt.ravel()
    bary = np.stack([1 - px - py - pz, px, py, pz], axis=1)
    return bary, wt


def tri_rule(n=6):
    """Barycentric points (q, 3) and weights (q,) summing to 1 (= |F| scale)."""
    x, w = _gl01(n)
    U, V = np.meshgrid(x, x, indexing="ij")
    WU, WV = np.meshgrid(w, w, indexing="ij")
    px = U
    py = V * (1 - U)
    wt = (WU * WV * (1 - U) * 2.0).ravel()
    px, py = px.ravel(), py.ravel()
    return np.stack([1 - px - py, px, py], axis=1), wt
