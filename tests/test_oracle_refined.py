"""The oracle's refined solve and its one-ulp sensitivity measure, pinned on
systems whose answers are known exactly.

- A tridiagonal SPD matrix with integer entries (a 1D diffusion operator
  with coefficients alternating between 1 and 1e4 in blocks, condition number
  ~1e9) and an integer solution: b = H x is exact in fp64, so the refined
  solve must return x to the last bit's order (a plain fp64 solve does not),
  and the binary128 residual of the exact solution is exactly zero.
- A diagonal system: moving every entry by one ulp moves each solution
  component by at most two ulps, so the sensitivity sits between 2^-54 and
  3 * 2^-52 (no amplification without coupling).
"""
import numpy as np
import scipy.sparse as sp

import oracle


def tridiagonal(n=20000, seed=0):
    a = np.where((np.arange(n + 1) // 50) % 2 == 0, 1, 10000).astype(np.int64)
    main, off = a[:-1] + a[1:], -a[1:-1]
    Hi = sp.diags([off, main, off], [-1, 0, 1], format="csr", dtype=np.int64)
    Hi.sort_indices()
    x = np.random.default_rng(seed).integers(-1000, 1000, n).astype(np.int64)
    b = (Hi @ x).astype(np.float64)  # integers below 2^53: exact
    return Hi.indptr.astype(np.int32), Hi.indices.astype(np.int32), Hi.data.astype(np.float64), b, x.astype(float)


def test_refined_solve_recovers_the_exact_solution():
    rp, ci, va, b, x = tridiagonal()
    assert np.all(oracle.residual(rp, ci, va, x, b) == 0.0)
    plain = oracle.solve(rp, ci, va, b)
    ref, steps, corr = oracle.solve_refined(rp, ci, va, b)
    nx = np.linalg.norm(x)
    assert np.linalg.norm(plain - x) / nx > 1e-11        # what refinement is for
    assert np.linalg.norm(ref - x) / nx <= 2.0 ** -52
    assert np.max(np.abs(ref - x)) <= 2.0 ** -52 * np.max(np.abs(x))
    assert 1 <= steps <= 6 and corr <= 2.0 ** -53


def test_residual_is_binary128_accurate():
    """b - H x for x = exact + one-ulp nudges: the binary128 residual equals
    the exact one (computed with Python integers and fractions)."""
    from fractions import Fraction
    rp, ci, va, b, x = tridiagonal(n=300, seed=3)
    xn = np.nextafter(x, np.inf)
    r = oracle.residual(rp, ci, va, xn, b)
    for i in range(0, 300, 7):
        exact = Fraction(b[i]) - sum(Fraction(va[j]) * Fraction(xn[ci[j]]) for j in range(rp[i], rp[i + 1]))
        assert r[i] == float(exact)


def test_ulp_sensitivity_of_a_diagonal_system():
    n = 500
    d = np.random.default_rng(1).uniform(0.5, 2.0, n)
    b = np.random.default_rng(2).standard_normal(n)
    rp = np.arange(n + 1, dtype=np.int32)
    ci = np.arange(n, dtype=np.int32)
    s = oracle.ulp_sensitivity(rp, ci, d, b, trials=3)
    assert 2.0 ** -54 <= s <= 3 * 2.0 ** -52
