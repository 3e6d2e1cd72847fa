"""Pins of the oracle's adjoint gradient: central finite differences of the
misfit computed by independent forward solves, and the Taylor remainder."""
import numpy as np
import pytest

import meshgen
import oracle


def _forward_J(p, a, U_obs):
    r = oracle.pipeline(p.coord, p.tet, a, p.c, p.f, p.uD, p.gN, p.neumann)
    return oracle.misfit(p.coord, p.tet, r["U"], U_obs), r


def _obs(p, seed):
    a_obs = meshgen.lognormal_field(p.nE, seed)
    r = oracle.pipeline(p.coord, p.tet, a_obs, p.c, p.f, p.uD, p.gN, p.neumann)
    return r["U"]


@pytest.mark.parametrize("case", ["kuhn_m1_k1", "paper_mixed1"])
def test_adjoint_matches_central_differences(case):
    if case == "paper_mixed1":
        p = meshgen.problem("paper_mixed", 1)
    else:
        p = meshgen.problem(case)
        p.c = 0.3
    U_obs = _obs(p, 51)
    theta = np.log(meshgen.lognormal_field(p.nE, 5))
    J, g, U, _ = oracle.adjoint_gradient(p.coord, p.tet, np.exp(theta), p.c, p.f, U_obs, p.uD, p.gN, p.neumann)
    J2, _ = _forward_J(p, np.exp(theta), U_obs)
    assert abs(J - J2) <= 1e-12 * abs(J)          # monolithic and condensed forward agree
    rng = np.random.default_rng(2)
    for t in rng.choice(p.nE, 6, replace=False):
        fd = []
        for eps in (1e-3, 5e-4):
            th_p, th_m = theta.copy(), theta.copy()
            th_p[t] += eps
            th_m[t] -= eps
            Jp, _ = _forward_J(p, np.exp(th_p), U_obs)
            Jm, _ = _forward_J(p, np.exp(th_m), U_obs)
            fd.append((Jp - Jm) / (2 * eps))
        rich = (4 * fd[1] - fd[0]) / 3              # Richardson: O(eps^4)
        assert abs(rich - g[t]) <= 1e-6 * abs(g).max(), (t, rich, g[t])


def test_adjoint_taylor_remainder():
    """J(theta + h d) - J(theta) - h g'd = O(h^2) along a random direction."""
    p = meshgen.problem("kuhn_m1_k1")
    U_obs = _obs(p, 61)
    theta = np.log(meshgen.lognormal_field(p.nE, 7))
    J0, g, _, _ = oracle.adjoint_gradient(p.coord, p.tet, np.exp(theta), p.c, p.f, U_obs)
    d = np.random.default_rng(3).standard_normal(p.nE)
    rem = []
    for h in (1e-2, 5e-3, 2.5e-3):
        Jh, _ = _forward_J(p, np.exp(theta + h * d), U_obs)
        rem.append(abs(Jh - J0 - h * g @ d))
    rates = np.log2(np.array(rem[:-1]) / np.array(rem[1:]))
    assert np.all(rates > 1.8), rates
