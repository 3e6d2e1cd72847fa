"""The hand-written adjoint (ph_adjoint_rhs / ph_adjoint_grad behind
MisfitFunction) against the oracle's adjoint, against its own autograd path,
and against central finite differences.

Full-size checks use the adjoint workload (Kuhn 6^3 cube refined 3 levels,
2,239,488 tets, c = 0.1, U_obs from a lognormal a with seed 5, gradient at a
lognormal a with seed 51): a Taylor check along a random direction, and
central differences on 20 random elements (four global solves each, with the
edge-patch Schwarz preconditioner; PH_FD_SMALL=1 runs them on a 279,936-tet
mesh of the same recipe instead).  Each difference is computed by difference
solves: with a' = a except
a'_t = a_t e^{+-eps},
      H' dLambda = dr - dH Lambda        (dr, dH: element t's changes only),
      dU = A'^-1 C' dLambda  (plus element t's own change of A^-1),
      dJ = sum_T e' M dU + 1/2 dU' M dU,
  so that no difference of two full solves is ever taken.
"""
import numpy as np
import pytest

import meshgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LF = [(0, 1, 2), (0, 2, 3), (0, 3, 1), (3, 2, 1)]


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


class Setup:
    def __init__(self, ph, p, a, U_obs):
        self.ph, self.p = ph, p
        neu = cu(p.neumann.astype(np.int32)) if p.neumann.size else None
        self.mesh = ph.Mesh(cu(p.coord), cu(p.tet.astype(np.int32)), neu)
        fcd = self.mesh.faces()
        self.fc = {k: v.cpu().numpy() for k, v in fcd.items()}
        cen = self.fc["face_centroid"]
        self.f = cu(np.asarray(p.f(cen), np.float64))
        self.uD = None if p.uD is None else cu(np.asarray(p.uD(cen), np.float64))
        self.gN = None if p.gN is None else cu(np.asarray(p.gN(cen), np.float64))
        self.rowptr, self.colind = self.mesh.csr_pattern()
        self.a = cu(a)
        self.U_obs = cu(U_obs)

    precond = "schwarz"

    def solve(self, values, rhs, rtol, P=None):
        lam, it, P = self.ph.solve_system(self.mesh, values, rhs, rtol, 200000, self.precond, P)
        return lam, it, P

    def forward(self, a, rtol=1e-12, keep_P=False):
        m = self.mesh
        values, rhs, factor = m.assemble(a, self.p.c, self.f, self.uD, self.gN, factor=True)
        lam, it, P = self.solve(values, rhs, rtol)
        u = m.recover_factored(factor, self.p.c, self.f, lam, self.gN)
        out = dict(values=values, rhs=rhs, factor=factor, lam=lam, u=u, J=m.misfit(u, self.U_obs), iters=it)
        if keep_P:
            out["P"] = P
        elif P is not None:
            P.close()
        return out

    def gradient(self, a, rtol=1e-12):
        fw = self.forward(a, rtol, keep_P=True)
        m = self.mesh
        rq = m.adjoint_rhs(fw["factor"], self.p.c, fw["u"], self.U_obs)
        q, _, P = self.solve(fw["values"], rq, rtol, fw.pop("P"))
        if P is not None:
            P.close()
        g = m.adjoint_grad(a, fw["factor"], self.p.c, fw["u"], self.U_obs, q)
        return fw, g


def obs_field(ph, p, seed):
    s = Setup(ph, p, meshgen.lognormal_field(p.nE, seed), np.zeros((p.nE, 4)))
    u = s.forward(s.a)["u"].cpu().numpy()
    s.mesh.close()
    return u


@pytest.mark.parametrize("precond", ["schwarz", "jacobi"])
@pytest.mark.parametrize("case", ["kuhn_m1_k1", "paper_mixed1", "kuhn_m2_k1"])
def test_adjoint_matches_oracle(ph, case, precond):
    if case == "paper_mixed1":
        p = meshgen.problem("paper_mixed", 1)
    else:
        p = meshgen.problem(case)
        p.c = 0.3
    # the observation: the oracle's own forward solve at another coefficient
    U_obs = oracle.pipeline(p.coord, p.tet, meshgen.lognormal_field(p.nE, 51), p.c, p.f, p.uD, p.gN,
                            p.neumann if p.neumann.size else None)["U"]
    a = meshgen.lognormal_field(p.nE, 5)
    s = Setup(ph, p, a, U_obs)
    s.precond = precond
    fw, g = s.gradient(s.a)
    J_o, g_o, U_o, _ = oracle.adjoint_gradient(p.coord, p.tet, a, p.c, p.f, U_obs, p.uD, p.gN, p.neumann)
    assert abs(fw["J"].item() - J_o) <= 1e-9 * abs(J_o)
    g = g.cpu().numpy()
    assert np.linalg.norm(g - g_o) <= 1e-9 * np.linalg.norm(g_o)
    # the misfit kernel on the oracle's own U
    Jm = s.mesh.misfit(cu(U_o), s.U_obs).item()
    assert abs(Jm - oracle.misfit(p.coord, p.tet, U_o, U_obs)) <= 1e-13 * abs(J_o)
    s.mesh.close()


def test_autograd_function(ph):
    p = meshgen.problem("kuhn_m2_k1")
    p.c = 0.5
    U_obs = obs_field(ph, p, 3)
    a = meshgen.lognormal_field(p.nE, 4)
    s = Setup(ph, p, a, U_obs)
    theta = torch.log(s.a).clone().requires_grad_(True)
    J = ph.misfit(theta, s.mesh, p.c, s.f, s.U_obs, rtol=1e-12)
    (gt,) = torch.autograd.grad(J, theta)
    _, g = s.gradient(torch.exp(theta.detach()), rtol=1e-12)
    assert torch.equal(gt, g)                      # same kernels, same inputs
    J2 = ph.misfit(theta, s.mesh, p.c, s.f, s.U_obs, rtol=1e-12)
    assert torch.equal(J2, J)
    (J2 * 3.0).backward()
    assert torch.allclose(theta.grad, 3.0 * g, rtol=1e-15, atol=0)
    s.mesh.close()


# ---------------------------------------------------------------------------
# full size
# ---------------------------------------------------------------------------
BIG_RTOL = 1e-10      # PCG residual of the gradient workload
FD_SOLVE_RTOL = 1e-12  # gradient and difference solves of the central-difference check
TAYLOR_RTOL = 1e-3
FD_RTOL = 2e-6


def make_adjoint_setup(ph, name, rtol=BIG_RTOL):
    p = meshgen.problem(name)
    p.c = 0.1
    s0 = Setup(ph, p, meshgen.lognormal_field(p.nE, 5), np.zeros((p.nE, 4)))
    U_obs = s0.forward(s0.a, rtol=rtol)["u"].cpu().numpy()
    s0.mesh.close()
    s = Setup(ph, p, meshgen.lognormal_field(p.nE, 51), U_obs)
    s.rtol = rtol
    fw, g = s.gradient(s.a, rtol=rtol)
    return s, fw, g.cpu().numpy()


@pytest.fixture(scope="module")
def big(ph):
    return make_adjoint_setup(ph, "kuhn_m6_k3")


def test_full_size_taylor(big):
    s, fw, g = big
    assert s.p.nE == 2239488
    d = np.random.default_rng(8).standard_normal(s.p.nE)
    theta = np.log(s.a.cpu().numpy())
    gd = g @ d
    fd = []
    for h in (1e-3, 5e-4):
        Jp = s.forward(cu(np.exp(theta + h * d)), rtol=BIG_RTOL)["J"].item()
        Jm = s.forward(cu(np.exp(theta - h * d)), rtol=BIG_RTOL)["J"].item()
        fd.append((Jp - Jm) / (2 * h))
    rich = (4 * fd[1] - fd[0]) / 3
    print("taylor: fd", fd, "richardson", rich, "adjoint", gd, "rel", abs(rich - gd) / abs(gd))
    # bounded by the accuracy of the solves (Jacobi PCG: true residual ~1e-10
    # on this system), not by the adjoint algebra
    assert abs(rich - gd) <= TAYLOR_RTOL * abs(gd), (rich, gd)


def _element_rows(s, t):
    tf = s.fc["tet_face"][t]
    F = tf & 0x7FFFFFFF
    l = s.fc["face_mult"][F]
    rowptr = s.rowptr_h
    colind = s.colind_h
    pos = np.zeros((4, 4), np.int64)
    for k in range(4):
        cols = colind[rowptr[l[k]]:rowptr[l[k] + 1]]
        for mm in range(4):
            pos[k, mm] = rowptr[l[k]] + int(np.searchsorted(cols, l[mm]))
    return l, pos


def _masses(s):
    P = s.p.coord[s.p.tet.astype(np.int64)]
    vol = np.abs(np.linalg.det(P[:, 1:] - P[:, :1])) / 6
    return vol


def _dJ(s, e, vol, dU):
    """sum_T e' M dU + 1/2 dU' M dU with M = |T|/20 (I + J), evaluated only
    where dU is nonzero."""
    nz = np.nonzero(np.abs(dU).max(axis=1) > 0)[0]
    ee, dd, v = e[nz], dU[nz], vol[nz] / 20
    lin = v * ((ee * dd).sum(1) + ee.sum(1) * dd.sum(1))
    quad = 0.5 * v * ((dd * dd).sum(1) + dd.sum(1) ** 2)
    return float(np.sum(lin + quad))


def _difference_solve(s, fw, t, eps):
    ph, m, p = s.ph, s.mesh, s.p
    a = s.a.clone()
    a[t] = a[t] * float(np.exp(eps))
    values2, rhs2, factor2 = m.assemble(a, p.c, s.f, s.uD, s.gN, factor=True)
    l, pos = _element_rows(s, t)
    v1, v2 = fw["values_h"], values2.cpu().numpy()
    r1, r2 = fw["rhs_h"], rhs2.cpu().numpy()
    lam = fw["lam_h"]
    dS = v2[pos] - v1[pos]
    rho = (r2[l] - r1[l]) - dS @ lam[l]
    rhs_loc = torch.zeros(m.L, dtype=torch.float64, device="cuda")
    rhs_loc[torch.as_tensor(l, device="cuda")] = cu(rho)
    dlam, _, P = s.solve(values2, rhs_loc, s.rtol)
    if P is not None:
        P.close()
    zero_f = torch.zeros_like(s.f)
    dU = m.recover_factored(factor2, p.c, zero_f, dlam).cpu().numpy()
    # element t: its own A changes too
    u_t_new = m.recover_factored(factor2, p.c, s.f, fw["lam"])[t].cpu().numpy()
    dU[t] += u_t_new - fw["u_h"][t]
    return _dJ(s, fw["e"], fw["vol"], dU)


@pytest.fixture(scope="module")
def fd_case(ph):
    """The full adjoint workload at the tighter solve tolerance (elements whose
    gradient is far below the typical one need it); PH_FD_SMALL=1: the
    279,936-tet mesh of the same recipe, for a quick run."""
    import os
    name = "kuhn_m3_k3" if os.environ.get("PH_FD_SMALL") == "1" else "kuhn_m6_k3"
    return make_adjoint_setup(ph, name, FD_SOLVE_RTOL)


def test_central_differences_20_elements(fd_case):
    s, fw, g = fd_case
    s.rowptr_h, s.colind_h = s.rowptr.cpu().numpy(), s.colind.cpu().numpy()
    fw["values_h"], fw["rhs_h"] = fw["values"].cpu().numpy(), fw["rhs"].cpu().numpy()
    fw["lam_h"], fw["u_h"] = fw["lam"].cpu().numpy(), fw["u"].cpu().numpy()
    fw["e"] = fw["u_h"] - s.U_obs.cpu().numpy()
    fw["vol"] = _masses(s)
    rng = np.random.default_rng(20)
    # Each difference dJ is a sum over all elements of terms that largely
    # cancel, so it carries an absolute rounding floor (~1e-20 here, i.e.
    # ~1e-17 on a difference quotient).  It shows only on elements whose
    # gradient is far below the typical one, so errors are measured against
    # max(|g_t|, rms(g)/10).
    scale_floor = np.sqrt(np.mean(g * g)) / 10
    worst = 0.0
    for t in rng.choice(s.p.nE, 20, replace=False):
        fd = []
        for eps in (1e-3, 5e-4):
            fd.append((_difference_solve(s, fw, t, eps) - _difference_solve(s, fw, t, -eps)) / (2 * eps))
        rich = (4 * fd[1] - fd[0]) / 3
        err = abs(rich - g[t]) / max(abs(g[t]), scale_floor)
        worst = max(worst, err)
        print("element", t, "fd", fd, "richardson", rich, "adjoint", g[t], "rel", err)
    print("worst relative FD error", worst)
    assert worst <= FD_RTOL
