"""Pins of the oracle's HDG pipeline (Sections 3-6, 9) against what the mathematics fixes.

* closed forms of the blocks: M_1^K = |K| I (orthonormal basis), tauDD = diag(T_l) (x) I,
  C_*^K against direct quadrature of int_K P_i d_* P_j with physical gradients;
* C^K symmetric, positive semi-definite, the energy identity
  u^T C u = (kappa^-1 q, q) + (c u, u) + <tau (u - u_hat), u - u_hat>  (from eq. 1.2a-b),
  and C^K 1 = 0 when c = 0 (u_hat = 1 gives u = 1, q = 0);
* eq. 6.3 reproduces P_k Dirichlet data; eq. 6.4 for constant g_N;
* brute force: the hybridised solution equals the dense solve of the full system eq. 1.2;
* exactness (the paper's closing remark on exact polynomial solutions): u in P_k, kappa
  constant, variable c -> q_h, u_h, u_hat are the projections of q, u and u* = u;
* observed convergence orders k+1 (q, u, u_hat) and k+2 (u*) as in Tables 2-3;
* a planted copy of the eq. 5.1 misprint (C_y for C_z) is caught by the exactness pin.
"""
import numpy as np
import pytest

from oracle import basis, hdg, quadrature
from oracle.geometry import ExpandedMesh
from workloads import boundary_faces, get_problem, kuhn_cube
from workloads.problems import Problem


def _setup(s, k, prob=None, jitter=0.15, mixed=True):
    c, e = kuhn_cube(s, jitter=jitter, seed=5)
    cls = (lambda ax, v: "D" if ax == 0 else "N") if mixed else (lambda ax, v: "D")
    d, n = boundary_faces(c, e, cls)
    m = ExpandedMesh(c, e, d, n)
    tab = hdg.Tables(k)
    return m, tab


def _varcoef():
    return (lambda x, y, z: 1 + 0.5 * np.sin(2 * x) * np.cos(y + z),
            lambda x, y, z: 1 + x ** 2 + 0.3 * y)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_block_closed_forms(k):
    m, tab = _setup(2, k)
    X, Y, Z = hdg.volume_nodes(m, tab)
    one = np.ones_like(X)
    blk = hdg.local_blocks(m, tab, one, 3.0 * one, one, tau=2.0)
    I = np.eye(tab.n)
    assert np.allclose(blk["M_kinv"], m.volume[:, None, None] * I, atol=1e-15)
    assert np.allclose(blk["M_c"], 3 * m.volume[:, None, None] * I, atol=1e-15)
    T = 2.0 * m.elem_area
    tDD = np.zeros_like(blk["tDD"])
    for l in range(4):
        tDD[:, l * tab.d2:(l + 1) * tab.d2, l * tab.d2:(l + 1) * tab.d2] = T[:, l, None, None] * np.eye(tab.d2)
    assert np.allclose(blk["tDD"], tDD, atol=1e-15)
    # C_* by direct quadrature with physical gradients B^-T grad_hat
    Binv_T = np.linalg.inv(m.B).transpose(0, 2, 1)
    grad = np.einsum("eab,bqi->eaqi", Binv_T, tab.Pstar)
    for s in range(3):
        direct = m.volume[:, None, None] * np.einsum("q,qi,eqj->eij", tab.w, tab.P, grad[:, s])
        assert np.allclose(blk["C"][s], direct, atol=1e-14)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_condensed_symmetry_energy_nullvector(k):
    m, tab = _setup(2, k)
    X, Y, Z = hdg.volume_nodes(m, tab)
    kap_f, c_f = _varcoef()
    kap, cq = kap_f(X, Y, Z), c_f(X, Y, Z)
    rng = np.random.default_rng(2)
    tau = rng.uniform(0.5, 2.0, size=(m.nelt, 4))
    blk = hdg.local_blocks(m, tab, kap, cq, np.zeros_like(X), tau=tau)
    CK, Cf, X2, xf = hdg.local_solvers(blk)
    scale = np.abs(CK).max()
    assert np.abs(CK - CK.transpose(0, 2, 1)).max() < 1e-13 * scale
    assert np.linalg.eigvalsh(0.5 * (CK + CK.transpose(0, 2, 1))).min() > -1e-12 * scale
    # energy identity for a random u_hat, f = 0
    uh = rng.normal(size=(m.nelt, 4 * tab.d2))
    sol = -np.einsum("eij,ej->ei", X2, uh)
    n = tab.n
    q = sol[:, :3 * n].reshape(-1, 3, n)
    u = sol[:, 3 * n:]
    lhs = np.einsum("ei,eij,ej->e", uh, CK, uh)
    e_q = sum(np.einsum("ei,eij,ej->e", q[:, a], blk["M_kinv"], q[:, a]) for a in range(3))
    e_c = np.einsum("ei,eij,ej->e", u, blk["M_c"], u)
    e_t = (np.einsum("ei,eij,ej->e", u, blk["tPP"], u)
           - 2 * np.einsum("ei,eji,ej->e", u, blk["tDP"], uh)
           + np.einsum("ei,eij,ej->e", uh, blk["tDD"], uh))
    assert np.allclose(lhs, e_q + e_c + e_t, rtol=1e-11, atol=1e-13)
    # c = 0: u_hat = 1 on dK gives u = 1, q = 0, zero flux
    blk0 = hdg.local_blocks(m, tab, kap, np.zeros_like(X), np.zeros_like(X), tau=tau)
    CK0, _, _, _ = hdg.local_solvers(blk0)
    ones = np.tile(np.eye(tab.d2)[0], 4)  # D_1 = 1 on every face
    assert np.abs(CK0 @ ones).max() < 1e-12 * np.abs(CK0).max()


@pytest.mark.parametrize("k", [1, 2, 3])
def test_boundary_data(k):
    tab = hdg.Tables(k)
    # eq. 6.3 reproduces any P_k(e) function given at the face nodes
    coef = np.random.default_rng(0).normal(size=(5, tab.d2))
    vals = coef @ tab.D.T
    assert np.allclose(hdg.dirichlet_data(tab, vals), coef, atol=1e-13)
    # eq. 6.4 with constant g: Phi_N = (g . n_e) e_1 (int_e D_i = |e| delta_i1)
    m, _ = _setup(1, k)
    g = np.array([0.3, -1.2, 2.0])
    gv = [np.full((len(m.neufaces), tab.nf), gc) for gc in g]
    Phi = hdg.neumann_data(m, tab, gv)
    nrm = np.zeros((m.nfc, 3))
    np.add.at(nrm, m.facebyele.ravel(), m.normals.reshape(-1, 3))
    ref = np.zeros_like(Phi)
    ref[:, 0] = nrm[m.neufaces] @ g
    assert np.allclose(Phi, ref, atol=1e-14)


def _poly_problem(k, s):
    """u in P_k, kappa constant, c variable: the HDG solution is exact (up to rounding)."""
    kap0 = 2.5
    cf = lambda x, y, z: 1 + x ** 2 + 0.5 * np.sin(y)  # noqa: E731
    if k == 1:
        u = lambda x, y, z: 1 + 0.3 * x - 0.7 * y + 0.5 * z  # noqa: E731
        gu = lambda x, y, z: (0.3 + 0 * x, -0.7 + 0 * x, 0.5 + 0 * x)  # noqa: E731
        lap = lambda x, y, z: 0 * x  # noqa: E731
    else:
        u = lambda x, y, z: 1 + 0.3 * x - 0.7 * y + 0.5 * z + 0.4 * x * y - 0.6 * z ** 2 + 0.2 * y * z  # noqa: E731
        gu = lambda x, y, z: (0.3 + 0.4 * y, -0.7 + 0.4 * x + 0.2 * z, 0.5 - 1.2 * z + 0.2 * y)  # noqa: E731
        lap = lambda x, y, z: -1.2 + 0 * x  # noqa: E731
    q = lambda x, y, z: tuple(-kap0 * g for g in gu(x, y, z))  # noqa: E731
    return Problem(
        name="poly", s=s, k=k, kappa=lambda x, y, z: kap0 + 0 * x, c=cf,
        f=lambda x, y, z: cf(x, y, z) * u(x, y, z) - kap0 * lap(x, y, z),
        uD=u, gN=lambda x, y, z: tuple(kap0 * g for g in gu(x, y, z)), u=u, q=q,
        dirichlet_planes=((0, 0.0), (0, 1.0)), jitter=0.15, seed=7)


def _projections(r, prob):
    m, tab, k = r["mesh"], r["tab"], prob.k
    X, Y, Z = hdg.volume_nodes(m, tab)
    u_ex = (prob.u(X, Y, Z) * tab.w) @ tab.P  # (1/|K|) int_K u P_i
    qv = prob.q(X, Y, Z)
    q_ex = np.stack([(qv[a] * tab.w) @ tab.P for a in range(3)], axis=1)
    FX, FY, FZ = hdg.face_nodes(m, tab)
    uh_ex = (prob.u(FX, FY, FZ) * tab.varpi) @ tab.D
    P1 = basis.dubiner3(k + 1, tab.p)
    us_ex = (prob.u(X, Y, Z) * tab.w) @ P1
    return q_ex, u_ex, uh_ex, us_ex


@pytest.mark.parametrize("k", [1, 2])
def test_exact_polynomial_solution(k):
    prob = _poly_problem(k, 2)
    r = hdg.solve_problem(prob)
    q_ex, u_ex, uh_ex, us_ex = _projections(r, prob)
    assert np.abs(r["u"] - u_ex).max() < 1e-11
    assert np.abs(r["q"] - q_ex).max() < 1e-11
    assert np.abs(r["uhat"] - uh_ex).max() < 1e-11
    assert np.abs(r["ustar"] - us_ex).max() < 1e-11


def test_planted_eq51_misprint_is_caught(monkeypatch):
    """Plant the misprint of eq. 5.1 (C_y where C_z belongs) in the oracle: the exactness pin fails."""
    orig = hdg.local_matrices

    def misprinted(blk):
        b2 = dict(blk)
        Cx, Cy, Cz = blk["C"]
        A1, A2, Af, A3 = orig(b2)
        n = Cx.shape[1]
        A1 = A1.copy()
        A1[:, 3 * n:, 2 * n:3 * n] = Cy
        return A1, A2, Af, A3

    monkeypatch.setattr(hdg, "local_matrices", misprinted)
    prob = _poly_problem(2, 2)  # q_z varies with y and z, so d_y q_z != d_z q_z
    r = hdg.solve_problem(prob)
    q_ex, u_ex, _, _ = _projections(r, prob)
    assert np.abs(r["u"] - u_ex).max() > 1e-3


@pytest.mark.parametrize("k,s", [(1, 1), (1, 2), (2, 1), (2, 2)])
def test_monolithic_equals_hybridised(k, s):
    kap_f, c_f = _varcoef()
    prob = get_problem("cube16_k3").at(s=s, k=k)
    prob.kappa, prob.c = prob.kappa, c_f
    c, e = kuhn_cube(s, jitter=0.1, seed=1)
    d, n = boundary_faces(c, e, prob.classify)
    r = hdg.solve_problem(prob, c, e, d, n)
    qm, um, uhm = hdg.monolithic_solve(r["mesh"], r["tab"], r["blk"], r["uhatD"], r["PhiN"])
    assert np.abs(uhm - r["uhat"]).max() < 1e-12 * max(1, np.abs(uhm).max())
    assert np.abs(um - r["u"]).max() < 1e-12 * max(1, np.abs(um).max())
    assert np.abs(qm - r["q"]).max() < 1e-12 * max(1, np.abs(qm).max())


@pytest.mark.parametrize("k", [1, 2])
def test_convergence_orders(k):
    prob = get_problem("cube4_k1").at(k=k)
    errs = []
    for s in (4, 8):
        r = hdg.solve_problem(prob.at(s=s))
        errs.append(hdg.errors(r["mesh"], k, r["q"], r["u"], r["uhat"], r["ustar"], prob.at(s=s)))
    rate = {a: np.log2(errs[0][a] / errs[1][a]) for a in errs[0]}
    for a in ("e_q", "e_u", "e_uhat"):
        assert abs(rate[a] - (k + 1)) < 0.25, rate
    assert rate["e_star"] > k + 2 - 0.25, rate
