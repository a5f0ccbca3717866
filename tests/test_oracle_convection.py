"""Pins of the oracle's convection-diffusion reading (Section 9, eq. 9.1 and the face
matrices after it): exactness for u in P_k (the scheme reproduces polynomial solutions
because q.nu and (beta.nu) u are single valued), the dense monolithic solve, the
integration-by-parts identity of the volume convection block, reduction to the
reaction-diffusion oracle at beta = 0, and the observed order k+1."""
import numpy as np
import pytest

from oracle import convection as cv
from oracle import hdg
from oracle.geometry import ExpandedMesh
from workloads import boundary_faces, get_problem, kuhn_cube
from workloads.problems import Problem


def _beta(x, y, z):
    return y, -x, 0.5 * z


def _poly_conv(k, s):
    kap0 = 1.7
    cf = lambda x, y, z: 1 + x ** 2  # noqa: E731
    if k == 1:
        u = lambda x, y, z: 1 + 0.3 * x - 0.7 * y + 0.5 * z  # noqa: E731
        gu = lambda x, y, z: (0.3 + 0 * x, -0.7 + 0 * x, 0.5 + 0 * x)  # noqa: E731
        lap = lambda x, y, z: 0 * x  # noqa: E731
    else:
        u = lambda x, y, z: 1 + 0.3 * x - 0.7 * y + 0.5 * z + 0.4 * x * y - 0.6 * z ** 2  # noqa: E731
        gu = lambda x, y, z: (0.3 + 0.4 * y, -0.7 + 0.4 * x, 0.5 - 1.2 * z)  # noqa: E731
        lap = lambda x, y, z: -1.2 + 0 * x  # noqa: E731

    def f(x, y, z):
        bx, by, bz = _beta(x, y, z)
        g = gu(x, y, z)
        return -kap0 * lap(x, y, z) + 0.5 * u(x, y, z) + bx * g[0] + by * g[1] + bz * g[2] + cf(x, y, z) * u(x, y, z)

    return Problem(name="polyconv", s=s, k=k, kappa=lambda x, y, z: kap0 + 0 * x, c=cf, f=f, uD=u, u=u,
                   q=lambda x, y, z: tuple(-kap0 * g for g in gu(x, y, z)), beta=_beta, tau=2.5,
                   jitter=0.15, seed=2)


def _mesh(prob):
    c, e = kuhn_cube(prob.s, prob.jitter, prob.seed)
    d, n = boundary_faces(c, e, lambda ax, v: "D")
    return c, e, d, n


@pytest.mark.parametrize("k", [1, 2])
def test_convection_exact_polynomial_solution(k):
    prob = _poly_conv(k, 2)
    r = cv.solve_problem_conv(prob, *_mesh(prob))
    mesh, tab = r["mesh"], r["tab"]
    X, Y, Z = hdg.volume_nodes(mesh, tab)
    u_ex = (prob.u(X, Y, Z) * tab.w) @ tab.P
    qv = prob.q(X, Y, Z)
    q_ex = np.stack([(qv[a] * tab.w) @ tab.P for a in range(3)], axis=1)
    FX, FY, FZ = hdg.face_nodes(mesh, tab)
    uh_ex = (prob.u(FX, FY, FZ) * tab.varpi) @ tab.D
    assert np.abs(r["u"] - u_ex).max() < 1e-11
    assert np.abs(r["q"] - q_ex).max() < 1e-11
    assert np.abs(r["uhat"] - uh_ex).max() < 1e-11
    # the trace matrix is genuinely non-symmetric
    CK = r["CK"]
    assert np.abs(CK - np.transpose(CK, (0, 2, 1))).max() > 1e-3 * np.abs(CK).max()


@pytest.mark.parametrize("k,s", [(1, 1), (2, 1), (1, 2)])
def test_convection_monolithic_equals_hybridised(k, s):
    prob = get_problem("cube48_k2_conv").at(s=s, k=k)
    r = cv.solve_problem_conv(prob, *_mesh(prob))
    qm, um, uhm = cv.monolithic_solve_conv(r["mesh"], r["tab"], r["mats"], r["blk"]["tDD"], r["aDD"], r["uhatD"])
    assert np.abs(uhm - r["uhat"]).max() < 1e-12 * np.abs(uhm).max()
    assert np.abs(um - r["u"]).max() < 1e-12 * np.abs(um).max()
    assert np.abs(qm - r["q"]).max() < 1e-12 * np.abs(qm).max()


def test_convection_block_integration_by_parts():
    """B_c + B_c^T = -(div beta) mass + sum_l <(beta.nu) P_i, P_j>_{e_l}  (by parts)."""
    k = 2
    c, e = kuhn_cube(2, 0.15, 1)
    d, n = boundary_faces(c, e, lambda ax, v: "D")
    mesh = ExpandedMesh(c, e, d, n)
    tab = hdg.Tables(k)
    X, Y, Z = hdg.volume_nodes(mesh, tab)
    FX, FY, FZ = cv.element_face_nodes(mesh, tab)
    Bc, _, _ = cv.convection_blocks(mesh, tab, _beta(X, Y, Z), _beta(FX, FY, FZ))
    # -(beta P_j, grad P_i) - (beta P_i, grad P_j) = (div beta P_i, P_j) - <beta.nu P_i, P_j>
    # so B_c + B_c^T = (div beta) M_1 - sum_l <beta.n_l P_i, P_j> / |e_l| |e_l|
    divb = 0.5
    lhs = Bc + np.transpose(Bc, (0, 2, 1))
    rhs = divb * mesh.volume[:, None, None] * np.eye(tab.n)
    for l in range(4):
        bn = sum(_beta(FX, FY, FZ)[s][:, l, :] * mesh.normals[:, l, s, None] for s in range(3))
        rhs = rhs - np.einsum("r,er,ri,rj->eij", tab.varpi, bn, tab.Pl[l], tab.Pl[l])
    assert np.abs(lhs - rhs).max() < 1e-14


def test_zero_beta_reduces_to_reaction_diffusion():
    prob = get_problem("cube16_k3").at(s=2, k=2)
    prob.dirichlet_planes = ((0, 0.0), (0, 1.0), (1, 0.0), (1, 1.0), (2, 0.0), (2, 1.0))
    prob.beta = lambda x, y, z: (0 * x, 0 * x, 0 * x)
    c, e, d, n = _mesh(prob)
    r1 = cv.solve_problem_conv(prob, c, e, d, n)
    prob.beta = None
    r0 = hdg.solve_problem(prob, c, e, d, n)
    assert np.abs(r1["CK"] - r0["CK"]).max() < 1e-13
    assert np.abs(r1["uhat"] - r0["uhat"]).max() < 1e-12


def test_convection_order():
    prob = get_problem("cube48_k2_conv").at(k=1)
    errs = []
    for s in (4, 8):
        p = prob.at(s=s)
        r = cv.solve_problem_conv(p, *_mesh(p))
        P = r["tab"].P
        mesh, tab = r["mesh"], r["tab"]
        pp, w, lam = __import__("oracle.quadrature", fromlist=["x"]).volume_rule(3)
        v = mesh.coordinates[mesh.elements]
        X, Y, Z = (v[:, :, dd] @ lam.T for dd in range(3))
        Pf = __import__("oracle.basis", fromlist=["x"]).dubiner3(1, pp)
        ue = p.u(X, Y, Z)
        uh = r["u"] @ Pf.T
        vol = mesh.volume
        errs.append(np.sqrt(np.sum(vol[:, None] * w * (ue - uh) ** 2) / np.sum(vol[:, None] * w * ue ** 2)))
        del P
    rate = np.log2(errs[0] / errs[1])
    assert abs(rate - 2.0) < 0.3, rate
