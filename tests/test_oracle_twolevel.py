"""Pins of the two-level preconditioner oracle (oracle/twolevel.py) against facts that do not
depend on it: traces of linear fields, the nesting of the Kuhn hierarchy, exactness on a
diagonal matrix, the projection identity of an exact coarse solve, symmetry and positivity,
the two-grid contraction, and convergence of PCG to the direct solution."""
import numpy as np
import pytest
import scipy.sparse as sps

from oracle import hdg as ohdg
from oracle import twolevel as tl
from oracle.geometry import ExpandedMesh
from workloads import boundary_faces, kuhn_cube, kuhn_p1_hierarchy
from workloads.problems import cube32_k2_grf, get_problem

ALL = ((0, 0.0), (0, 1.0), (1, 0.0), (1, 1.0), (2, 0.0), (2, 1.0))


def _system(prob, s):
    c, e = kuhn_cube(s, prob.jitter, prob.seed)
    d, n = boundary_faces(c, e, prob.classify)
    mesh = ExpandedMesh(c, e, d, n)
    tab = ohdg.Tables(prob.k)
    X, Y, Z = ohdg.volume_nodes(mesh, tab)
    blk = ohdg.local_blocks(mesh, tab, prob.kappa(X, Y, Z), prob.c(X, Y, Z), prob.f(X, Y, Z), tau=prob.tau)
    CK, Cf, _, _ = ohdg.local_solvers(blk)
    H, F = ohdg.assemble(mesh, tab.d2, CK, Cf)
    return mesh, tab, H, F


@pytest.mark.parametrize("k", [1, 2, 3])
def test_prolongation_reproduces_linear_traces(k):
    s = 2
    c, e = kuhn_cube(s, 0.15, 3)
    d, n = boundary_faces(c, e, lambda ax, val: "N")
    mesh = ExpandedMesh(c, e, d, n)
    tab = ohdg.Tables(k)
    sizes, nodes, weights = kuhn_p1_hierarchy(s, (), max_coarsest=8)
    nver = len(c)
    Pi = tl.prolongation(mesh, tab, nodes[:nver], weights[:nver], sizes[0])
    g = np.array([0.3, -1.2, 0.7])
    lin = lambda x, y, z: 0.5 + g[0] * x + g[1] * y + g[2] * z  # noqa: E731
    uh = (Pi @ lin(c[:, 0], c[:, 1], c[:, 2])).reshape(mesh.nfc, tab.d2)
    FX, FY, FZ = ohdg.face_nodes(mesh, tab)
    assert np.abs(uh @ tab.D.T - lin(FX, FY, FZ)).max() < 1e-13


def test_hierarchy_is_nested_p1():
    # a linear field on the coarser grid, interpolated level by level, stays the same field
    s = 8
    sizes, nodes, weights = kuhn_p1_hierarchy(s, (), max_coarsest=30)
    assert sizes == [729, 125, 27]
    Ps = tl.level_interpolations(sizes, nodes, weights, (s + 1) ** 3)
    for lvl, P in enumerate(Ps):
        sf, sc = s >> lvl, s >> (lvl + 1)
        gf = np.stack(np.meshgrid(*(np.arange(sf + 1) / sf,) * 3, indexing="ij"), -1).transpose(2, 1, 0, 3).reshape(-1, 3)
        gc = np.stack(np.meshgrid(*(np.arange(sc + 1) / sc,) * 3, indexing="ij"), -1).transpose(2, 1, 0, 3).reshape(-1, 3)
        f = lambda p: 1.0 + p @ np.array([2.0, -3.0, 0.5])  # noqa: E731
        assert np.abs(P @ f(gc) - f(gf)).max() < 1e-13


def test_vcycle_exact_on_diagonal_matrix():
    rng = np.random.default_rng(0)
    A0 = sps.diags(rng.uniform(1, 3, 20)).tocsr()
    P = sps.random(20, 5, density=0.3, random_state=1, format="csr")
    As = [A0, (P.T @ A0 @ P).tocsr() + sps.identity(5, format="csr")]
    b = rng.normal(size=20)
    assert np.abs(tl.vcycle(As, [P], b) - b / A0.diagonal()).max() < 1e-14


@pytest.fixture(scope="module")
def grf_s4():
    prob = cube32_k2_grf(4, s=4)
    mesh, tab, H, F = _system(prob, 4)
    sizes, nodes, weights = kuhn_p1_hierarchy(4, ALL, max_coarsest=1)
    return mesh, tab, H, F, sizes, nodes, weights


def test_exact_coarse_solve_is_a_projection(grf_s4):
    mesh, tab, H, F, sizes, nodes, weights = grf_s4
    assert sizes == [27, 1]
    Binv, Pi, As, Ps = tl.setup(mesh, tab, H, sizes, nodes, weights)
    A0 = As[0].toarray()
    assert np.abs(A0 - (Pi.T @ H @ Pi).toarray()).max() < 1e-13 * np.abs(A0).max()
    # with the first level as the coarsest, V = A_0^-1 and Pi V Pi^T H Pi = Pi
    Q = Pi @ tl.vcycle([As[0]], [], (Pi.T @ (H @ Pi)).toarray())
    assert np.abs(Q - Pi.toarray()).max() < 1e-11


def test_preconditioner_symmetric_positive(grf_s4):
    mesh, tab, H, F, sizes, nodes, weights = grf_s4
    Binv, Pi, As, Ps = tl.setup(mesh, tab, H, sizes, nodes, weights)
    free = np.ones(mesh.nfc * tab.d2, bool)
    free[(mesh.dirfaces[:, None] * tab.d2 + np.arange(tab.d2)).ravel()] = False
    rng = np.random.default_rng(1)
    x, y = rng.normal(size=(2, free.size)) * free
    Mx, My = tl.apply(Binv, Pi, As, Ps, x) * free, tl.apply(Binv, Pi, As, Ps, y) * free
    assert abs(y @ Mx - x @ My) < 1e-12 * abs(x @ Mx)
    assert x @ Mx > 0 and y @ My > 0


def test_two_grid_contraction(grf_s4):
    # E = (I - D^-1 A)(I - P A_c^-1 P^T A)(I - D^-1 A) has A-norm below one
    mesh, tab, H, F, sizes, nodes, weights = grf_s4
    _, _, As, Ps = tl.setup(mesh, tab, H, sizes, nodes, weights)
    A = As[0].toarray()
    P = Ps[0].toarray()
    D = np.abs(A).sum(axis=1)
    S = np.eye(len(A)) - A / D[:, None]
    E = S @ (np.eye(len(A)) - P @ np.linalg.solve(P.T @ A @ P, P.T @ A)) @ S
    L = np.linalg.cholesky(A)
    assert np.linalg.norm(L.T @ E @ np.linalg.inv(L.T), 2) < 1.0


def test_pcg_reaches_direct_solution_in_fewer_iterations():
    prob = get_problem("cube16_k3").at(s=4, k=2)
    mesh, tab, H, F = _system(prob, 4)
    planes = prob.dirichlet_planes
    sizes, nodes, weights = kuhn_p1_hierarchy(4, planes, max_coarsest=40)
    Binv, Pi, As, Ps = tl.setup(mesh, tab, H, sizes, nodes, weights)
    d2 = tab.d2
    free = np.ones(mesh.nfc * d2, bool)
    free[(mesh.dirfaces[:, None] * d2 + np.arange(d2)).ravel()] = False
    b = np.where(free, F, 0.0)
    x_tl, it_tl = tl.pcg(H, b, lambda r: tl.apply(Binv, Pi, As, Ps, r), free)
    x_bj, it_bj = tl.pcg(H, b, lambda r: np.einsum("fab,fb->fa", Binv, r.reshape(-1, d2)).ravel(), free)
    fi = np.nonzero(free)[0]
    x_d = np.zeros_like(b)
    x_d[fi] = sps.linalg.spsolve(H[fi][:, fi].tocsc(), b[fi])
    assert np.abs(x_tl - x_d).max() < 1e-8 * np.abs(x_d).max()
    assert it_tl < it_bj
