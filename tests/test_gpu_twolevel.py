"""The two-level trace preconditioner on the GPU against the FP64 oracle (oracle/twolevel.py):
one application of M^-1 (FP32 V-cycle: 1e-5 relative), solves with it against the oracle's
direct solve, fewer iterations than block-Jacobi, and the argument checks."""
import numpy as np
import pytest

from oracle import hdg as ohdg
from oracle import twolevel as tl
from oracle.geometry import ExpandedMesh
from workloads import kuhn_p1_hierarchy
from workloads.problems import cube32_k2_grf, get_problem

from hdg_cases import gpu_setup, make_mesh, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1305_1489_gb300 import build
    build()


def _case(name, s, k):
    if name == "grf":
        prob = cube32_k2_grf(7, s=s, k=k)
    else:
        prob = get_problem("cube16_k3").at(s=s, k=k)
    c, e, d, n = make_mesh(prob)
    return prob, c, e, d, n


def _oracle(prob, c, e, d, n, sizes, nodes, weights):
    mesh = ExpandedMesh(c, e, d, n)
    tab = ohdg.Tables(prob.k)
    X, Y, Z = ohdg.volume_nodes(mesh, tab)
    blk = ohdg.local_blocks(mesh, tab, prob.kappa(X, Y, Z), prob.c(X, Y, Z), prob.f(X, Y, Z), tau=prob.tau)
    CK, Cf, _, _ = ohdg.local_solvers(blk)
    H, F = ohdg.assemble(mesh, tab.d2, CK, Cf)
    return mesh, tab, H, tl.setup(mesh, tab, H, sizes, nodes, weights)


@pytest.mark.parametrize("name,s,k,maxc,tail", [("grf", 4, 2, 1, None), ("poly", 4, 1, 30, None),
                                                ("poly", 4, 3, 30, None), ("grf", 8, 2, 64, None),
                                                ("poly", 4, 4, 30, None), ("grf", 8, 2, 1, "8")])
def test_precond_apply_matches_oracle(name, s, k, maxc, tail, monkeypatch):
    # tail = largest level of the single-CTA part; "8" puts the 27-node level on grid kernels
    if tail is not None:
        monkeypatch.setenv("HDG_COARSE_TAIL_MAX", tail)
    prob, c, e, d, n = _case(name, s, k)
    sizes, nodes, weights = kuhn_p1_hierarchy(s, prob.dirichlet_planes, max_coarsest=maxc)
    mesh, tab, H, (Binv, Pi, As, Ps) = _oracle(prob, c, e, d, n, sizes, nodes, weights)
    M = gpu_setup(prob, c, e, d, n)
    M.assemble_condense()
    M.set_coarse_space(sizes, nodes, weights)
    rng = np.random.default_rng(s + k)
    r = rng.normal(size=(M.nfc, M.d2))
    r[mesh.dirfaces] = 0.0
    z = M.precond_apply(torch.from_numpy(r).cuda()).cpu().numpy().ravel()
    zo = tl.apply(Binv, Pi, As, Ps, r.ravel())
    zo = zo.reshape(-1, tab.d2)
    zo[mesh.dirfaces] = 0.0
    assert rel(z, zo.ravel()) < 1e-5
    # the coarse part is not negligible: the block-Jacobi part alone differs
    zb = np.einsum("fab,fb->fa", Binv, r).ravel()
    assert rel(zb, zo.ravel()) > 1e-3


@pytest.mark.parametrize("precision", [0, 1])
def test_two_level_solve_matches_direct_and_saves_iterations(precision):
    from paper_1305_1489_gb300 import HDG_FP64, HDG_MIXED_FP32
    prec = HDG_FP64 if precision == 0 else HDG_MIXED_FP32
    prob, c, e, d, n = _case("grf", 8, 2)
    M = gpu_setup(prob, c, e, d, n)
    M.assemble_condense()
    M.set_inner_tolerance(1e-6)
    u_bj, it_bj, rr_bj = M.solve_trace(1e-10, 5000, precision=prec)
    sizes, nodes, weights = kuhn_p1_hierarchy(8, prob.dirichlet_planes)
    M.set_coarse_space(sizes, nodes, weights)
    u_tl, it_tl, rr_tl = M.solve_trace(1e-10, 5000, precision=prec)
    assert rr_tl <= 1e-10 and rr_bj <= 1e-10
    assert it_tl < 0.6 * it_bj
    assert rel(u_tl.cpu().numpy(), u_bj.cpu().numpy()) < 1e-8
    # oracle direct solve
    mesh = ExpandedMesh(c, e, d, n)
    tab = ohdg.Tables(2)
    X, Y, Z = ohdg.volume_nodes(mesh, tab)
    blk = ohdg.local_blocks(mesh, tab, prob.kappa(X, Y, Z), prob.c(X, Y, Z), prob.f(X, Y, Z), tau=prob.tau)
    CK, Cf, _, _ = ohdg.local_solvers(blk)
    H, F = ohdg.assemble(mesh, tab.d2, CK, Cf)
    uo, _, _, _ = ohdg.solve_trace(mesh, tab.d2, H, F, np.zeros((len(mesh.dirfaces), tab.d2)))
    assert rel(u_tl.cpu().numpy(), uo) < 1e-8
    # a new assembly rebuilds the Galerkin hierarchy; removing the space restores block-Jacobi
    M.assemble_condense()
    u2, it2, _ = M.solve_trace(1e-10, 5000, precision=prec)
    assert abs(it2 - it_tl) <= 2 and rel(u2.cpu().numpy(), uo) < 1e-8
    M.set_coarse_space(None, None, None)
    _, it3, _ = M.solve_trace(1e-10, 5000, precision=prec)
    assert it3 == it_bj
    # setting the coarse space again (new device arrays) after solves with cached graphs
    M.set_coarse_space(sizes, nodes, weights)
    u4, it4, _ = M.solve_trace(1e-10, 5000, precision=prec)
    M.set_coarse_space(sizes, nodes, weights)
    u5, it5, _ = M.solve_trace(1e-10, 5000, precision=prec)
    assert it4 == it5 and abs(it4 - it_tl) <= 2 and rel(u5.cpu().numpy(), uo) < 1e-8


def test_two_level_with_neumann_faces_and_k3():
    prob, c, e, d, n = _case("poly", 8, 3)
    M = gpu_setup(prob, c, e, d, n)
    M.assemble_condense()
    _, it_bj, _ = M.solve_trace(1e-10, 5000)
    sizes, nodes, weights = kuhn_p1_hierarchy(8, prob.dirichlet_planes)
    M.set_coarse_space(sizes, nodes, weights)
    u, it, rr = M.solve_trace(1e-12, 5000)
    assert rr <= 1e-12 and it < it_bj
    mesh = ExpandedMesh(c, e, d, n)
    res = ohdg.solve_problem(prob, c, e, d, n)
    assert rel(u.cpu().numpy(), res["uhat"]) < 1e-9
    del mesh


def test_coarse_space_argument_errors():
    from paper_1305_1489_gb300 import HDGError
    prob, c, e, d, n = _case("grf", 4, 1)
    M = gpu_setup(prob, c, e, d, n)
    M.assemble_condense()
    sizes, nodes, weights = kuhn_p1_hierarchy(4, prob.dirichlet_planes, max_coarsest=1)
    with pytest.raises(HDGError):
        M.precond_apply(torch.zeros(M.nfc, M.d2, dtype=torch.float64, device="cuda"))
    with pytest.raises(HDGError):
        M.set_coarse_space(sizes[:1], nodes[:len(c)], weights[:len(c)])  # one level
    bad = nodes.copy()
    bad[3, 0] = sizes[0]  # out of range
    with pytest.raises(HDGError):
        M.set_coarse_space(sizes, bad, weights)
    # a coarsest level above 128 nodes is refused
    nodes2 = np.concatenate([nodes[:len(c)], np.zeros((sizes[0], 4), np.int32) - 1])
    nodes2[len(c):, 0] = 0
    weights2 = np.concatenate([weights[:len(c)], np.ones((sizes[0], 4))])
    with pytest.raises(HDGError):
        M.set_coarse_space([sizes[0], 129], nodes2, weights2)
    M.set_coarse_space(sizes, nodes, weights)
    z = M.precond_apply(torch.ones(M.nfc, M.d2, dtype=torch.float64, device="cuda"))
    assert torch.isfinite(z).all()


def test_precond_apply_coarse_level0_matches_oracle():
    """Level 0 on the 2h grid (each mesh vertex interpolates from up to two level-0 nodes):
    the general prolongation and restriction paths against the oracle."""
    from workloads import kuhn_coarse_interpolation
    prob, c, e, d, n = _case("grf", 8, 2)
    nodes0, weights0, n0 = kuhn_coarse_interpolation(8, 4, interior_only=True)
    sz, nd, wt = kuhn_p1_hierarchy(4, prob.dirichlet_planes, max_coarsest=1)
    assert sz[0] == n0
    skip = 5 ** 3  # the vertex rows of the 4^3 grid's own hierarchy
    sizes = sz
    nodes = np.concatenate([nodes0, nd[skip:]]).astype(np.int32)
    weights = np.concatenate([weights0, wt[skip:]])
    mesh, tab, H, (Binv, Pi, As, Ps) = _oracle(prob, c, e, d, n, sizes, nodes, weights)
    M = gpu_setup(prob, c, e, d, n)
    M.assemble_condense()
    M.set_coarse_space(sizes, nodes, weights)
    rng = np.random.default_rng(3)
    r = rng.normal(size=(M.nfc, M.d2))
    r[mesh.dirfaces] = 0.0
    z = M.precond_apply(torch.from_numpy(r).cuda()).cpu().numpy()
    zo = tl.apply(Binv, Pi, As, Ps, r.ravel()).reshape(-1, tab.d2)
    zo[mesh.dirfaces] = 0.0
    assert rel(z.ravel(), zo.ravel()) < 1e-5
    u, it, rr = M.solve_trace(1e-10, 5000)
    assert rr <= 1e-10
