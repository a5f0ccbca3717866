"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Staged as the method is (solver tolerance must not pollute the comparison):
  C^K, C_f^K per element                 <= 1e-12 relative (max norm over the mesh)
  recovery from the oracle's u_hat        <= 1e-12
  end-to-end, both solves to 1e-14        <= 1e-11 (u_hat, q, u, u*)
  mixed-precision trace after refinement  <= 1e-9
Sizes span several elements per face pattern, all four degrees, jittered geometry, variable
coefficients, random tau, and both boundary types.
"""
import numpy as np
import pytest

from oracle import hdg as ohdg
from oracle.geometry import ExpandedMesh
from workloads import get_problem

from hdg_cases import gpu_setup, make_mesh, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _varprob(k):
    prob = get_problem("cube16_k3").at(k=k)
    prob.jitter, prob.seed = 0.18, 11
    return prob


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1305_1489_gb300 import build
    build()


@pytest.mark.parametrize("k,s", [(1, 3), (2, 2), (3, 2), (4, 1)])
def test_condensed_blocks(k, s):
    prob = _varprob(k)
    c, e, d, n = make_mesh(prob, s=s)
    rng = np.random.default_rng(k)
    tau = rng.uniform(0.5, 2.0, size=(len(e), 4))
    M = gpu_setup(prob, c, e, d, n, tau=tau)
    M.assemble_condense()
    Cg, Cfg = (t.cpu().numpy() for t in M.condensed())
    mesh = ExpandedMesh(c, e, d, n)
    tab = ohdg.Tables(k)
    X, Y, Z = ohdg.volume_nodes(mesh, tab)
    blk = ohdg.local_blocks(mesh, tab, prob.kappa(X, Y, Z), prob.c(X, Y, Z), prob.f(X, Y, Z), tau=tau)
    CK, Cf, _, _ = ohdg.local_solvers(blk)
    assert rel(Cg, CK) < 1e-12
    assert rel(Cfg, Cf) < 1e-12


@pytest.mark.parametrize("k", [1, 3])
def test_quadrature_nodes(k):
    prob = _varprob(k)
    c, e, d, n = make_mesh(prob, s=2)
    M = gpu_setup(prob, c, e, d, n)
    mesh = ExpandedMesh(c, e, d, n)
    tab = ohdg.Tables(k)
    for g, o in zip(M.volume_nodes(), ohdg.volume_nodes(mesh, tab)):
        assert np.abs(g.cpu().numpy() - o).max() < 1e-15
    for g, o in zip(M.face_nodes(), ohdg.face_nodes(mesh, tab)):
        assert np.abs(g.cpu().numpy() - o).max() < 1e-15
    faces, fbe, perm = M.faces()
    assert np.array_equal(faces[:, :3], mesh.faces) and np.array_equal(fbe, mesh.facebyele)
    assert np.array_equal(perm, mesh.perm)


@pytest.mark.parametrize("k,s", [(0, 3), (1, 4), (2, 2), (3, 2), (4, 1)])
def test_end_to_end(k, s):
    prob = _varprob(k)
    c, e, d, n = make_mesh(prob, s=s)
    ref = ohdg.solve_problem(prob, c, e, d, n)
    M = gpu_setup(prob, c, e, d, n)
    M.assemble_condense()
    # recovery from the oracle's trace isolates eq. 5.3
    q1, u1 = M.recover(torch.from_numpy(ref["uhat"]).cuda())
    assert rel(u1.cpu().numpy(), ref["u"]) < 1e-12
    assert rel(q1.cpu().numpy(), ref["q"]) < 1e-12
    uhat, it, rr = M.solve_trace(rtol=1e-14, maxit=5000)
    assert rr <= 1e-14
    assert rel(uhat.cpu().numpy(), ref["uhat"]) < 1e-11
    q, u = M.recover(uhat)
    assert rel(u.cpu().numpy(), ref["u"]) < 1e-11
    assert rel(q.cpu().numpy(), ref["q"]) < 1e-11
    us = M.postprocess(q, u)
    assert rel(us.cpu().numpy(), ref["ustar"]) < 1e-11
    # the postprocess alone, from the oracle's (q, u)
    us2 = M.postprocess(torch.from_numpy(ref["q"]).cuda(), torch.from_numpy(ref["u"]).cuda())
    assert rel(us2.cpu().numpy(), ref["ustar"]) < 1e-12


@pytest.mark.parametrize("k,s", [(1, 4), (3, 2)])
def test_mixed_precision_solve(k, s):
    from paper_1305_1489_gb300 import HDG_MIXED_FP32
    prob = _varprob(k)
    c, e, d, n = make_mesh(prob, s=s)
    ref = ohdg.solve_problem(prob, c, e, d, n)
    M = gpu_setup(prob, c, e, d, n)
    M.assemble_condense()
    uhat, it, rr = M.solve_trace(rtol=1e-12, maxit=5000, precision=HDG_MIXED_FP32)
    assert rr <= 1e-12
    assert rel(uhat.cpu().numpy(), ref["uhat"]) < 1e-9


def test_dirichlet_only_sinsinsin():
    prob = get_problem("cube4_k1")
    c, e, d, n = make_mesh(prob)
    ref = ohdg.solve_problem(prob, c, e, d, n)
    M = gpu_setup(prob, c, e, d, n)
    M.assemble_condense()
    # 1e-13: the attainable FP64 residual of this small trace system is ~1e-14
    uhat, it, rr = M.solve_trace(rtol=1e-13, maxit=5000)
    assert rel(uhat.cpu().numpy(), ref["uhat"]) < 1e-11
    q, u = M.recover(uhat)
    assert rel(u.cpu().numpy(), ref["u"]) < 1e-11


def test_error_paths():
    from paper_1305_1489_gb300 import HDGError
    prob = _varprob(1)
    c, e, d, n = make_mesh(prob, s=2)
    M = gpu_setup(prob, c, e, d, n)
    with pytest.raises(HDGError) as ei:
        M.solve_trace()  # before assembly
    assert ei.value.code == 5
    M.assemble_condense()
    uhat, it, rr = M.solve_trace(rtol=1e-14, maxit=1, raise_on_fail=False)
    assert it == 1 and rr > 1e-14
    with pytest.raises(HDGError) as ei:
        M.solve_trace(rtol=1e-14, maxit=1)
    assert ei.value.code == 7
    # kappa <= 0 on some nodes: the kernel's own check reports it, no fault
    X, Y, Z = M.volume_nodes()
    kap = torch.ones_like(X)
    kap[3, 5] = -1.0
    M.set_coefficients(kap, torch.ones_like(X), torch.ones_like(X))
    with pytest.raises(HDGError) as ei:
        M.assemble_condense()
    assert ei.value.code == 8
    e2 = e.copy()
    e2[0, [2, 3]] = e2[0, [3, 2]]
    from paper_1305_1489_gb300 import HDGMesh
    with pytest.raises(HDGError) as ei:
        HDGMesh(c, e2, d, n, 1)
    assert ei.value.code == 2


@pytest.mark.parametrize("k,s,shape", [(0, 3, "0"), (1, 3, "0"), (1, 3, "1"), (2, 2, "0"), (2, 2, "1"), (2, 2, "2"),
                                     (3, 2, "0"), (3, 2, "1"),
                                     (3, 2, "2"), (4, 1, "0"), (4, 2, "1"), (4, 1, "2"),
                                     (4, 2, "3"), (4, 1, "4")])
def test_double_float_assembly(k, s, shape, monkeypatch):
    """HDG_DF32: the same condensation in double-float arithmetic on the FP32 pipe, for every
    launch shape the autotuner may pick (HDG_K1_VARIANT forces one; shapes 3 and 4 at k = 4
    are the kernel that streams W_* one direction at a time)."""
    from paper_1305_1489_gb300 import HDG_DF32
    monkeypatch.setenv("HDG_K1_VARIANT", shape)
    prob = _varprob(k)
    c, e, d, n = make_mesh(prob, s=s)
    rng = np.random.default_rng(k + 10)
    tau = rng.uniform(0.5, 2.0, size=(len(e), 4))
    M = gpu_setup(prob, c, e, d, n, tau=tau)
    M.assemble_condense(precision=HDG_DF32)
    Cg, Cfg = (t.cpu().numpy() for t in M.condensed())
    mesh = ExpandedMesh(c, e, d, n)
    tab = ohdg.Tables(k)
    X, Y, Z = ohdg.volume_nodes(mesh, tab)
    blk = ohdg.local_blocks(mesh, tab, prob.kappa(X, Y, Z), prob.c(X, Y, Z), prob.f(X, Y, Z), tau=tau)
    CK, Cf, X2, xf = ohdg.local_solvers(blk)
    assert rel(Cg, CK) < 1e-11
    assert rel(Cfg, Cf) < 1e-11
    # recovery operators through the oracle's trace, and the whole solve
    ref = ohdg.solve_problem(prob, c, e, d, n)
    M2 = gpu_setup(prob, c, e, d, n)
    M2.assemble_condense(precision=HDG_DF32)
    q1, u1 = M2.recover(torch.from_numpy(ref["uhat"]).cuda())
    assert rel(u1.cpu().numpy(), ref["u"]) < 1e-11
    assert rel(q1.cpu().numpy(), ref["q"]) < 1e-11
    # the double-float postprocess (it follows a double-float assembly) from the oracle's q, u
    us = M2.postprocess(torch.from_numpy(ref["q"]).cuda(), torch.from_numpy(ref["u"]).cuda())
    assert rel(us.cpu().numpy(), ref["ustar"]) < 1e-11
    uhat, it, rr = M2.solve_trace(rtol=1e-14, maxit=5000)
    assert rel(uhat.cpu().numpy(), ref["uhat"]) < 1e-11


@pytest.mark.parametrize("k,s", [(2, 4), (3, 3)])
def test_mixed_precision_field_errors(k, s):
    """The mixed-precision path of the bench (double-float condensation, FP32 inner / FP64 outer
    two-level PCG to 1e-10): every field against the FP64 oracle, and the discretisation
    errors of eq. 10.1/10.2 unchanged to 3 digits."""
    from paper_1305_1489_gb300 import HDG_DF32, HDG_MIXED_FP32
    from workloads import kuhn_p1_hierarchy
    prob = _varprob(k)
    c, e, d, n = make_mesh(prob, s=s)
    ref = ohdg.solve_problem(prob, c, e, d, n)
    M = gpu_setup(prob, c, e, d, n)
    M.set_inner_tolerance(1e-6)
    M.set_coarse_space(*kuhn_p1_hierarchy(s, prob.dirichlet_planes, max_coarsest=8, strict=False))
    M.assemble_condense(HDG_DF32)
    uhat, it, rr = M.solve_trace(rtol=1e-10, maxit=5000, precision=HDG_MIXED_FP32)
    assert rr <= 1e-10
    q, u = M.recover(uhat)
    us = M.postprocess(q, u)
    got = {"uhat": uhat.cpu().numpy(), "q": q.cpu().numpy(), "u": u.cpu().numpy(), "ustar": us.cpu().numpy()}
    errs = {f: rel(got[f], ref[f]) for f in got}
    print(f"k={k} s={s} field errors vs the FP64 oracle: " + ", ".join(f"{f} {v:.1e}" for f, v in errs.items()))
    for f in got:
        assert errs[f] < 1e-8, (f, errs[f])
    mesh = ExpandedMesh(c, e, d, n)
    e_gpu = ohdg.errors(mesh, k, got["q"], got["u"], got["uhat"], got["ustar"], prob)
    e_ref = ohdg.errors(mesh, k, ref["q"], ref["u"], ref["uhat"], ref["ustar"], prob)
    for key in e_ref:
        assert abs(e_gpu[key] - e_ref[key]) <= 1e-3 * e_ref[key], (key, e_gpu[key], e_ref[key])


def test_host_loop_matches_device_loop(monkeypatch):
    """HDG_HOST_LOOP=1 (host replays instead of the conditional WHILE node) runs the same
    iterations and reaches the same trace."""
    prob = _varprob(2)
    c, e, d, n = make_mesh(prob, s=3)
    M = gpu_setup(prob, c, e, d, n)
    M.assemble_condense()
    u1, it1, r1 = M.solve_trace(rtol=1e-12, maxit=5000)
    monkeypatch.setenv("HDG_HOST_LOOP", "1")
    M2 = gpu_setup(prob, c, e, d, n)
    M2.assemble_condense()
    u2, it2, r2 = M2.solve_trace(rtol=1e-12, maxit=5000)
    assert it1 == it2 and abs(r1 - r2) <= 1e-15 * max(r1, 1e-300) + 1e-30
    assert np.array_equal(u1.cpu().numpy(), u2.cpu().numpy())
