"""Convection-diffusion (the Section 9 reading of oracle/convection.py) on the paths of the
headline workload: the double-float condensation (LU of the non-symmetric S_u in double-float
arithmetic), the FP32-inner / FP64-outer BiCGStab, and BiCGStab with the two-level
preconditioner, each against the FP64 oracle.

Bars: C^K, C_f^K and recovery from the oracle's trace <= 1e-11 (double-float, as for
reaction-diffusion); FP64 BiCGStab to 1e-14 <= 1e-11; mixed precision after refinement
<= 1e-9 in the trace; one application of the two-level preconditioner <= 1e-5 (FP32 V-cycle);
the workload's own pipeline (double-float K1, two-level mixed BiCGStab to 1e-10, recovery,
postprocess) <= 1e-8 per field with the discretisation errors of eq. 10.1/10.2 unchanged to 3
digits.
"""
import numpy as np
import pytest

from oracle import convection as cv
from oracle import hdg as ohdg
from oracle import twolevel as tl
from workloads import get_problem, kuhn_p1_hierarchy

from hdg_cases import make_mesh, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1305_1489_gb300 import build
    build()


def _conv_mesh(prob, c, e, d, n):
    from paper_1305_1489_gb300 import HDGMesh
    M = HDGMesh(c, e, d, n, prob.k)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()  # noqa: E731
    X, Y, Z = (t.cpu().numpy() for t in M.volume_nodes())
    EX, EY, EZ = (t.cpu().numpy() for t in M.element_face_nodes())
    tau = np.full((len(e), 4), prob.tau)
    M.set_coefficients(dev(prob.kappa(X, Y, Z)), dev(prob.c(X, Y, Z)), dev(prob.f(X, Y, Z)), dev(tau),
                       beta=dev(np.stack(prob.beta(X, Y, Z))), beta_faces=dev(np.stack(prob.beta(EX, EY, EZ))))
    FX, FY, FZ = (t.cpu().numpy() for t in M.face_nodes())
    M.set_boundary_data(dev(prob.uD(FX, FY, FZ)))
    return M


def _case(k, s):
    prob = get_problem("cube48_k2_conv").at(s=s, k=k)
    c, e, d, n = make_mesh(prob)
    return prob, c, e, d, n


@pytest.mark.parametrize("k,s,shape", [(1, 3, "0"), (1, 3, "1"), (2, 2, "0"), (2, 2, "1"), (2, 2, "2"), (3, 1, "0"),
                                       (3, 1, "1"), (3, 1, "2"), (4, 1, "0"), (4, 1, "1"), (4, 1, "2")])
def test_double_float_convection_condensation(k, s, shape, monkeypatch):
    from paper_1305_1489_gb300 import HDG_DF32
    monkeypatch.setenv("HDG_K1_VARIANT", shape)
    prob, c, e, d, n = _case(k, s)
    ref = cv.solve_problem_conv(prob, c, e, d, n)
    M = _conv_mesh(prob, c, e, d, n)
    M.assemble_condense(HDG_DF32)
    Cg, Cfg = (t.cpu().numpy() for t in M.condensed())
    assert rel(Cg, ref["CK"]) < 1e-11
    assert rel(Cfg, ref["Cf"]) < 1e-11
    q1, u1 = M.recover(torch.from_numpy(ref["uhat"]).cuda())
    assert rel(u1.cpu().numpy(), ref["u"]) < 1e-11
    assert rel(q1.cpu().numpy(), ref["q"]) < 1e-11
    uhat, it, rr = M.solve_trace(rtol=1e-14, maxit=5000)
    assert rr <= 1e-14
    assert rel(uhat.cpu().numpy(), ref["uhat"]) < 1e-11
    M.close()


@pytest.mark.parametrize("k,s", [(1, 3), (2, 3), (3, 2)])
def test_mixed_precision_bicgstab(k, s):
    from paper_1305_1489_gb300 import HDG_DF32, HDG_MIXED_FP32
    prob, c, e, d, n = _case(k, s)
    ref = cv.solve_problem_conv(prob, c, e, d, n)
    M = _conv_mesh(prob, c, e, d, n)
    M.set_inner_tolerance(1e-6)
    M.assemble_condense(HDG_DF32)
    uhat, it, rr = M.solve_trace(rtol=1e-12, maxit=5000, precision=HDG_MIXED_FP32)
    assert rr <= 1e-12
    assert rel(uhat.cpu().numpy(), ref["uhat"]) < 1e-9
    M.close()


@pytest.mark.parametrize("k,s,maxc,tail", [(2, 4, 8, None), (1, 4, 1, "8"), (3, 3, 1, None)])
def test_two_level_precond_apply_convection(k, s, maxc, tail, monkeypatch):
    if tail is not None:
        monkeypatch.setenv("HDG_COARSE_TAIL_MAX", tail)
    prob, c, e, d, n = _case(k, s)
    ref = cv.solve_problem_conv(prob, c, e, d, n)
    mesh, tab = ref["mesh"], ref["tab"]
    H, _ = ohdg.assemble(mesh, tab.d2, ref["CK"], ref["Cf"])
    sizes, nodes, weights = kuhn_p1_hierarchy(s, prob.dirichlet_planes, max_coarsest=maxc, strict=False)
    Binv, Pi, As, Ps = tl.setup(mesh, tab, H, sizes, nodes, weights)
    M = _conv_mesh(prob, c, e, d, n)
    M.assemble_condense()
    M.set_coarse_space(sizes, nodes, weights)
    rng = np.random.default_rng(s + 10 * k)
    r = rng.normal(size=(M.nfc, M.d2))
    r[mesh.dirfaces] = 0.0
    z = M.precond_apply(torch.from_numpy(r).cuda()).cpu().numpy().ravel()
    zo = tl.apply(Binv, Pi, As, Ps, r.ravel()).reshape(-1, tab.d2)
    zo[mesh.dirfaces] = 0.0
    assert rel(z, zo.ravel()) < 1e-5
    zb = np.einsum("fab,fb->fa", Binv, r).ravel()
    assert rel(zb, zo.ravel()) > 1e-3  # the coarse part is not negligible
    M.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_two_level_bicgstab_matches_oracle(precision):
    from paper_1305_1489_gb300 import HDG_DF32, HDG_FP64, HDG_MIXED_FP32
    prec = HDG_FP64 if precision == 0 else HDG_MIXED_FP32
    k, s = 2, 6
    prob, c, e, d, n = _case(k, s)
    ref = cv.solve_problem_conv(prob, c, e, d, n)
    M = _conv_mesh(prob, c, e, d, n)
    M.set_inner_tolerance(1e-6)
    M.assemble_condense(HDG_DF32)
    u_bj, it_bj, rr_bj = M.solve_trace(1e-12, 5000, precision=prec)
    M.set_coarse_space(*kuhn_p1_hierarchy(s, prob.dirichlet_planes, max_coarsest=8, strict=False))
    u_tl, it_tl, rr_tl = M.solve_trace(1e-12, 5000, precision=prec)
    assert rr_tl <= 1e-12 and rr_bj <= 1e-12
    assert it_tl < 0.7 * it_bj, (it_tl, it_bj)
    assert rel(u_tl.cpu().numpy(), ref["uhat"]) < 1e-9
    assert rel(u_bj.cpu().numpy(), ref["uhat"]) < 1e-9
    # a new assembly rebuilds the Galerkin hierarchy; removing the space restores block-Jacobi
    M.assemble_condense(HDG_DF32)
    u2, it2, _ = M.solve_trace(1e-12, 5000, precision=prec)
    assert abs(it2 - it_tl) <= 3 and rel(u2.cpu().numpy(), ref["uhat"]) < 1e-9
    M.set_coarse_space(None, None, None)
    _, it3, _ = M.solve_trace(1e-12, 5000, precision=prec)
    assert abs(it3 - it_bj) <= 3
    M.close()


@pytest.mark.parametrize("blocks", [None, "6"])
def test_convection_workload_pipeline(blocks, monkeypatch):
    """The convection workload's step at s = 4 (jittered, k = 2, beta = (y, -x, z/2)):
    double-float condensation, two-level FP32-inner / FP64-outer BiCGStab to 1e-10 (inner
    tolerance 1e-6), recovery and postprocess, on the default grid and on a 6-block grid
    (several face tiles per block); each field against the FP64 oracle and the errors of
    eq. 10.1/10.2 unchanged to 3 digits."""
    from paper_1305_1489_gb300 import HDG_DF32, HDG_MIXED_FP32
    if blocks:
        monkeypatch.setenv("HDG_FACE_BLOCKS", blocks)
    k, s = 2, 4
    prob, c, e, d, n = _case(k, s)
    ref = cv.solve_problem_conv(prob, c, e, d, n)
    mesh = ref["mesh"]
    ref_ustar = ohdg.postprocess(mesh, k, ref["kappa_q"], ref["q"], ref["u"])
    M = _conv_mesh(prob, c, e, d, n)
    if blocks:
        assert (M.nfc + 128 // M.d2 - 1) // (128 // M.d2) >= 5 * int(blocks)
    M.set_inner_tolerance(1e-6)
    M.set_coarse_space(*kuhn_p1_hierarchy(s, prob.dirichlet_planes, max_coarsest=8, strict=False))
    M.assemble_condense(HDG_DF32)
    uhat, it, rr = M.solve_trace(rtol=1e-10, maxit=5000, precision=HDG_MIXED_FP32)
    assert rr <= 1e-10
    q, u = M.recover(uhat)
    us = M.postprocess(q, u)
    got = {"uhat": uhat.cpu().numpy(), "q": q.cpu().numpy(), "u": u.cpu().numpy(), "ustar": us.cpu().numpy()}
    want = {"uhat": ref["uhat"], "q": ref["q"], "u": ref["u"], "ustar": ref_ustar}
    errs = {f: rel(got[f], want[f]) for f in got}
    print(f"convection pipeline s={s} k={k} blocks={blocks}: iterations {it}, " +
          ", ".join(f"{f} {v:.1e}" for f, v in errs.items()))
    for f in got:
        assert errs[f] < 1e-8, (f, errs[f])
    e_gpu = ohdg.errors(mesh, k, got["q"], got["u"], got["uhat"], got["ustar"], prob)
    e_ref = ohdg.errors(mesh, k, ref["q"], ref["u"], ref["uhat"], ref_ustar, prob)
    for key in e_ref:
        assert abs(e_gpu[key] - e_ref[key]) <= 1e-3 * e_ref[key], (key, e_gpu[key], e_ref[key])
    M.close()
