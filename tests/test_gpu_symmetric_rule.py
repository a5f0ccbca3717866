"""The smaller symmetric volume rule (hdg_set_volume_rule(HDG_RULE_SYMMETRIC), Grundmann-Moller
of degree 2k+3) on the GPU against the oracle on the same rule: the library's nodes, the FP64
condensation (C^K, C_f^K <= 1e-12), the whole FP64 pipeline (u_hat, q, u, u* <= 1e-11, both
solves to 1e-14), convection, the mixed-precision solve after refinement (<= 1e-9), and the
refusal of the double-float assembly, which needs the conical rule."""
import numpy as np
import pytest

from oracle import convection as cv
from oracle import hdg as ohdg
from oracle.geometry import ExpandedMesh
from workloads import get_problem

from hdg_cases import make_mesh, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1305_1489_gb300 import build
    build()


def _setup(prob, c, e, d, n, conv=False):
    from paper_1305_1489_gb300 import HDG_RULE_SYMMETRIC, HDGMesh
    M = HDGMesh(c, e, d, n, prob.k)
    nq0 = M.nq
    M.set_volume_rule(HDG_RULE_SYMMETRIC)
    assert M.nq == (prob.k + 2) * (prob.k + 3) * (prob.k + 4) * (prob.k + 5) // 24 < nq0
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()  # noqa: E731
    X, Y, Z = (t.cpu().numpy() for t in M.volume_nodes())
    if conv:
        EX, EY, EZ = (t.cpu().numpy() for t in M.element_face_nodes())
        M.set_coefficients(dev(prob.kappa(X, Y, Z)), dev(prob.c(X, Y, Z)), dev(prob.f(X, Y, Z)),
                           dev(np.full((len(e), 4), prob.tau)), beta=dev(np.stack(prob.beta(X, Y, Z))),
                           beta_faces=dev(np.stack(prob.beta(EX, EY, EZ))))
    else:
        M.set_coefficients(dev(prob.kappa(X, Y, Z)), dev(prob.c(X, Y, Z)), dev(prob.f(X, Y, Z)))
    FX, FY, FZ = (t.cpu().numpy() for t in M.face_nodes())
    gN = dev(np.stack(prob.gN(FX, FY, FZ))) if prob.gN is not None else None
    M.set_boundary_data(dev(prob.uD(FX, FY, FZ)), gN)
    return M


@pytest.mark.parametrize("k,s", [(1, 3), (2, 2), (3, 2), (4, 2)])
def test_symmetric_rule_pipeline(k, s):
    prob = get_problem("cube16_k3").at(k=k)
    prob.jitter, prob.seed = 0.18, 11
    c, e, d, n = make_mesh(prob, s=s)
    ref = ohdg.solve_problem(prob, c, e, d, n, rule="symmetric")
    M = _setup(prob, c, e, d, n)
    mesh = ExpandedMesh(c, e, d, n)
    for g, o in zip(M.volume_nodes(), ohdg.volume_nodes(mesh, ohdg.Tables(k, "symmetric"))):
        assert np.abs(g.cpu().numpy() - o).max() < 1e-15
    M.assemble_condense()
    Cg, Cfg = (t.cpu().numpy() for t in M.condensed())
    assert rel(Cg, ref["CK"]) < 1e-12
    assert rel(Cfg, ref["Cf"]) < 1e-12
    uhat, it, rr = M.solve_trace(rtol=1e-14, maxit=5000)
    assert rel(uhat.cpu().numpy(), ref["uhat"]) < 1e-11
    q, u = M.recover(uhat)
    assert rel(q.cpu().numpy(), ref["q"]) < 1e-11
    assert rel(u.cpu().numpy(), ref["u"]) < 1e-11
    us = M.postprocess(q, u)
    assert rel(us.cpu().numpy(), ref["ustar"]) < 1e-11
    M.close()


def test_symmetric_rule_mixed_solve_and_df_refusal():
    from paper_1305_1489_gb300 import HDG_DF32, HDG_MIXED_FP32, HDGError
    prob = get_problem("cube16_k3").at(k=2)
    prob.jitter, prob.seed = 0.18, 11
    c, e, d, n = make_mesh(prob, s=3)
    ref = ohdg.solve_problem(prob, c, e, d, n, rule="symmetric")
    M = _setup(prob, c, e, d, n)
    with pytest.raises(HDGError) as ei:
        M.assemble_condense(HDG_DF32)
    assert ei.value.code == 9  # HDG_ERR_UNSUPPORTED
    M.assemble_condense()
    M.set_inner_tolerance(1e-6)
    uhat, it, rr = M.solve_trace(rtol=1e-12, maxit=5000, precision=HDG_MIXED_FP32)
    assert rel(uhat.cpu().numpy(), ref["uhat"]) < 1e-9
    M.close()


@pytest.mark.parametrize("k,s", [(2, 2), (3, 1)])
def test_symmetric_rule_convection(k, s):
    prob = get_problem("cube48_k2_conv").at(s=s, k=k)
    c, e, d, n = make_mesh(prob)
    ref = cv.solve_problem_conv(prob, c, e, d, n, rule="symmetric")
    M = _setup(prob, c, e, d, n, conv=True)
    M.assemble_condense()
    Cg, _ = (t.cpu().numpy() for t in M.condensed())
    assert rel(Cg, ref["CK"]) < 1e-12
    uhat, it, rr = M.solve_trace(rtol=1e-14, maxit=5000)
    assert rel(uhat.cpu().numpy(), ref["uhat"]) < 1e-11
    M.close()


def test_symmetric_rule_unresolved_coefficient_is_reported():
    """Some weights of the symmetric rule are negative, so M_{kappa^-1} is positive definite
    only while kappa is resolved on the element: on the single-cube mesh (s = 1) at k = 4 the
    oracle's M_{kappa^-1} has negative eigenvalues on 5 elements, and the FP64 assembly reports
    HDG_ERR_LOCAL_SINGULAR with that count instead of returning a factorisation."""
    from paper_1305_1489_gb300 import HDGError
    prob = get_problem("cube16_k3").at(k=4)
    prob.jitter, prob.seed = 0.18, 11
    c, e, d, n = make_mesh(prob, s=1)
    mesh = ExpandedMesh(c, e, d, n)
    tab = ohdg.Tables(4, "symmetric")
    X, Y, Z = ohdg.volume_nodes(mesh, tab)
    blk = ohdg.local_blocks(mesh, tab, prob.kappa(X, Y, Z), prob.c(X, Y, Z), prob.f(X, Y, Z))
    nbad = int((np.linalg.eigvalsh(blk["M_kinv"])[:, 0] <= 0).sum())
    assert nbad > 0
    M = _setup(prob, c, e, d, n)
    with pytest.raises(HDGError) as ei:
        M.assemble_condense()
    assert ei.value.code == 6 and str(nbad) in str(ei.value)
    M.close()
