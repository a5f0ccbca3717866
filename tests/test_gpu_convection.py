"""Convection-diffusion (the Section 9 reading, see oracle/convection.py) on the GPU:
C^K (non-symmetric) against the oracle, BiCGStab trace solve and recovery end to end."""
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


def _gpu_conv(prob, c, e, d, n):
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


@pytest.mark.parametrize("k,s", [(1, 3), (2, 2), (3, 1), (4, 1)])
def test_convection_condensed_and_solution(k, s):
    prob = get_problem("cube48_k2_conv").at(s=s, k=k)
    c, e, d, n = make_mesh(prob)
    ref = cv.solve_problem_conv(prob, c, e, d, n)
    M = _gpu_conv(prob, c, e, d, n)
    EX, EY, EZ = (t.cpu().numpy() for t in M.element_face_nodes())
    mesh = ExpandedMesh(c, e, d, n)
    for g, o in zip((EX, EY, EZ), cv.element_face_nodes(mesh, ohdg.Tables(k))):
        assert np.abs(g - o).max() < 1e-15
    M.assemble_condense()
    Cg, Cfg = (t.cpu().numpy() for t in M.condensed())
    assert rel(Cg, ref["CK"]) < 1e-12
    assert rel(Cfg, ref["Cf"]) < 1e-12
    q1, u1 = M.recover(torch.from_numpy(ref["uhat"]).cuda())
    assert rel(u1.cpu().numpy(), ref["u"]) < 1e-12
    assert rel(q1.cpu().numpy(), ref["q"]) < 1e-12
    uhat, it, rr = M.solve_trace(rtol=1e-14, maxit=5000)
    assert rr <= 1e-14
    assert rel(uhat.cpu().numpy(), ref["uhat"]) < 1e-11
    q, u = M.recover(uhat)
    assert rel(u.cpu().numpy(), ref["u"]) < 1e-11
    assert rel(q.cpu().numpy(), ref["q"]) < 1e-11
