"""GPU parity of the hybridised BDM element (Section 9, "BDM": tau = 0, u_h in P_{k-1})
against the oracle, through the C ABI, for both assembly precisions."""
import numpy as np
import pytest
import torch

from hdg_cases import gpu_setup, make_mesh, rel
from oracle import bdm as obdm
from oracle import hdg as ohdg
from oracle.geometry import ExpandedMesh
from workloads import get_problem

pytestmark = pytest.mark.gpu


def _prob(k):
    p = get_problem("cube16_k3").at(k=k)
    p.c = lambda x, y, z: 1 + x ** 2 + 0.3 * y
    return p


@pytest.mark.parametrize("k,s,prec", [(1, 3, 0), (2, 2, 0), (3, 2, 0), (4, 1, 0), (1, 3, 2), (2, 2, 2), (3, 2, 2),
                                      (4, 1, 2)])
def test_bdm_condensed_parity(k, s, prec):
    from paper_1305_1489_gb300 import HDG_METHOD_BDM
    prob = _prob(k)
    c, e, d, n = make_mesh(prob, s=s, jitter=0.15, seed=6)
    tau = np.random.default_rng(k).uniform(0.5, 2.0, size=(len(e), 4))  # ignored by BDM
    M = gpu_setup(prob, c, e, d, n, tau=tau)
    M.set_method(HDG_METHOD_BDM)
    M.assemble_condense(precision=prec)
    Cg, Cfg = (t.cpu().numpy() for t in M.condensed())
    mesh = ExpandedMesh(c, e, d, n)
    tab = ohdg.Tables(k)
    X, Y, Z = ohdg.volume_nodes(mesh, tab)
    blk = ohdg.local_blocks(mesh, tab, prob.kappa(X, Y, Z), prob.c(X, Y, Z), prob.f(X, Y, Z), tau=0.0)
    CK, Cf, _, _ = obdm.local_solvers(blk, tab.d2)
    bar = 1e-12 if prec == 0 else 1e-11
    assert rel(Cg, CK) < bar
    assert rel(Cfg, Cf) < bar


@pytest.mark.parametrize("k,s,prec", [(1, 4, 0), (2, 2, 2), (3, 2, 2)])
def test_bdm_end_to_end(k, s, prec):
    from paper_1305_1489_gb300 import HDG_METHOD_BDM
    prob = _prob(k)
    c, e, d, n = make_mesh(prob, s=s, jitter=0.15, seed=8)
    ref = obdm.solve_problem(prob, c, e, d, n)
    M = gpu_setup(prob, c, e, d, n)
    M.set_method(HDG_METHOD_BDM)
    M.assemble_condense(precision=prec)
    uhat, it, rr = M.solve_trace(rtol=1e-14, maxit=20000)
    assert rel(uhat.cpu().numpy(), ref["uhat"]) < 1e-11
    q, u = M.recover(uhat)
    ug = u.cpu().numpy()
    assert np.abs(ug[:, ug.shape[1] - M.d2:]).max() == 0.0
    assert rel(ug, ref["u"]) < 1e-11
    assert rel(q.cpu().numpy(), ref["q"]) < 1e-11
    us = M.postprocess(q, u)
    assert rel(us.cpu().numpy(), ref["ustar"]) < 1e-11


def test_bdm_method_argument_and_switch_back():
    from paper_1305_1489_gb300 import HDG_METHOD_BDM, HDG_METHOD_HDG, HDGError
    prob = _prob(2)
    c, e, d, n = make_mesh(prob, s=2)
    M = gpu_setup(prob, c, e, d, n)
    with pytest.raises(HDGError) as ei:
        M.set_method(7)
    assert ei.value.code == 1
    M.set_method(HDG_METHOD_BDM)
    M.assemble_condense()
    Cb = M.condensed()[0].cpu().numpy()
    M.set_method(HDG_METHOD_HDG)
    M.assemble_condense()
    Ch = M.condensed()[0].cpu().numpy()
    ref = ohdg.solve_problem(prob, c, e, d, n)
    assert rel(Ch, ref["CK"]) < 1e-12
    assert rel(Cb, Ch) > 1e-3


@pytest.mark.parametrize("k,shape", [(4, "3"), (4, "4")])
def test_bdm_streamed_k1_shapes(k, shape, monkeypatch):
    """The double-float kernel that streams W_* one direction at a time (reaction-diffusion,
    k = 4): the BDM identity rows of S_u and the zero rows of G^T are set after its last
    direction, and its condensed blocks match the oracle's like the other shapes'."""
    from paper_1305_1489_gb300 import HDG_DF32, HDG_METHOD_BDM
    monkeypatch.setenv("HDG_K1_VARIANT", shape)
    prob = _prob(k)
    c, e, d, n = make_mesh(prob, s=2, jitter=0.15, seed=6)
    M = gpu_setup(prob, c, e, d, n)
    M.set_method(HDG_METHOD_BDM)
    M.assemble_condense(precision=HDG_DF32)
    Cg, Cfg = (t.cpu().numpy() for t in M.condensed())
    mesh = ExpandedMesh(c, e, d, n)
    tab = ohdg.Tables(k)
    X, Y, Z = ohdg.volume_nodes(mesh, tab)
    blk = ohdg.local_blocks(mesh, tab, prob.kappa(X, Y, Z), prob.c(X, Y, Z), prob.f(X, Y, Z), tau=0.0)
    CK, Cf, _, _ = obdm.local_solvers(blk, tab.d2)
    assert rel(Cg, CK) < 1e-11
    assert rel(Cfg, Cf) < 1e-11
    ref = obdm.solve_problem(prob, c, e, d, n)
    uhat, it, rr = M.solve_trace(rtol=1e-14, maxit=20000)
    q, u = M.recover(uhat)
    assert rel(u.cpu().numpy(), ref["u"]) < 1e-11
    assert rel(q.cpu().numpy(), ref["q"]) < 1e-11
