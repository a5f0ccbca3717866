"""Pins of the oracle's hybridised BDM element (Section 9, "BDM") against what the
mathematics of mixed methods fixes.

* exactness: with u in P_{k-1}, kappa constant and variable c, the exact (q, u) lies in the
  BDM spaces, so q_h, u_h equal the L2 projections of q, u (the degree-k part of u_h is zero)
  and u_hat the face projection of u;
* q_h is H(div)-conforming: its normal component agrees from both sides of every interior
  face (HDG with tau > 0 does not have this; the test checks that too);
* the local equilibrium of eq. 1.2b with tau = 0: (div q_h + c u_h - f, w)_K = 0 for every w in
  P_{k-1}(K), with div q_h formed from the basis gradients;
* observed orders k + 1 for q and k for u.
"""
import numpy as np
import pytest

from oracle import basis, bdm, hdg
from workloads import get_problem

from test_oracle_hdg import _poly_problem, _varcoef


@pytest.mark.parametrize("k", [2, 3])
def test_bdm_exact_for_u_in_P_k_minus_1(k):
    prob = _poly_problem(k - 1, 2).at(k=k)
    r = bdm.solve_problem(prob)
    m, tab = r["mesh"], r["tab"]
    X, Y, Z = hdg.volume_nodes(m, tab)
    u_ex = (prob.u(X, Y, Z) * tab.w) @ tab.P
    qv = prob.q(X, Y, Z)
    q_ex = np.stack([(qv[a] * tab.w) @ tab.P for a in range(3)], axis=1)
    FX, FY, FZ = hdg.face_nodes(m, tab)
    uh_ex = (prob.u(FX, FY, FZ) * tab.varpi) @ tab.D
    assert np.abs(r["u"][:, tab.n - tab.d2:]).max() == 0.0
    assert np.abs(r["u"] - u_ex).max() < 1e-11
    assert np.abs(r["q"] - q_ex).max() < 1e-11
    assert np.abs(r["uhat"] - uh_ex).max() < 1e-11


def _normal_jumps(r, k):
    """max over interior faces and face nodes of |q_K1.nu - q_K2.nu|, and max |q.nu|."""
    m, tab = r["mesh"], r["tab"]
    FX, FY, FZ = hdg.face_nodes(m, tab)
    pts = np.stack([FX, FY, FZ], axis=2)  # [Nfc, Nf, 3]
    owners = [[] for _ in range(m.nfc)]
    for K in range(m.nelt):
        for l in range(4):
            owners[m.facebyele[K, l]].append((K, l))
    Binv = np.linalg.inv(m.B)
    v0 = m.coordinates[m.elements[:, 0]]
    jump, scale = 0.0, 0.0
    for e in range(m.nfc):
        if len(owners[e]) != 2:
            continue
        (K1, l1), (K2, _) = owners[e]
        nu = m.normals[K1, l1] / np.linalg.norm(m.normals[K1, l1])
        vals = []
        for K in (K1, K2):
            xh = (pts[e] - v0[K]) @ Binv[K].T
            P = basis.dubiner3(k, xh)
            vals.append((r["q"][K] @ P.T).T @ nu)
        jump = max(jump, np.abs(vals[0] - vals[1]).max())
        scale = max(scale, np.abs(vals[0]).max())
    return jump, scale


@pytest.mark.parametrize("k", [1, 2])
def test_bdm_flux_is_normal_continuous(k):
    kap_f, c_f = _varcoef()
    prob = get_problem("cube16_k3").at(s=2, k=k)
    prob.c = c_f
    prob.jitter, prob.seed = 0.15, 9
    jb, sb = _normal_jumps(bdm.solve_problem(prob), k)
    assert jb < 1e-11 * sb
    jh, sh = _normal_jumps(hdg.solve_problem(prob), k)
    assert jh > 1e-4 * sh  # the HDG flux q_h alone jumps (its trace adds tau (u - u_hat))


@pytest.mark.parametrize("k", [1, 2, 3])
def test_bdm_local_equilibrium(k):
    kap_f, c_f = _varcoef()
    prob = get_problem("cube16_k3").at(s=2, k=k)
    prob.c = c_f
    prob.jitter, prob.seed = 0.15, 11
    r = bdm.solve_problem(prob)
    m, tab = r["mesh"], r["tab"]
    X, Y, Z = hdg.volume_nodes(m, tab)
    Binv_T = np.transpose(np.linalg.inv(m.B), (0, 2, 1))
    grad = np.einsum("eab,bqi->eaqi", Binv_T, tab.Pstar)  # physical gradients [e, 3, Nq, n]
    div = np.einsum("eai,eaqi->eq", r["q"], grad)
    uh = r["u"] @ tab.P.T
    res = (div + prob.c(X, Y, Z) * uh - prob.f(X, Y, Z)) * tab.w
    nlow = tab.n - tab.d2
    moments = m.volume[:, None] * (res @ tab.P[:, :nlow])
    scale = np.abs(m.volume[:, None] * ((prob.f(X, Y, Z) * tab.w) @ tab.P[:, :nlow])).max()
    assert np.abs(moments).max() < 1e-11 * scale


@pytest.mark.parametrize("k", [1, 2])
def test_bdm_convergence_orders(k):
    prob = get_problem("cube4_k1").at(k=k)
    errs = []
    for s in (4, 8):
        r = bdm.solve_problem(prob.at(s=s))
        errs.append(hdg.errors(r["mesh"], k, r["q"], r["u"], r["uhat"], r["ustar"], prob.at(s=s)))
    rate = {a: np.log2(errs[0][a] / errs[1][a]) for a in errs[0]}
    assert abs(rate["e_q"] - (k + 1)) < 0.3, rate
    assert abs(rate["e_u"] - k) < 0.3, rate
