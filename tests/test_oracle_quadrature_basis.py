"""Pins of the oracle's quadrature rules and Dubiner bases (CPU only).

Closed forms: int_{K_hat} x^a y^b z^c = a! b! c! / (a+b+c+3)!, int_{K_hat_2} s^a t^b =
a! b! / (a+b+2)!; orthonormality of the bases (eq. 3.3, Section 4); hand-derived degree-1
Dubiner functions; central finite differences for the complex-step derivatives; integration
by parts on K_hat for C_hat (eq. 3.6-3.7); the F_mu maps of eq. 2.2 against their vertex table.
"""
from math import factorial

import numpy as np
import pytest

from oracle import basis, quadrature
from oracle.geometry import F_MU_TABLE


@pytest.mark.parametrize("k", [0, 1, 2, 3, 4])
def test_volume_rule_exact_to_degree_2k_plus_3(k):
    p, w, lam = quadrature.volume_rule(k)
    assert p.shape[0] == (k + 2) ** 3
    assert abs(w.sum() - 1) < 1e-14
    assert np.allclose(lam.sum(axis=1), 1) and np.all(lam > 0)
    for a in range(2 * k + 4):
        for b in range(2 * k + 4 - a):
            for c in range(2 * k + 4 - a - b):
                exact = factorial(a) * factorial(b) * factorial(c) / factorial(a + b + c + 3)
                got = np.sum(w * p[:, 0] ** a * p[:, 1] ** b * p[:, 2] ** c) / 6.0
                assert abs(got - exact) < 1e-15 + 1e-13 * exact, (a, b, c)


@pytest.mark.parametrize("k", [0, 1, 2, 3, 4])
def test_face_rule_exact_to_degree_2k_plus_3(k):
    q, w, xi = quadrature.face_rule(k)
    assert abs(w.sum() - 1) < 1e-14
    for a in range(2 * k + 4):
        for b in range(2 * k + 4 - a):
            exact = factorial(a) * factorial(b) / factorial(a + b + 2)
            got = np.sum(w * q[:, 0] ** a * q[:, 1] ** b) / 2.0
            assert abs(got - exact) < 1e-15 + 1e-13 * exact


def test_volume_rule_not_exact_beyond_degree():
    # z^(2k+4) is integrated inexactly: the rule is exactly of the claimed order.
    k = 2
    p, w, _ = quadrature.volume_rule(k)
    a = 2 * k + 4
    exact = factorial(a) / factorial(a + 3)
    assert abs(np.sum(w * p[:, 2] ** a) / 6 - exact) > 1e-8


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_dubiner3_orthonormal_and_hierarchical(k):
    p, w, _ = quadrature.volume_rule(k)
    P = basis.dubiner3(k, p)
    assert P.shape[1] == basis.d3(k)
    G = (w[:, None] * P).T @ P / 6.0  # int_{K_hat} P_i P_j
    assert np.allclose(G, np.eye(P.shape[1]) / 6.0, atol=1e-13)
    Pk1 = basis.dubiner3(k + 1, p)
    assert np.allclose(Pk1[:, :P.shape[1]], P, atol=1e-13)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_dubiner2_orthonormal_and_permuted(k):
    q, w, _ = quadrature.face_rule(k)
    D = basis.dubiner2(k, q)
    assert np.allclose((w[:, None] * D).T @ D / 2.0, np.eye(D.shape[1]) / 2.0, atol=1e-13)
    for mu in range(1, 7):
        Dm = basis.dubiner2(k, quadrature.F_mu(mu, q))
        # F_mu is an affine bijection of K_hat_2 with |det| = 1
        assert np.allclose((w[:, None] * Dm).T @ Dm, np.eye(D.shape[1]), atol=1e-13)


def test_dubiner_degree_one_closed_forms():
    rng = np.random.default_rng(0)
    pts = rng.dirichlet(np.ones(4), size=50)[:, 1:]
    x, y, z = pts.T
    P = basis.dubiner3(1, pts)
    assert np.allclose(P[:, 0], 1.0)
    # order: (p,q,r) = (0,0,1), (0,1,0), (1,0,0)
    assert np.allclose(P[:, 1], np.sqrt(5 / 3) * (4 * z - 1))
    assert np.allclose(P[:, 2], np.sqrt(10 / 3) * (3 * y + z - 1))
    assert np.allclose(P[:, 3], np.sqrt(10) * (2 * x + y + z - 1))
    tri = rng.dirichlet(np.ones(3), size=50)[:, 1:]
    s, t = tri.T
    D = basis.dubiner2(1, tri)
    assert np.allclose(D[:, 0], 1.0)
    assert np.allclose(D[:, 1], np.sqrt(2) * (3 * t - 1))
    assert np.allclose(D[:, 2], np.sqrt(6) * (2 * s + t - 1))


@pytest.mark.parametrize("k", [1, 3, 5])
def test_dubiner3_gradient_matches_finite_differences(k):
    rng = np.random.default_rng(1)
    pts = rng.dirichlet(np.ones(4), size=30)[:, 1:] * 0.9 + 0.02
    G = basis.dubiner3_grad(k, pts)
    h = 1e-6
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        fd = (basis.dubiner3(k, pts + e) - basis.dubiner3(k, pts - e)) / (2 * h)
        assert np.allclose(G[d], fd, atol=1e-6 * max(1, np.abs(fd).max()))


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_Chat_integration_by_parts(k):
    """C_hat^# + C_hat^#T = sum_l |e_l| nu_{l,#} (varpi . P^l)^T P^l over the faces of K_hat."""
    from oracle.hdg import Tables
    tab = Tables(k)
    S = [(tab.varpi[:, None] * tab.Pl[l]).T @ tab.Pl[l] for l in range(4)]
    # |e_l| nu_l: face 1 (z=0): (0,0,-1)/2; face 2 (y=0): (0,-1,0)/2; face 3 (x=0): (-1,0,0)/2;
    # face 4 (x+y+z=1): (1,1,1)/2
    bnd = [0.5 * (S[3] - S[2]), 0.5 * (S[3] - S[1]), 0.5 * (S[3] - S[0])]
    for s in range(3):
        assert np.allclose(tab.Chat[s] + tab.Chat[s].T, bnd[s], atol=1e-13)


def test_F_mu_vertex_table():
    w = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    for mu, img in F_MU_TABLE.items():
        out = quadrature.F_mu(mu, w)
        for i in range(3):
            assert np.allclose(out[i], w[img[i] - 1])
