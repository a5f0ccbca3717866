"""Quadrature rules on the reference tetrahedron and triangle (oracle; test infrastructure).

The paper leaves the rules open (eq. 3.1 and Section 4 "Integrals on faces": any rule of
sufficient order, weights summing to one).  Reading used on both sides of the parity tests:
conical-product Gauss-Jacobi rules with n = k + 2 points per collapsed direction, exact for
total degree 2n - 1 = 2k + 3.

Volume (eq. 3.1): with t1 ~ Gauss-Jacobi weight (1-t)^2, t2 ~ (1-t)^1, t3 ~ Gauss-Legendre on
[0,1],  z = t1,  y = t2 (1 - t1),  x = t3 (1 - t1)(1 - t2).  Node index q = (i n + j) n + l
for (t1_i, t2_j, t3_l).  Weights omega_hat = 6 w so that sum omega_hat = 1.

Face (Section 4): t = u1 ~ weight (1-u)^1, s = u2 (1 - u1), u2 ~ Gauss-Legendre.  Node index
r = i n + j.  Weights varpi = 2 w, summing to one.

The 1-D Gauss-Jacobi nodes come from scipy (library primitive).
"""

import numpy as np
from scipy.special import roots_jacobi


def gauss_jacobi01(n, alpha):
    """n-point Gauss rule on [0,1] for the weight (1-t)^alpha (maps scipy's [-1,1] rule)."""
    x, w = roots_jacobi(n, alpha, 0.0)
    return (x + 1.0) / 2.0, w / 2.0 ** (alpha + 1)


def volume_rule(k):
    """Nodes p_hat [Nq,3], weights omega_hat [Nq] (sum 1), barycentrics Lambda [Nq,4] (eq. 3.1)."""
    n = k + 2
    t1, w1 = gauss_jacobi01(n, 2.0)
    t2, w2 = gauss_jacobi01(n, 1.0)
    t3, w3 = gauss_jacobi01(n, 0.0)
    pts, wts = [], []
    for i in range(n):
        for j in range(n):
            for l in range(n):
                z = t1[i]
                y = t2[j] * (1 - t1[i])
                x = t3[l] * (1 - t1[i]) * (1 - t2[j])
                pts.append((x, y, z))
                wts.append(w1[i] * w2[j] * w3[l])
    p = np.array(pts)
    w = 6.0 * np.array(wts)
    lam = np.column_stack([1 - p.sum(axis=1), p[:, 0], p[:, 1], p[:, 2]])
    return p, w, lam


def face_rule(k):
    """Nodes q_hat [Nf,2] = (s,t), weights varpi [Nf] (sum 1), barycentrics Xi [Nf,3]."""
    n = k + 2
    u1, w1 = gauss_jacobi01(n, 1.0)
    u2, w2 = gauss_jacobi01(n, 0.0)
    pts, wts = [], []
    for i in range(n):
        for j in range(n):
            t = u1[i]
            s = u2[j] * (1 - u1[i])
            pts.append((s, t))
            wts.append(w1[i] * w2[j])
    q = np.array(pts)
    w = 2.0 * np.array(wts)
    xi = np.column_stack([1 - q.sum(axis=1), q[:, 0], q[:, 1]])
    return q, w, xi


def face_points_on_reference_tet(qhat):
    """The four groups q_hat^l of Section 4 "Integrals on boundaries of tetrahedra":
    (s,t,0), (s,0,t), (0,s,t), (s,t,1-s-t).  Returns [4, Nf, 3]."""
    s, t = qhat[:, 0], qhat[:, 1]
    zero = np.zeros_like(s)
    return np.stack([
        np.column_stack([s, t, zero]),
        np.column_stack([s, zero, t]),
        np.column_stack([zero, s, t]),
        np.column_stack([s, t, 1 - s - t]),
    ])


def F_mu(mu, qhat):
    """The six affine maps F_mu of the reference triangle, eq. 2.2 (mu = 1..6)."""
    s, t = qhat[..., 0], qhat[..., 1]
    r = 1 - s - t
    table = {
        1: (s, t),
        2: (t, s),
        3: (t, r),
        4: (s, r),
        5: (r, s),
        6: (r, t),
    }
    a, b = table[mu]
    return np.stack([a, b], axis=-1)


def symmetric_volume_rule(k):
    """Grundmann-Moller rule of index s = k + 1 on the reference tetrahedron (Grundmann and
    Moller, SIAM J. Numer. Anal. 15, 1978): exact to degree 2s + 1 = 2k + 3 like volume_rule(k)
    but with C(s + 4, 4) nodes instead of (k + 2)^3 (k = 2: 35 against 64; k = 3: 70 against
    125) -- the smaller symmetric rule of the paper's remark on quadrature.  With d = 2s + 1 and
    dimension 3, level i = 0..s contributes the nodes with barycentric coordinates
    (2 beta_j + 1) / (d + 3 - 2i) for every beta in N^4 with |beta| = s - i, all with the weight
    (-1)^i 2^-2s (d + 3 - 2i)^d / (i! (d + 3 - i)!) (a rule for the simplex of volume 1/3!; the
    weights here are scaled by 3! to sum to one, the paper's convention).  Some weights are
    negative.  Returns the same triple as volume_rule: nodes [Nq,3], weights [Nq], barycentrics."""
    from itertools import product
    from math import factorial

    s = k + 1
    d = 2 * s + 1
    pts, wts = [], []
    for i in range(s + 1):
        wt = (-1) ** i * 2.0 ** (-2 * s) * float(d + 3 - 2 * i) ** d / (factorial(i) * factorial(d + 3 - i))
        m = s - i
        for beta in product(range(m + 1), repeat=4):
            if sum(beta) != m:
                continue
            lam = [(2 * b + 1) / (d + 3 - 2 * i) for b in beta]
            pts.append((lam[1], lam[2], lam[3]))
            wts.append(wt)
    p = np.array(pts)
    w = 6.0 * np.array(wts)
    lam = np.column_stack([1 - p.sum(axis=1), p[:, 0], p[:, 1], p[:, 2]])
    return p, w, lam
