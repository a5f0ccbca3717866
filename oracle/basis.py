"""Dubiner bases on the reference tetrahedron and triangle (oracle; test infrastructure).

Eq. 3.3 and Section 4 "Bases, faces, and boundaries": hierarchical Dubiner bases, orthogonal
on the enlarged elements 2K-(1,1,1) and 2K_2-(1,1), pulled back to K_hat and K_hat_2.

Readings (the paper fixes neither normalisation nor the order inside one degree):
  * normalisation: int_{K_hat} P_i P_j = |K_hat| delta_ij and int_{K_hat_2} D_i D_j = (1/2) delta_ij,
    so int_K P_i^K P_j^K = |K| delta_ij and int_e D_i^e D_j^e = |e| delta_ij;
  * order: by total degree, then (p, q[, r]) lexicographically with p outermost.

In collapsed coordinates (Kirby 2010; Karniadakis-Sherwin), with xi = 2 x_hat - 1:
  3-D: P_pqr = N * P_p(a) (1-y-z)^p * P_q^(2p+1,0)(b) (1-z)^q * P_r^(2p+2q+2,0)(c),
       a = 2x/(1-y-z) - 1, b = 2y/(1-z) - 1, c = 2z - 1,  N^2 = (2p+1)(p+q+1)(2p+2q+2r+3)/3
  2-D: D_pq  = N * P_p(a) (1-t)^p * P_q^(2p+1,0)(b),  a = 2s/(1-t) - 1, b = 2t - 1,
       N^2 = (2p+1)(p+q+1)
The Jacobi polynomials are scipy's (library primitive).  Derivatives are taken by complex-step
differentiation (Squire and Trapp 1998), d f/dx = Im f(x + i h)/h, which is exact to rounding
for these real-analytic expressions and independent of any hand-derived chain rule.
"""

import numpy as np
from scipy.special import eval_jacobi

_H = 1e-30


def index3(k):
    """(p, q, r) of the 3-D basis functions, hierarchical order; length d3 = C(k+3,3)."""
    return [(p, q, d - p - q) for d in range(k + 1) for p in range(d + 1) for q in range(d - p + 1)]


def index2(k):
    """(p, q) of the 2-D basis functions, hierarchical order; length d2 = C(k+2,2)."""
    return [(p, d - p) for d in range(k + 1) for p in range(d + 1)]


def d3(k):
    return (k + 1) * (k + 2) * (k + 3) // 6


def d2(k):
    return (k + 1) * (k + 2) // 2


def _p3(p, q, r, x, y, z):
    a = 2 * x / (1 - y - z) - 1
    b = 2 * y / (1 - z) - 1
    c = 2 * z - 1
    nrm = np.sqrt((2 * p + 1) * (p + q + 1) * (2 * p + 2 * q + 2 * r + 3) / 3.0)
    return (nrm * eval_jacobi(p, 0.0, 0.0, a) * (1 - y - z) ** p
            * eval_jacobi(q, 2 * p + 1.0, 0.0, b) * (1 - z) ** q
            * eval_jacobi(r, 2 * p + 2 * q + 2.0, 0.0, c))


def _p2(p, q, s, t):
    a = 2 * s / (1 - t) - 1
    b = 2 * t - 1
    nrm = np.sqrt((2 * p + 1) * (p + q + 1.0))
    return nrm * eval_jacobi(p, 0.0, 0.0, a) * (1 - t) ** p * eval_jacobi(q, 2 * p + 1.0, 0.0, b)


def dubiner3(k, pts):
    """Values [npts, d3] of P_hat_i at reference points pts [npts,3] (eq. 3.5)."""
    x, y, z = (np.asarray(pts[:, i], dtype=np.float64) for i in range(3))
    return np.column_stack([_p3(p, q, r, x, y, z) for (p, q, r) in index3(k)])


def dubiner3_grad(k, pts):
    """Derivatives [3, npts, d3]: d/dx_hat, d/dy_hat, d/dz_hat of P_hat_i (eq. 3.66)."""
    x, y, z = (np.asarray(pts[:, i], dtype=np.float64) for i in range(3))
    out = []
    for dx, dy, dz in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
        xc = x + 1j * _H * dx
        yc = y + 1j * _H * dy
        zc = z + 1j * _H * dz
        out.append(np.column_stack([np.imag(_p3(p, q, r, xc, yc, zc)) / _H for (p, q, r) in index3(k)]))
    return np.stack(out)


def dubiner2(k, pts):
    """Values [npts, d2] of D_hat_i at reference triangle points pts [npts,2] (eq. 4.7)."""
    s, t = np.asarray(pts[:, 0], dtype=np.float64), np.asarray(pts[:, 1], dtype=np.float64)
    return np.column_stack([_p2(p, q, s, t) for (p, q) in index2(k)])
