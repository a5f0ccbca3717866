"""HDG projection (eq. 9.13), face L2 projection (eq. 9.12) and the superconvergence
diagnostics of eq. 10.2, in FP64 (oracle; test infrastructure only).

hdg_projection   eq. 9.13: per element, (q_h, u_h) in P_k(K)^3 x P_k(K) with
                 (q_h, r)_K = (q, r)_K for r in P_{k-1}(K)^3, (u_h, w)_K = (u, w)_K for w in
                 P_{k-1}(K), <q_h.nu + tau u_h, v>_dK = <q.nu + tau u, v>_dK for v in R_k(dK);
                 the square 4n x 4n system of the paper (the tilde-M rows, then the row
                 [n_x DP, n_y DP, n_z DP, tau DP]), solved densely
face_projection  eq. 9.12 (the formula of eq. 6.3 on every face)
norm2_volume     sum_K |K| sum_q omega_q (v - sum_j c_j P_j)^2 on a volume rule
norm2_faces      ||.||_h^2 of eq. 10.2: sum_e |e| ||.||_e^2, ||v||_e^2 = |e| sum_r varpi_r v_r^2
superconvergence the ratios eps^u and eps^uhat of eq. 10.2

The projection is defined with the same volume and face rules as the rest of the oracle (the
degree-k rules, exact to total degree 2k + 3): the integrals of q and u against P_{k-1} and
against the traces are then exact for polynomial data up to degree k + 4 (volume) and k + 3
(faces).  Inputs are the values of q and u at those nodes, as for the coefficients.
"""

import numpy as np

from . import basis, quadrature
from .hdg import dirichlet_data, local_blocks


def element_face_points(mesh, tab):
    """F_K(q_hat_r^l) of eq. 4.1: the element-local face nodes, [Nelt, 4, Nf, 3]."""
    v0 = mesh.coordinates[mesh.elements[:, 0]]  # [Nelt, 3]
    return v0[:, None, None, :] + np.einsum("edj,lrj->elrd", mesh.B, tab.qhat_l)


def hdg_projection(mesh, tab, q_vol, u_vol, q_face, u_face, tau=1.0):
    """eq. 9.13.  q_vol [3, Nelt, Nq] and u_vol [Nelt, Nq]: q and u at the volume nodes;
    q_face [3, Nelt, 4, Nf] and u_face [Nelt, 4, Nf]: at the element-local face nodes
    F_K(q_hat_r^l).  tau: scalar or [Nelt, 4].  Returns Pi q [Nelt, 3, n], Pi u [Nelt, n]."""
    n, d2 = tab.n, tab.d2
    nlow = n - d2  # dim P_{k-1}(K): the basis is hierarchical, ordered by degree
    ne = mesh.nelt
    vol = mesh.volume
    zero = np.zeros((ne, tab.nq))
    blk = local_blocks(mesh, tab, np.ones((ne, tab.nq)), zero, zero, tau=tau)
    # tilde-M: the first nlow rows of the unit-weight mass matrix (eq. 3.55 with m = 1)
    Mt = vol[:, None, None] * np.einsum("q,qi,qj->ij", tab.w, tab.P[:, :nlow], tab.P)[None]
    A = np.zeros((ne, 4 * n, 4 * n))
    rhs = np.zeros((ne, 4 * n))
    for c in range(4):
        A[:, c * nlow:(c + 1) * nlow, c * n:(c + 1) * n] = Mt
        vals = q_vol[c] if c < 3 else u_vol
        rhs[:, c * nlow:(c + 1) * nlow] = vol[:, None] * np.einsum("eq,q,qi->ei", vals, tab.w, tab.P[:, :nlow])
    r0 = 4 * nlow
    for c in range(3):
        A[:, r0:, c * n:(c + 1) * n] = blk["nDP"][c]
    A[:, r0:, 3 * n:] = blk["tDP"]
    # <q.nu + tau u, D_a>_{e_l} = sum_r varpi_r (q.N_l + T_l u)(x_r^l) D^mu_a(q_hat_r), with
    # N_l = |e_l| nu_l and T_l = tau_l |e_l| (eq. 4.22); mu = perm(K, l)
    N = mesh.normals  # [Nelt, 4, 3]
    T = np.broadcast_to(np.asarray(tau, dtype=np.float64), (ne, 4)) * mesh.elem_area
    g = sum(N[:, :, c, None] * q_face[c] for c in range(3)) + T[:, :, None] * u_face  # [Nelt,4,Nf]
    for l in range(4):
        Dl = tab.Dmu[mesh.perm[:, l] - 1]  # [Nelt, Nf, d2]
        rhs[:, r0 + l * d2:r0 + (l + 1) * d2] = np.einsum("r,er,era->ea", tab.varpi, g[:, l], Dl)
    x = np.linalg.solve(A, rhs[:, :, None])[:, :, 0]
    return x[:, :3 * n].reshape(ne, 3, n), x[:, 3 * n:]


def face_projection(tab, u_fnodes):
    """eq. 9.12 on every face: P u = ((varpi . D)^T D)^-1 (varpi . D)^T u(face nodes).
    u_fnodes [Nfc, Nf] at the face nodes of the sorted-vertex parametrisation (eq. 6.2)."""
    return dirichlet_data(tab, u_fnodes)


def norm2_volume(mesh, k, coef, vals, degree):
    """(sum_K |K| sum_q omega_q (vals - sum_j coef_j P_j)^2, sum_K |K| sum_q omega_q vals^2) on
    the degree-k volume rule; coef in the degree-`degree` basis ([Nelt, d3(degree)]) or None,
    vals [Nelt, Nq] or None (zero)."""
    p, w, _ = quadrature.volume_rule(k)
    vol = mesh.volume
    v = np.zeros((mesh.nelt, p.shape[0])) if vals is None else np.asarray(vals)
    f = v - (0.0 if coef is None else coef @ basis.dubiner3(degree, p).T)
    return float(np.sum(vol[:, None] * w[None, :] * f ** 2)), float(np.sum(vol[:, None] * w[None, :] * v ** 2))


def norm2_faces(mesh, k, coef, vals):
    """(||vals - sum_a coef_a D_a||_h^2, ||vals||_h^2) of eq. 10.2 on the degree-k face rule;
    coef [Nfc, d2] or None, vals [Nfc, Nf] or None (zero)."""
    qf, wf, _ = quadrature.face_rule(k)
    a2 = mesh.area[:, None] ** 2
    v = np.zeros((mesh.nfc, qf.shape[0])) if vals is None else np.asarray(vals)
    f = v - (0.0 if coef is None else coef @ basis.dubiner2(k, qf).T)
    return float(np.sum(a2 * wf * f ** 2)), float(np.sum(a2 * wf * v ** 2))


def superconvergence(mesh, k, Pi_u, u_h, Pu, uhat, u_vol, u_fnodes):
    """eps^u = ||Pi u - u_h||_Omega / ||u||_Omega and eps^uhat = ||P u - uhat_h||_h / ||u||_h
    (eq. 10.2), on the degree-k rules."""
    e_u, r_u = norm2_volume(mesh, k, Pi_u - u_h, None, k)
    _, r_u = norm2_volume(mesh, k, None, u_vol, k)
    e_f, _ = norm2_faces(mesh, k, Pu - uhat, None)
    _, r_f = norm2_faces(mesh, k, None, u_fnodes)
    return dict(eps_u=float(np.sqrt(e_u / r_u)), eps_uhat=float(np.sqrt(e_f / r_f)))
