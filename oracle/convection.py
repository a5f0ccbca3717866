"""HDG for convection-diffusion with variable convection (oracle; test infrastructure).

The paper (Section 9, "Matrices for convection-diffusion problems", eq. 9.1 and the two
surface matrices after it) provides the matrices
    int_K m P_i d_* P_j,   (xi/|e|) int_e alpha D_i P_j,   (xi/|e|) int_e alpha D_i D_j
and names the bilinear forms (beta . grad u, w)_K, <(beta.nu) u, v>, <(beta.nu) u_hat, v_hat>,
but does not write out the scheme.  Reading used (conservative form, flux of Chen-Cockburn
type):   div(q + beta u) + c u = f,  q = -kappa grad u,
  (kappa^-1 q, r) - (u, div r) + <u_hat, r.nu> = 0
  (div q, w) - (beta u, grad w) + <(beta.nu) u_hat + tau (u - u_hat), w> + (c u, w) = (f, w)
  sum_K <q.nu + (beta.nu) u_hat + tau (u - u_hat), v_hat> = 0 on interior faces.
So, against the reaction-diffusion blocks of hdg.py:
  A_1 last diagonal block   M_c + tauPP + B_c,   (B_c)_{ij} = -(beta P_j, grad P_i)_K
                            = -sum_* (int_K beta_* P_j d_* P_i)   (eq. 9.1 with m = beta_*)
  A_2 last block row        -(tauDP)^T + (alphaDP)^T,  alphaDP_{ij} = int_e (beta.nu) D_i P_j
  C^K = A_3 A_1^-1 A_2 + tauDD - alphaDD,  alphaDD_{ij} = int_e (beta.nu) D_i D_j
with A_3 unchanged.  The face integrals use the element parametrisation of eq. 4.1
(beta evaluated at the element's face nodes F_K(q_hat_r^l)), exactly as eq. 4.10 does.
The resulting trace matrix is not symmetric.
"""

import numpy as np

from . import hdg
from .geometry import piola_cofactors


def element_face_nodes(mesh, tab):
    """F_K(q_hat_r^l) for every element, local face and face node: [Nelt, 4, Nf] x 3."""
    v = mesh.coordinates[mesh.elements]  # [Nelt, 4, 3]
    B = mesh.B
    ql = tab.qhat_l  # [4, Nf, 3]
    pts = np.einsum("eab,lrb->elra", B, ql) + v[:, 0, None, None, :]
    return pts[..., 0], pts[..., 1], pts[..., 2]


def convection_blocks(mesh, tab, beta_q, beta_f, elems=None):
    """B_c [Nelt,n,n], alphaDP [Nelt,4 d2,n], alphaDD [Nelt,4 d2,4 d2].

    beta_q: (bx, by, bz) at the volume nodes, each [Nelt, Nq];
    beta_f: (bx, by, bz) at the element face nodes, each [Nelt, 4, Nf]."""
    idx = np.arange(mesh.nelt) if elems is None else np.asarray(elems)
    vol = mesh.volume[idx]
    a = piola_cofactors(mesh.coordinates, mesh.elements[idx])
    det = mesh.detB[idx]
    # eq. 9.1: int_K beta_* P_i d_* P_j with d_* P_j = sum_# (a_{*#}/det) d_hat_# P_hat_j
    grad = np.einsum("esh,hqj->esqj", a / det[:, None, None], tab.Pstar)  # [e, *, q, j]
    Cb = sum(vol[:, None, None] * np.einsum("q,eq,qi,eqj->eij", tab.w, beta_q[s][idx], tab.P, grad[:, s])
             for s in range(3))
    Bc = -np.transpose(Cb, (0, 2, 1))
    d2 = tab.d2
    perm = mesh.perm[idx]
    N = mesh.normals[idx]  # |n_l| = |e_l|, so |e| (beta . nu) = beta . n_l
    aDP = np.zeros((len(idx), 4 * d2, tab.n))
    aDD = np.zeros((len(idx), 4 * d2, 4 * d2))
    for l in range(4):
        bn = sum(beta_f[s][idx][:, l, :] * N[:, l, s, None] for s in range(3))  # [e, Nf]
        for mu in range(1, 7):
            sel = perm[:, l] == mu
            if not np.any(sel):
                continue
            Dm = tab.Dmu[mu - 1]
            aDP[sel, l * d2:(l + 1) * d2, :] = np.einsum("r,er,ri,rj->eij", tab.varpi, bn[sel], Dm, tab.Pl[l])
            aDD[sel, l * d2:(l + 1) * d2, l * d2:(l + 1) * d2] = np.einsum("r,er,ri,rj->eij", tab.varpi, bn[sel], Dm, Dm)
    return Bc, aDP, aDD


def local_solvers_conv(blk, Bc, aDP, aDD):
    """C^K, C_f^K and the eq. 5.3 pieces for the convection reading above (LU of A_1)."""
    A1, A2, Af, A3 = hdg.local_matrices(blk)
    n = blk["M_kinv"].shape[1]
    A1 = A1.copy()
    A1[:, 3 * n:, 3 * n:] += Bc
    A2 = A2.copy()
    A2[:, 3 * n:, :] += np.transpose(aDP, (0, 2, 1))
    rhs = np.concatenate([A2, Af[:, :, None]], axis=2)
    X = np.linalg.solve(A1, rhs)
    X2, xf = X[:, :, :-1], X[:, :, -1]
    CK = A3 @ X2 + blk["tDD"] - aDD
    Cf = np.einsum("eij,ej->ei", A3, xf)
    return CK, Cf, X2, xf, (A1, A2, Af, A3)


def solve_problem_conv(prob, coords, elems, dirichlet, neumann, rule="conical"):
    """Whole pipeline for a convection problem with Dirichlet data on every face, on the
    volume rule `rule`."""
    from .geometry import ExpandedMesh

    mesh = ExpandedMesh(coords, elems, dirichlet, neumann)
    tab = hdg.Tables(prob.k, rule)
    X, Y, Z = hdg.volume_nodes(mesh, tab)
    kap, cq, fq = prob.kappa(X, Y, Z), prob.c(X, Y, Z), prob.f(X, Y, Z)
    blk = hdg.local_blocks(mesh, tab, kap, cq, fq, tau=prob.tau)
    bq = prob.beta(X, Y, Z)
    FX, FY, FZ = element_face_nodes(mesh, tab)
    bf = prob.beta(FX, FY, FZ)
    Bc, aDP, aDD = convection_blocks(mesh, tab, bq, bf)
    CK, Cf, X2, xf, mats = local_solvers_conv(blk, Bc, aDP, aDD)
    H, F = hdg.assemble(mesh, tab.d2, CK, Cf)
    DX, DY, DZ = hdg.face_nodes(mesh, tab, mesh.dirfaces)
    uhatD = hdg.dirichlet_data(tab, prob.uD(DX, DY, DZ))
    PhiN = None
    if len(mesh.neufaces):
        raise NotImplementedError("the convection workloads use Dirichlet data on every face")
    uhat, H, b, free = hdg.solve_trace(mesh, tab.d2, H, F, uhatD, PhiN)
    q, u = hdg.recover(mesh, X2, xf, uhat)
    return dict(mesh=mesh, tab=tab, blk=blk, Bc=Bc, aDP=aDP, aDD=aDD, CK=CK, Cf=Cf, X2=X2, xf=xf,
                H=H, b=b, free=free, uhatD=uhatD, uhat=uhat, q=q, u=u, kappa_q=kap, mats=mats)


def monolithic_solve_conv(mesh, tab, mats, tDD, aDD, uhatD):
    """Dense solve of the full convection system in (q, u, u_hat) (tiny meshes)."""
    A1, A2, Af, A3 = mats
    ne, n4 = A1.shape[0], A1.shape[1]
    d2 = tab.d2
    nloc = ne * n4
    ntot = nloc + mesh.nfc * d2
    A = np.zeros((ntot, ntot))
    b = np.zeros(ntot)
    dof = hdg.dofs(mesh, d2) + nloc
    for K in range(ne):
        r = slice(K * n4, (K + 1) * n4)
        A[r, r] = A1[K]
        A[r, dof[K]] = A2[K]
        b[r] = Af[K]
        A[np.ix_(dof[K], np.arange(K * n4, (K + 1) * n4))] += -A3[K]
        A[np.ix_(dof[K], dof[K])] += tDD[K] - aDD[K]
    for i, e in enumerate(mesh.dirfaces):
        rr = slice(nloc + e * d2, nloc + (e + 1) * d2)
        A[rr, :] = 0.0
        A[rr, rr] = np.eye(d2)
        b[rr] = uhatD[i]
    x = np.linalg.solve(A, b)
    loc = x[:nloc].reshape(ne, n4)
    n = n4 // 4
    return loc[:, :3 * n].reshape(ne, 3, n), loc[:, 3 * n:], x[nloc:].reshape(mesh.nfc, d2)
