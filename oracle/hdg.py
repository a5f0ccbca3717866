"""HDG for variable-coefficient reaction-diffusion in FP64 (oracle; test infrastructure).

Follows Sections 3-6 and 9 of Fu, Gatica, Sayas (arXiv 1305.1489) step by step:

  Tables            eq. 3.5, 3.66, 3.7 (P, P^*, C_hat^*), eq. 4.4, 4.7 and Section 4 type (c)
                    (P^l, D, D^mu)
  local_blocks      eq. 3.55 (mass), 3.56 (C_*), 4.5 (tauPP), 4.8 (tauDD), 4.10 (n_*DP, tauDP),
                    Section 3 "Source terms" (f^K)
  local_solvers     eq. 5.1, 5.2, 5.4, 5.5, 5.6: A_1 (with C_z in the last block row, see below)
                    is factored by dense LU with partial pivoting (numpy.linalg.solve)
  assemble          Section 6 "Assembly process", eq. 6.5 (CSR via scipy.sparse, accumarray)
  dirichlet_data    eq. 6.1-6.3;  neumann_data  eq. 6.4
  solve_trace       Dirichlet elimination (Section 6) + sparse direct solve (scipy spsolve)
  recover           Section 6 "Reconstruction", eq. 5.3
  postprocess       eq. 9.11 (bordered system for the mean constraint)
  errors            eq. 10.1 and Section 9 "Error functions"
  monolithic_solve  the full square system eq. 1.2 in (q_h, u_h, u_hat), dense

Readings of the paper where it is silent or misprinted:
  * eq. 5.1 prints C_y twice in the last block row of A_1; eq. 1.2b, (div q, w), requires
    (C_x, C_y, C_z).
  * the bilinear form a_1 after eq. 5.2 prints "kappa^-1 boldsymbol_h" and <tau u_h, v_h>;
    read (kappa^-1 q_h, r_h) and <tau u_h, w_h>.
  * eq. 6.1 prints D_j(q_hat_j); read D_j(q_hat_r).
  * quadrature rules and basis normalisation/ordering: see quadrature.py and basis.py.
Array layout: element-major, i.e. [Nelt, ...] (the paper stores the transpose, d x Nelt).
"""

import numpy as np
import scipy.sparse as sps
import scipy.sparse.linalg as spla

from . import basis, quadrature
from .geometry import ExpandedMesh, piola_cofactors


def volume_rule(k, rule="conical"):
    """The volume rule of eq. 3.1: the conical product (default) or the smaller symmetric rule
    of the same degree (quadrature.symmetric_volume_rule)."""
    if rule == "conical":
        return quadrature.volume_rule(k)
    if rule == "symmetric":
        return quadrature.symmetric_volume_rule(k)
    raise ValueError(rule)


class Tables:
    """Reference-element tables for degree k (Sections 3 and 4) on the volume rule `rule`."""

    def __init__(self, k, rule="conical"):
        self.k = k
        self.rule = rule
        self.n = basis.d3(k)
        self.d2 = basis.d2(k)
        self.p, self.w, self.Lambda = volume_rule(k, rule)  # eq. 3.1
        self.P = basis.dubiner3(k, self.p)  # eq. 3.5
        self.Pstar = basis.dubiner3_grad(k, self.p)  # eq. 3.66, [3, Nq, n]
        # eq. 3.7: C_hat^* = (1/6) (omega_hat . P)^T P^*
        self.Chat = np.stack([(self.w[:, None] * self.P).T @ self.Pstar[s] / 6.0 for s in range(3)])
        self.qf, self.varpi, self.Xi = quadrature.face_rule(k)
        self.qhat_l = quadrature.face_points_on_reference_tet(self.qf)  # [4, Nf, 3]
        self.Pl = np.stack([basis.dubiner3(k, self.qhat_l[l]) for l in range(4)])  # eq. 4.4
        self.D = basis.dubiner2(k, self.qf)  # eq. 4.7
        self.Dmu = np.stack([basis.dubiner2(k, quadrature.F_mu(mu, self.qf)) for mu in range(1, 7)])

    @property
    def nq(self):
        return self.p.shape[0]

    @property
    def nf(self):
        return self.qf.shape[0]


def volume_nodes(mesh, tab):
    """X, Y, Z of eq. 3.4 as [Nelt, Nq] (X = Lambda X^T, transposed)."""
    v = mesh.coordinates[mesh.elements]  # [Nelt, 4, 3]
    return tuple(v[:, :, d] @ tab.Lambda.T for d in range(3))


def face_nodes(mesh, tab, which=None):
    """Face quadrature points q_r^e = phi_e(q_hat_r) as in eq. 6.2, [len(which), Nf] x 3."""
    f = mesh.faces if which is None else mesh.faces[which]
    v = mesh.coordinates[f]  # [F, 3, 3], sorted-vertex parametrisation
    return tuple(v[:, :, d] @ tab.Xi.T for d in range(3))


def local_blocks(mesh, tab, kappa_q, c_q, f_q, tau=1.0, elems=None):
    """All per-element matrices of Sections 3-5 for the elements `elems` (default: all).

    kappa_q, c_q, f_q: coefficient values at the volume nodes, [Nelt, Nq].
    tau: scalar or [Nelt, 4] (piecewise constant on each face of each element).
    """
    idx = np.arange(mesh.nelt) if elems is None else np.asarray(elems)
    vol = mesh.volume[idx]
    a = piola_cofactors(mesh.coordinates, mesh.elements[idx])  # eq. 3.8
    tauK = np.broadcast_to(np.asarray(tau, dtype=np.float64), (mesh.nelt, 4))[idx]
    area = mesh.elem_area[idx]  # |e_l^K|
    T = tauK * area  # eq. 4.22
    N = mesh.normals[idx]  # N^*_{l,K} = n^K_{l,*}, eq. 4.22
    perm = mesh.perm[idx]

    # eq. 3.55: M = vol . m(X,Y,Z);  sum_q m_q (x) (omega_q p_q p_q^T)
    def mass(m):
        Mq = vol[:, None] * m[idx]
        return np.einsum("eq,q,qi,qj->eij", Mq, tab.w, tab.P, tab.P)

    M_kinv = mass(1.0 / kappa_q)
    M_c = mass(c_q)
    # eq. 3.56: C_* = sum_# a_{*#} (x) C_hat^#
    C = tuple(np.einsum("es,sij->eij", a[:, s], tab.Chat) for s in range(3))
    # eq. 4.5: tauPP = sum_l t_l (x) ((varpi . P^l)^T P^l)
    S_l = np.stack([(tab.varpi[:, None] * tab.Pl[l]).T @ tab.Pl[l] for l in range(4)])
    tPP = np.einsum("el,lij->eij", T, S_l)
    # eq. 4.8: tauDD block diagonal, block l = t_l (varpi . D)^T D
    DD = (tab.varpi[:, None] * tab.D).T @ tab.D
    d2 = tab.d2
    tDD = np.zeros((len(idx), 4 * d2, 4 * d2))
    for l in range(4):
        tDD[:, l * d2:(l + 1) * d2, l * d2:(l + 1) * d2] = T[:, l, None, None] * DD
    # eq. 4.9-4.10: xi DP, block l = sum_mu xi_{l,mu} (varpi . D^mu)^T P^l
    E = np.stack([[(tab.varpi[:, None] * tab.Dmu[mu]).T @ tab.Pl[l] for mu in range(6)]
                  for l in range(4)])  # [4 (l), 6 (mu), d2, n]

    def xiDP(xi):
        out = np.zeros((len(idx), 4 * d2, tab.n))
        for l in range(4):
            for mu in range(1, 7):
                xi_lmu = xi[:, l] * (perm[:, l] == mu)
                out[:, l * d2:(l + 1) * d2, :] += xi_lmu[:, None, None] * E[l, mu - 1]
        return out

    nDP = tuple(xiDP(N[:, :, s]) for s in range(3))
    tDP = xiDP(T)
    # Section 3 "Source terms": vol^T . ((omega . P)^T f(X,Y,Z))
    fK = vol[:, None] * (f_q[idx] * tab.w[None, :]) @ tab.P
    return dict(M_kinv=M_kinv, M_c=M_c, C=C, tPP=tPP, tDD=tDD, nDP=nDP, tDP=tDP, f=fK)


def local_matrices(blk):
    """A_1, A_2, A_f, A_3 of eq. 5.1, 5.2, 5.4 (last block row of A_1: C_x, C_y, C_z)."""
    M = blk["M_kinv"]
    Cx, Cy, Cz = blk["C"]
    ne, n, _ = M.shape
    Z = np.zeros_like(M)
    tr = lambda X: np.transpose(X, (0, 2, 1))  # noqa: E731
    A1 = np.concatenate([
        np.concatenate([M, Z, Z, -tr(Cx)], axis=2),
        np.concatenate([Z, M, Z, -tr(Cy)], axis=2),
        np.concatenate([Z, Z, M, -tr(Cz)], axis=2),
        np.concatenate([Cx, Cy, Cz, blk["M_c"] + blk["tPP"]], axis=2),
    ], axis=1)
    nx, ny, nz = blk["nDP"]
    A2 = np.concatenate([tr(nx), tr(ny), tr(nz), -tr(blk["tDP"])], axis=1)
    Af = np.concatenate([np.zeros((ne, 3 * n)), blk["f"]], axis=1)
    A3 = np.concatenate([nx, ny, nz, blk["tDP"]], axis=2)
    return A1, A2, Af, A3


def local_solvers(blk):
    """C^K = A_3 A_1^-1 A_2 + tauDD (eq. 5.5), C_f^K = A_3 A_1^-1 A_f (eq. 5.6).

    Also returns the pieces of eq. 5.3: X2 = A_1^-1 A_2 and xf = A_1^-1 A_f, so that
    [q_K; u_K] = -X2 u_dK + xf.
    """
    A1, A2, Af, A3 = local_matrices(blk)
    rhs = np.concatenate([A2, Af[:, :, None]], axis=2)
    X = np.linalg.solve(A1, rhs)  # LU with partial pivoting, per element
    X2, xf = X[:, :, :-1], X[:, :, -1]
    CK = A3 @ X2 + blk["tDD"]
    Cf = np.einsum("eij,ej->ei", A3, xf)
    return CK, Cf, X2, xf


def dofs(mesh, d2):
    """dof(K) of Section 6: face blocks of R_k(dK) in T.facebyele order, [Nelt, 4 d2]."""
    return (mesh.facebyele[:, :, None] * d2 + np.arange(d2)[None, None, :]).reshape(mesh.nelt, -1)


def assemble(mesh, d2, CK, Cf):
    """Sparse H (sparse builder) and F (accumarray) of Section 6, eq. 6.5."""
    dof = dofs(mesh, d2)
    m = dof.shape[1]
    rows = np.repeat(dof[:, :, None], m, axis=2)
    cols = np.repeat(dof[:, None, :], m, axis=1)
    ndof = d2 * mesh.nfc
    H = sps.coo_matrix((CK.ravel(), (rows.ravel(), cols.ravel())), shape=(ndof, ndof)).tocsr()
    F = np.zeros(ndof)
    np.add.at(F, dof.ravel(), Cf.ravel())
    return H, F


def dirichlet_data(tab, uD_vals):
    """eq. 6.3: u_hat_D = ((varpi . D)^T D)^-1 (varpi . D)^T u_D(X^dir, ...), [Ndir, d2].

    uD_vals: u_D at the face nodes of the Dirichlet faces, [Ndir, Nf]."""
    WD = tab.varpi[:, None] * tab.D
    return np.linalg.solve(WD.T @ tab.D, WD.T @ np.asarray(uD_vals).T).T


def neumann_data(mesh, tab, gN_vals):
    """eq. 6.4: Phi_N = sum_* n_* . ((varpi . D)^T g_*(X^neu, ...)), [Nneu, d2].

    gN_vals: (g_x, g_y, g_z) at the face nodes of the Neumann faces, each [Nneu, Nf].
    n_e is the outward normal of the element that owns the face (|n_e| = |e|)."""
    nrm = np.zeros((mesh.nfc, 3))
    np.add.at(nrm, mesh.facebyele.ravel(), mesh.normals.reshape(-1, 3))  # one owner per boundary face
    ne = nrm[mesh.neufaces]
    WD = tab.varpi[:, None] * tab.D
    return sum(ne[:, s, None] * (np.asarray(gN_vals[s]) @ WD) for s in range(3))


def solve_trace(mesh, d2, H, F, uhatD, PhiN=None):
    """eq. 6.5 with Dirichlet elimination (Section 6); sparse direct solve.  Returns u_hat [Nfc, d2]."""
    ndof = d2 * mesh.nfc
    b = F.copy()
    if PhiN is not None and len(mesh.neufaces):
        G = np.zeros(ndof)
        G[(mesh.neufaces[:, None] * d2 + np.arange(d2)).ravel()] = np.asarray(PhiN).ravel()
        b += G
    ddof = (mesh.dirfaces[:, None] * d2 + np.arange(d2)).ravel()
    free = np.setdiff1d(np.arange(ndof), ddof)
    x = np.zeros(ndof)
    x[ddof] = np.asarray(uhatD).ravel()
    rhs = b[free] - H[free][:, ddof] @ x[ddof]
    x[free] = spla.spsolve(H[free][:, free].tocsc(), rhs)
    return x.reshape(mesh.nfc, d2), H, b, free


def recover(mesh, X2, xf, uhat, elems=None):
    """eq. 5.3: [q_K; u_K] = -A_1^-1 A_2 u_dK + A_1^-1 A_f.  Returns q [Nelt,3,n], u [Nelt,n]."""
    idx = np.arange(mesh.nelt) if elems is None else np.asarray(elems)
    ud = uhat[mesh.facebyele[idx]].reshape(len(idx), -1)
    sol = -np.einsum("eij,ej->ei", X2, ud) + xf
    n = sol.shape[1] // 4
    return sol[:, :3 * n].reshape(-1, 3, n), sol[:, 3 * n:]


def postprocess(mesh, k, kappa_q, q, u, elems=None, rule="conical"):
    """eq. 9.11: u* in P_{k+1}(K) with (grad u*, grad w)_K = -(kappa^-1 q_h, grad w)_K and
    (u*, 1)_K = (u_h, 1)_K, on the degree-k volume rule `rule` (the one kappa_q is given on);
    bordered (Lagrange) system per element.  Returns u* coefficients in the degree-(k+1)
    basis, [Nelt, d3(k+1)]."""
    idx = np.arange(mesh.nelt) if elems is None else np.asarray(elems)
    p, w, _ = volume_rule(k, rule)
    P = basis.dubiner3(k, p)
    P1 = basis.dubiner3(k + 1, p)
    G1 = basis.dubiner3_grad(k + 1, p)  # [3, Nq, n']
    Binv_T = np.linalg.inv(mesh.B[idx]).transpose(0, 2, 1)
    vol = mesh.volume[idx]
    grad = np.einsum("eab,bqi->eaqi", Binv_T, G1)  # physical gradients [e,3,Nq,n']
    Kst = vol[:, None, None] * np.einsum("q,eaqi,eaqj->eij", w, grad, grad)
    qh = np.einsum("qi,eai->eaq", P, q)  # q_h at nodes [e,3,Nq]
    rhs = -vol[:, None] * np.einsum("q,eq,eaq,eaqi->ei", w, 1.0 / kappa_q[idx], qh, grad)
    ones = vol[:, None] * (w @ P1)[None, :]  # (P'_i, 1)_K
    mean_u = vol * ((u @ P.T) @ w)  # (u_h, 1)_K
    n1 = P1.shape[1]
    A = np.zeros((len(idx), n1 + 1, n1 + 1))
    A[:, :n1, :n1] = Kst
    A[:, :n1, n1] = ones
    A[:, n1, :n1] = ones
    r = np.concatenate([rhs, mean_u[:, None]], axis=1)
    return np.linalg.solve(A, r[:, :, None])[:, :n1, 0]


def errors(mesh, k, q, u, uhat, ustar, prob):
    """Relative errors of eq. 10.1 and e^* of eq. 10.2 against the exact (q, u) of `prob`.
    Integrals use the volume/face rules of degree k+2 (exact to degree 2k+7)."""
    kk = k + 2
    p, w, lam = quadrature.volume_rule(kk)
    v = mesh.coordinates[mesh.elements]
    X, Y, Z = (v[:, :, d] @ lam.T for d in range(3))
    vol = mesh.volume
    integ = lambda g: float(np.sum(vol[:, None] * g * w[None, :]))  # noqa: E731
    P = basis.dubiner3(k, p)
    P1 = basis.dubiner3(k + 1, p)
    ue = prob.u(X, Y, Z)
    qe = prob.q(X, Y, Z)
    uh = u @ P.T
    qh = np.einsum("qi,eai->eaq", P, q)
    us = ustar @ P1.T
    e_u = np.sqrt(integ((ue - uh) ** 2) / integ(ue ** 2))
    e_q = np.sqrt(integ(sum((qe[a] - qh[:, a]) ** 2 for a in range(3))) / integ(sum(qe[a] ** 2 for a in range(3))))
    e_s = np.sqrt(integ((ue - us) ** 2) / integ(ue ** 2))
    qf, wf, xi = quadrature.face_rule(kk)
    fv = mesh.coordinates[mesh.faces]
    FX, FY, FZ = (fv[:, :, d] @ xi.T for d in range(3))
    D = basis.dubiner2(k, qf)
    uef = prob.u(FX, FY, FZ)
    uhf = uhat @ D.T
    # ||v||_h^2 = sum_e |e| ||v||_e^2, with ||v||_e^2 = |e| sum_r varpi_r v_r^2
    a2 = mesh.area[:, None] ** 2
    e_uh = np.sqrt(np.sum(a2 * wf * (uef - uhf) ** 2) / np.sum(a2 * wf * uef ** 2))
    return dict(e_q=e_q, e_u=e_u, e_uhat=e_uh, e_star=e_s)


def monolithic_solve(mesh, tab, blk, uhatD, PhiN=None):
    """The square system eq. 1.2 in all unknowns (q_h, u_h, u_hat), assembled densely:
    per element  A_1 [q;u] + A_2 u_dK = A_f  (eq. 1.2a-b, i.e. eq. 5.3 before inversion);
    per non-Dirichlet face  sum_K ( -A_3 [q;u] + tauDD u_dK ) = G_N  (eq. 1.2c, 1.2e via eq. 5.7);
    per Dirichlet face  u_hat = u_hat_D  (eq. 1.2d, 6.3).  For tiny meshes only."""
    A1, A2, Af, A3 = local_matrices(blk)
    ne = mesh.nelt
    n4 = A1.shape[1]
    d2 = tab.d2
    nloc = ne * n4
    ntot = nloc + mesh.nfc * d2
    A = np.zeros((ntot, ntot))
    b = np.zeros(ntot)
    dof = dofs(mesh, d2) + nloc
    for K in range(ne):
        r = slice(K * n4, (K + 1) * n4)
        A[r, r] = A1[K]
        A[r, dof[K]] = A2[K]
        b[r] = Af[K]
        A[np.ix_(dof[K], np.arange(K * n4, (K + 1) * n4))] += -A3[K]
        A[np.ix_(dof[K], dof[K])] += blk["tDD"][K]
    if PhiN is not None:
        for i, e in enumerate(mesh.neufaces):
            b[nloc + e * d2: nloc + (e + 1) * d2] += PhiN[i]
    for i, e in enumerate(mesh.dirfaces):
        rr = slice(nloc + e * d2, nloc + (e + 1) * d2)
        A[rr, :] = 0.0
        A[rr, rr] = np.eye(d2)
        b[rr] = uhatD[i]
    x = np.linalg.solve(A, b)
    loc = x[:nloc].reshape(ne, n4)
    n = n4 // 4
    return loc[:, :3 * n].reshape(ne, 3, n), loc[:, 3 * n:], x[nloc:].reshape(mesh.nfc, d2)


def solve_problem(prob, coords=None, elems=None, dirichlet=None, neumann=None, rule="conical"):
    """The whole pipeline of Section 3 (i)-(8): mesh, tables, blocks, local solvers, assembly,
    boundary data, trace solve, recovery, postprocess, on the volume rule `rule`.  Returns a
    dict of everything."""
    from workloads import boundary_faces, kuhn_cube

    if coords is None:
        coords, elems = kuhn_cube(prob.s, prob.jitter, prob.seed)
        dirichlet, neumann = boundary_faces(coords, elems, prob.classify)
    mesh = ExpandedMesh(coords, elems, dirichlet, neumann)
    tab = Tables(prob.k, rule)
    X, Y, Z = volume_nodes(mesh, tab)
    kap, cq, fq = prob.kappa(X, Y, Z), prob.c(X, Y, Z), prob.f(X, Y, Z)
    blk = local_blocks(mesh, tab, kap, cq, fq, tau=prob.tau)
    CK, Cf, X2, xf = local_solvers(blk)
    H, F = assemble(mesh, tab.d2, CK, Cf)
    FX, FY, FZ = face_nodes(mesh, tab, mesh.dirfaces)
    uhatD = dirichlet_data(tab, prob.uD(FX, FY, FZ))
    PhiN = None
    if len(mesh.neufaces):
        NX, NY, NZ = face_nodes(mesh, tab, mesh.neufaces)
        PhiN = neumann_data(mesh, tab, prob.gN(NX, NY, NZ))
    uhat, H, b, free = solve_trace(mesh, tab.d2, H, F, uhatD, PhiN)
    q, u = recover(mesh, X2, xf, uhat)
    ustar = postprocess(mesh, prob.k, kap, q, u, rule=rule)
    return dict(mesh=mesh, tab=tab, blk=blk, CK=CK, Cf=Cf, X2=X2, xf=xf, H=H, F=F, b=b, free=free,
                uhatD=uhatD, PhiN=PhiN, uhat=uhat, q=q, u=u, ustar=ustar, kappa_q=kap)
