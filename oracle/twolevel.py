"""FP64 reference of the two-level preconditioner of the trace system (oracle; test
infrastructure only -- the product path never imports it).

The paper solves eq. 6.5 directly and says nothing about the solver.  The GPU solver
preconditions PCG with an additive two-level method: the block-Jacobi part of Section 6's
matrix plus a coarse correction in the space of continuous piecewise-linear fields,
    M^-1 r = B^-1 r + Pi V(Pi^T r),
where Pi maps P1 nodal values to face unknowns (the field's trace on each face, which lies in
P_k(e) for k >= 1, in the face basis of eq. 6.3), and V is one symmetric V-cycle for the
Galerkin matrix A_0 = Pi^T H Pi over a nested hierarchy A_{l+1} = P_l^T A_l P_l, with one
l1-Jacobi sweep before and after each coarse correction and an exact solve on the coarsest
level.  Everything below is written from those definitions with dense / scipy algebra.
"""

import numpy as np
import scipy.sparse as sps


def prolongation(mesh, tab, vertex_nodes, vertex_weights, n0):
    """Pi as a sparse [nfc * d2, n0] matrix.  Vertex v carries the field value
    sum_j vertex_weights[v, j] c[vertex_nodes[v, j]]; a face's coefficients are the eq. 6.3
    projection of the field's values at its quadrature nodes.  Dirichlet faces get 0."""
    d2 = tab.d2
    WD = tab.varpi[:, None] * tab.D
    Tm = np.linalg.solve(WD.T @ tab.D, WD.T @ tab.Xi)  # [d2, 3]: face nodes from the 3 vertices
    free = np.ones(mesh.nfc, bool)
    free[mesh.dirfaces] = False
    rows, cols, vals = [], [], []
    fidx = np.nonzero(free)[0]
    for i in range(3):
        v = mesh.faces[fidx, i]
        for j in range(vertex_nodes.shape[1]):
            nd = vertex_nodes[v, j]
            w = vertex_weights[v, j]
            ok = (nd >= 0) & (w != 0.0)
            for a in range(d2):
                rows.append(fidx[ok] * d2 + a)
                cols.append(nd[ok])
                vals.append(Tm[a, i] * w[ok])
    rows, cols, vals = (np.concatenate(x) for x in (rows, cols, vals))
    return sps.coo_matrix((vals, (rows, cols)), shape=(mesh.nfc * d2, n0)).tocsr()


def level_interpolations(sizes, nodes, weights, nver):
    """The P_l [sizes[l], sizes[l+1]] from the stacked per-node rows after the mesh vertices."""
    Ps = []
    off = nver
    for l in range(len(sizes) - 1):
        nd, wt = nodes[off:off + sizes[l]], weights[off:off + sizes[l]]
        r = np.repeat(np.arange(sizes[l]), nd.shape[1])
        ok = (nd.ravel() >= 0) & (wt.ravel() != 0.0)
        Ps.append(sps.coo_matrix((wt.ravel()[ok], (r[ok], nd.ravel()[ok])), shape=(sizes[l], sizes[l + 1])).tocsr())
        off += sizes[l]
    return Ps


def galerkin_hierarchy(H, Pi, Ps):
    """A_0 = Pi^T H Pi (H with Dirichlet rows/columns irrelevant: Pi vanishes there),
    A_{l+1} = P_l^T A_l P_l."""
    As = [(Pi.T @ (H @ Pi)).tocsr()]
    for P in Ps:
        As.append((P.T @ As[-1] @ P).tocsr())
    return As


def vcycle(As, Ps, b, level=0):
    """One symmetric V-cycle: l1-Jacobi from zero, coarse correction, l1-Jacobi; exact on the
    coarsest level."""
    A = As[level]
    if level == len(As) - 1:
        return np.linalg.solve(A.toarray(), b)
    d = np.asarray(abs(A).sum(axis=1)).ravel()
    x = b / d
    x = x + Ps[level] @ vcycle(As, Ps, Ps[level].T @ (b - A @ x), level + 1)
    return x + (b - A @ x) / d


def block_jacobi_inverse(H, mesh, d2):
    """Inverses of the free faces' d2 x d2 diagonal blocks of H ([nfc, d2, d2], 0 on Dirichlet faces)."""
    Binv = np.zeros((mesh.nfc, d2, d2))
    Hc = H.tocsr()
    dirf = set(np.asarray(mesh.dirfaces).tolist())
    for e in range(mesh.nfc):
        if e in dirf:
            continue
        idx = e * d2 + np.arange(d2)
        Binv[e] = np.linalg.inv(Hc[idx][:, idx].toarray())
    return Binv


def apply(Binv, Pi, As, Ps, r):
    """M^-1 r = B^-1 r + Pi V(Pi^T r) on the full face vector (Dirichlet entries of r ignored)."""
    d2 = Binv.shape[1]
    z = np.einsum("fab,fb->fa", Binv, r.reshape(-1, d2)).ravel()
    return z + Pi @ vcycle(As, Ps, Pi.T @ r)


def pcg(H, b, prec, free, tol=1e-10, maxit=10000):
    """Textbook PCG on the free entries (zero start); returns (x, iterations)."""
    x = np.zeros_like(b)
    r = np.where(free, b, 0.0)
    z = np.where(free, prec(r), 0.0)
    p = z.copy()
    rz = r @ z
    bn = np.linalg.norm(r)
    for it in range(maxit):
        if np.linalg.norm(r) <= tol * bn:
            return x, it
        q = np.where(free, H @ p, 0.0)
        al = rz / (p @ q)
        x += al * p
        r -= al * q
        z = np.where(free, prec(r), 0.0)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, maxit


def setup(mesh, tab, H, sizes, nodes, weights):
    """Everything apply() needs for one assembled system."""
    nver = mesh.coordinates.shape[0]
    Pi = prolongation(mesh, tab, nodes[:nver], weights[:nver], sizes[0])
    Ps = level_interpolations(sizes, nodes, weights, nver)
    As = galerkin_hierarchy(H, Pi, Ps)
    Binv = block_jacobi_inverse(H, mesh, tab.d2)
    return Binv, Pi, As, Ps


__all__ = ["prolongation", "level_interpolations", "galerkin_hierarchy", "vcycle", "block_jacobi_inverse",
           "apply", "pcg", "setup"]
