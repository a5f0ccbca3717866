"""Hybridised BDM element (Section 9, "BDM") in FP64 (oracle; test infrastructure only).

The local solvers of the HDG oracle with tau = 0 and u_h in P_{k-1}(K): following the paper,
the last d2 rows and columns of A_1 (the degree-k members of the hierarchical u basis), the
last d2 rows of A_2 and A_f and the last d2 columns of A_3 are erased, then eq. 5.3, 5.5 and
5.6 apply unchanged.  Reading: the paper's sentence tests eq. 1.2a in P_{k-1}(K)^3; the
erasures it then lists (u rows and columns only) test eq. 1.2b in P_{k-1}(K) and keep
q_h in P_k(K)^3, which is the BDM pair, so that reading is used.
"""

import numpy as np

from . import hdg


def local_solvers(blk, d2):
    """C^K, C_f^K and the recovery pieces X2, xf of the BDM element (blk built with tau = 0).
    X2 and xf keep 4n rows, the erased u coefficients being zero."""
    A1, A2, Af, A3 = hdg.local_matrices(blk)
    N = A1.shape[1]
    r = N - d2
    rhs = np.concatenate([A2[:, :r, :], Af[:, :r, None]], axis=2)
    X = np.linalg.solve(A1[:, :r, :r], rhs)
    X2r, xfr = X[:, :, :-1], X[:, :, -1]
    CK = A3[:, :, :r] @ X2r + blk["tDD"]
    Cf = np.einsum("eij,ej->ei", A3[:, :, :r], xfr)
    X2 = np.zeros((A1.shape[0], N, A2.shape[2]))
    xf = np.zeros((A1.shape[0], N))
    X2[:, :r] = X2r
    xf[:, :r] = xfr
    return CK, Cf, X2, xf


def solve_problem(prob, coords=None, elems=None, dirichlet=None, neumann=None):
    """The pipeline of hdg.solve_problem with the BDM local solvers (tau = 0)."""
    from workloads import boundary_faces, kuhn_cube

    if coords is None:
        coords, elems = kuhn_cube(prob.s, prob.jitter, prob.seed)
        dirichlet, neumann = boundary_faces(coords, elems, prob.classify)
    mesh = hdg.ExpandedMesh(coords, elems, dirichlet, neumann)
    tab = hdg.Tables(prob.k)
    X, Y, Z = hdg.volume_nodes(mesh, tab)
    kap, cq, fq = prob.kappa(X, Y, Z), prob.c(X, Y, Z), prob.f(X, Y, Z)
    blk = hdg.local_blocks(mesh, tab, kap, cq, fq, tau=0.0)
    CK, Cf, X2, xf = local_solvers(blk, tab.d2)
    H, F = hdg.assemble(mesh, tab.d2, CK, Cf)
    FX, FY, FZ = hdg.face_nodes(mesh, tab, mesh.dirfaces)
    uhatD = hdg.dirichlet_data(tab, prob.uD(FX, FY, FZ))
    PhiN = None
    if len(mesh.neufaces):
        NX, NY, NZ = hdg.face_nodes(mesh, tab, mesh.neufaces)
        PhiN = hdg.neumann_data(mesh, tab, prob.gN(NX, NY, NZ))
    uhat, H, b, free = hdg.solve_trace(mesh, tab.d2, H, F, uhatD, PhiN)
    q, u = hdg.recover(mesh, X2, xf, uhat)
    ustar = hdg.postprocess(mesh, prob.k, kap, q, u)
    return dict(mesh=mesh, tab=tab, blk=blk, CK=CK, Cf=Cf, X2=X2, xf=xf, H=H, F=F, b=b, free=free,
                uhatD=uhatD, PhiN=PhiN, uhat=uhat, q=q, u=u, ustar=ustar, kappa_q=kap)
