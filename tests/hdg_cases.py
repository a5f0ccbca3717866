"""Shared set-up for the GPU tests: one seeded workload run through both the CUDA path
(via the C ABI) and the oracle.  Inputs come from workloads/; nothing flows from the
CUDA path into the oracle."""
import numpy as np

from workloads import boundary_faces, kuhn_cube


def make_mesh(prob, s=None, jitter=None, seed=None):
    s = prob.s if s is None else s
    c, e = kuhn_cube(s, prob.jitter if jitter is None else jitter, prob.seed if seed is None else seed)
    d, n = boundary_faces(c, e, prob.classify)
    return c, e, d, n


def gpu_setup(prob, c, e, d, n, tau=None):
    """Create the GPU mesh, evaluate the PDE data at the library's nodes, set them."""
    import torch
    from paper_1305_1489_gb300 import HDGMesh
    M = HDGMesh(c, e, d, n, prob.k)
    X, Y, Z = (t.cpu().numpy() for t in M.volume_nodes())
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()  # noqa: E731
    kap, cq, fq = dev(prob.kappa(X, Y, Z)), dev(prob.c(X, Y, Z)), dev(prob.f(X, Y, Z))
    tau_t = None if tau is None else dev(tau)
    M.set_coefficients(kap, cq, fq, tau_t)
    FX, FY, FZ = (t.cpu().numpy() for t in M.face_nodes())
    uD = dev(prob.uD(FX, FY, FZ))
    gN = dev(np.stack(prob.gN(FX, FY, FZ))) if prob.gN is not None else None
    M.set_boundary_data(uD, gN)
    return M


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
