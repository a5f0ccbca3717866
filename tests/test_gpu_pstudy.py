"""The p-study (eq. 10.3, Table 4) on the GPU: the whole pipeline for k = 0..4 on a fixed
mesh, the relative errors of eq. 10.1 from the library's norm kernels, against the oracle's
errors on the same (degree-k) rules, and the ratios of eq. 10.3 close to 1."""
import numpy as np
import pytest
import torch

from hdg_cases import gpu_setup, make_mesh
from oracle import hdg as ohdg
from oracle import projection as oproj
from workloads import get_problem

from test_oracle_pstudy import p_ratios

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def test_p_study_on_gpu():
    gerr, oerr = [], []
    for k in (0, 1, 2, 3, 4):
        prob = get_problem("cube4_k1").at(s=2, k=k)
        c, e, d, n = make_mesh(prob)
        M = gpu_setup(prob, c, e, d, n)
        M.assemble_condense()
        uhat, _, _ = M.solve_trace(rtol=1e-14, maxit=20000)
        q, u = M.recover(uhat)
        X, Y, Z = (t.cpu().numpy() for t in M.volume_nodes())
        FX, FY, FZ = (t.cpu().numpy() for t in M.face_nodes())
        qe = prob.q(X, Y, Z)
        eq = [M.volume_norm2(q[:, a].contiguous(), _dev(qe[a])) for a in range(3)]
        eu = M.volume_norm2(u, _dev(prob.u(X, Y, Z)))
        ef = M.face_norm2(uhat, _dev(prob.u(FX, FY, FZ)))
        gerr.append({"e_q": np.sqrt(sum(x[0] for x in eq) / sum(x[1] for x in eq)),
                     "e_u": np.sqrt(eu[0] / eu[1]), "e_uhat": np.sqrt(ef[0] / ef[1])})
        r = ohdg.solve_problem(prob, c, e, d, n)
        mesh, tab = r["mesh"], r["tab"]
        VX, VY, VZ = ohdg.volume_nodes(mesh, tab)
        OX, OY, OZ = ohdg.face_nodes(mesh, tab)
        qo = prob.q(VX, VY, VZ)
        oq = [oproj.norm2_volume(mesh, k, r["q"][:, a], qo[a], k) for a in range(3)]
        ou = oproj.norm2_volume(mesh, k, r["u"], prob.u(VX, VY, VZ), k)
        of = oproj.norm2_faces(mesh, k, r["uhat"], prob.u(OX, OY, OZ))
        oerr.append({"e_q": np.sqrt(sum(x[0] for x in oq) / sum(x[1] for x in oq)),
                     "e_u": np.sqrt(ou[0] / ou[1]), "e_uhat": np.sqrt(of[0] / of[1])})
    for key in ("e_q", "e_u", "e_uhat"):
        for g, o in zip(gerr, oerr):
            assert abs(g[key] - o[key]) < 1e-8 * o[key]
        for ratio in p_ratios(gerr, key):
            assert 0.7 < ratio < 1.3, (key, ratio)
