"""The dense quadrature contraction of the volume masses (eq. 3.55) on the tensor cores
(hdg_mass_contraction, tcgen05.mma with BF16 operands and FP32 accumulation), through the C ABI.

Checked three ways: against the CUDA-core FP32 sum of the same BF16-rounded operands (the same
products, only the order of the FP32 additions differs: 1e-5 relative), against the CUDA-core
FP32-operand sum (BF16 operand rounding, 2^-9 per operand: 2e-2 normwise), and that FP32
operands reproduce the FP64 oracle's M_{kappa^-1} to 1e-5.  Every degree, so N tiles of 16,
64, 224 and three tiles of 224 columns and K of 32 to 224 are exercised, and a ragged last
tile of 128 elements."""
import numpy as np
import pytest

from oracle import hdg as ohdg
from oracle.geometry import ExpandedMesh
from workloads import get_problem

from hdg_cases import gpu_setup, make_mesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1305_1489_gb300 import build
    build()


def _nrel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("k,s", [(1, 3), (2, 3), (3, 2), (4, 2)])
def test_tensor_core_mass_contraction(k, s):
    prob = get_problem("cube16_k3").at(k=k)
    prob.jitter, prob.seed = 0.18, 11
    c, e, d, n = make_mesh(prob, s=s)
    M = gpu_setup(prob, c, e, d, n)
    assert M.nelt % 128 != 0  # a ragged last tile
    X, Y, Z = (t.cpu().numpy() for t in M.volume_nodes())
    ginv = torch.from_numpy(1.0 / prob.kappa(X, Y, Z)).cuda()
    tc = M.mass_contraction(ginv, 0).cpu().numpy()
    ref16 = M.mass_contraction(ginv, 1).cpu().numpy()
    ref32 = M.mass_contraction(ginv, 2).cpu().numpy()
    assert _nrel(tc, ref16) < 1e-5
    assert _nrel(tc, ref32) < 2e-2
    # the FP32-operand contraction against the oracle's literal eq. 3.55 masses
    mesh = ExpandedMesh(c, e, d, n)
    tab = ohdg.Tables(k)
    Xo, Yo, Zo = ohdg.volume_nodes(mesh, tab)
    blk = ohdg.local_blocks(mesh, tab, prob.kappa(Xo, Yo, Zo), prob.c(Xo, Yo, Zo), prob.f(Xo, Yo, Zo))
    iu = np.triu_indices(M.n)
    Mk = blk["M_kinv"][:, iu[0], iu[1]]
    assert _nrel(ref32, Mk) < 1e-5
    assert _nrel(tc, Mk) < 2e-2
    # two calls in a row give the same result (tensor memory and barriers are reused)
    tc2 = M.mass_contraction(ginv, 0).cpu().numpy()
    assert np.array_equal(tc, tc2)
    M.close()
