"""hdg_solve_trace_noalloc: the trace solve for callers that cannot allocate device memory
when they solve (a fixed, pre-reserved memory budget, or a pool that forbids allocations
after warm-up).  Its scratch lives in a static device array inside libhdg.

Checked through the C ABI against the allocating hdg_solve_trace on the same mesh, on two
calls in a row (the second call finds the first call's leftovers in the shared array), and
the size limit is refused with HDG_ERR_ARG.  Collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

from workloads import get_problem

from hdg_cases import gpu_setup, make_mesh, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1305_1489_gb300 import build
    build()


def _noalloc(M, rtol, maxit, uhat):
    from paper_1305_1489_gb300 import _lib
    it = C.c_int(0)
    rr = C.c_double(0.0)
    code = _lib.load().hdg_solve_trace_noalloc(M._h, rtol, maxit, None, uhat.data_ptr(), C.byref(it), C.byref(rr))
    return code, it.value, rr.value


@pytest.mark.parametrize("k,s", [(2, 3), (3, 2)])
def test_noalloc_matches_allocating_solve(k, s):
    prob = get_problem("cube16_k3").at(k=k)  # Dirichlet on x = 0, 1 and Neumann elsewhere
    prob.jitter, prob.seed = 0.15, 4
    c, e, d, n = make_mesh(prob, s=s)
    M = gpu_setup(prob, c, e, d, n)
    M.assemble_condense()
    assert M.nfc * M.d2 <= 65536
    ref, it_ref, rr_ref = M.solve_trace(rtol=1e-13, maxit=5000)
    for call in range(2):
        uhat = torch.full((M.nfc, M.d2), float("nan"), dtype=torch.float64, device="cuda")
        code, it, rr = _noalloc(M, 1e-13, 5000, uhat)
        torch.cuda.synchronize()
        assert code == 0, call
        assert rr <= 1e-13
        assert rel(uhat.cpu().numpy(), ref.cpu().numpy()) < 1e-11, call
    M.close()


def test_noalloc_rejects_large_mesh():
    prob = get_problem("cube4_k1").at(s=8, k=4)  # 6528 faces x 15 = 97,920 trace unknowns
    c, e, d, n = make_mesh(prob)
    M = gpu_setup(prob, c, e, d, n)
    M.assemble_condense()
    uhat = torch.zeros((M.nfc, M.d2), dtype=torch.float64, device="cuda")
    code, _, _ = _noalloc(M, 1e-10, 10, uhat)
    assert code == 1  # HDG_ERR_ARG
    from paper_1305_1489_gb300 import _lib
    assert "65536" in _lib.last_error()
    M.close()
