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


def _noalloc(M, rtol, maxit, uhat, x0=None):
    from paper_1305_1489_gb300 import _lib
    it = C.c_int(0)
    rr = C.c_double(0.0)
    code = _lib.load().hdg_solve_trace_noalloc(M._h, rtol, maxit, None if x0 is None else x0.data_ptr(),
                                               uhat.data_ptr(), C.byref(it), C.byref(rr))
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


def test_noalloc_warm_start_from_previous_solution():
    """A previous u_hat (which carries u_hat_D on the Dirichlet faces) as the initial guess of
    both solves: the Dirichlet entries of the guess are ignored, so both reach the same trace
    as a cold solve, the warm start in fewer iterations."""
    prob = get_problem("cube16_k3").at(k=2)  # Dirichlet on x = 0, 1 with u_D != 0
    prob.jitter, prob.seed = 0.15, 4
    c, e, d, n = make_mesh(prob, s=3)
    M = gpu_setup(prob, c, e, d, n)
    M.assemble_condense()
    ref, it_ref, _ = M.solve_trace(rtol=1e-13, maxit=5000)
    rough, _, _ = M.solve_trace(rtol=1e-4, maxit=5000)
    faces, _, _ = M.faces()
    dirf = faces[:, 3] == 1
    assert np.abs(rough.cpu().numpy()[dirf]).max() > 1e-3  # the guess carries u_hat_D
    warm, it_w, rr_w = M.solve_trace(rtol=1e-13, maxit=5000, x0=rough)
    assert rr_w <= 1e-13 and it_w < it_ref
    assert rel(warm.cpu().numpy(), ref.cpu().numpy()) < 1e-11
    for call in range(2):
        uhat = torch.full((M.nfc, M.d2), float("nan"), dtype=torch.float64, device="cuda")
        code, it, rr = _noalloc(M, 1e-13, 5000, uhat, x0=rough)
        torch.cuda.synchronize()
        assert code == 0, call
        assert rr <= 1e-13 and it < it_ref
        assert rel(uhat.cpu().numpy(), ref.cpu().numpy()) < 1e-11, call
    M.close()


def test_noalloc_refuses_convection():
    """The allocation-free solve is the symmetric CG solve; a convection field (non-symmetric
    trace matrix) is refused with HDG_ERR_UNSUPPORTED instead of being run."""
    from paper_1305_1489_gb300 import HDGMesh, _lib
    prob = get_problem("cube48_k2_conv").at(s=2, k=1)
    c, e, d, n = make_mesh(prob)
    M = HDGMesh(c, e, d, n, prob.k)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()  # noqa: E731
    X, Y, Z = (t.cpu().numpy() for t in M.volume_nodes())
    EX, EY, EZ = (t.cpu().numpy() for t in M.element_face_nodes())
    M.set_coefficients(dev(prob.kappa(X, Y, Z)), dev(prob.c(X, Y, Z)), dev(prob.f(X, Y, Z)),
                       dev(np.full((len(e), 4), prob.tau)), beta=dev(np.stack(prob.beta(X, Y, Z))),
                       beta_faces=dev(np.stack(prob.beta(EX, EY, EZ))))
    FX, FY, FZ = (t.cpu().numpy() for t in M.face_nodes())
    M.set_boundary_data(dev(prob.uD(FX, FY, FZ)))
    M.assemble_condense()
    uhat = torch.zeros((M.nfc, M.d2), dtype=torch.float64, device="cuda")
    code, _, _ = _noalloc(M, 1e-10, 10, uhat)
    assert code == 9  # HDG_ERR_UNSUPPORTED
    assert "beta" in _lib.last_error()
    M.close()
