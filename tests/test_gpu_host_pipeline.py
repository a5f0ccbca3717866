"""hdg_assemble_condense_host / hdg_recover_host: the assembly from host arrays with the
copies overlapped chunk by chunk (HDG_DF32), and the recovery into host arrays.  The kernels
and inputs are those of the device-input calls, so the condensed blocks, the solution and the
recovered fields must be bitwise equal to them, for any number of chunks (including more
chunks than a block of elements divides evenly), with and without convection, and for the
FP64 assembly (copied first, not pipelined)."""
import numpy as np
import pytest

from workloads import get_problem

from hdg_cases import make_mesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1305_1489_gb300 import build
    build()


def _inputs(prob, M, conv):
    X, Y, Z = (t.cpu().numpy() for t in M.volume_nodes())
    FX, FY, FZ = (t.cpu().numpy() for t in M.face_nodes())
    host = {"kappa": prob.kappa(X, Y, Z), "c": prob.c(X, Y, Z), "f": prob.f(X, Y, Z), "uD": prob.uD(FX, FY, FZ)}
    if conv:
        EX, EY, EZ = (t.cpu().numpy() for t in M.element_face_nodes())
        host["beta"] = np.stack(prob.beta(X, Y, Z))
        host["beta_f"] = np.stack(prob.beta(EX, EY, EZ))
        host["tau"] = np.full((M.nelt, 4), prob.tau)
    elif prob.gN is not None:
        host["gN"] = np.stack(prob.gN(FX, FY, FZ))
    return {k: torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64)).pin_memory() for k, v in host.items()}


def _device_run(M, host, conv, precision):
    dev = {k: v.cuda() for k, v in host.items()}
    M.set_coefficients(dev["kappa"], dev["c"], dev["f"], dev.get("tau"),
                       beta=dev.get("beta"), beta_faces=dev.get("beta_f"))
    M.set_boundary_data(dev["uD"], dev.get("gN"))
    M.assemble_condense(precision)
    return dev


@pytest.mark.parametrize("conv,k,s", [(False, 2, 3), (False, 3, 2), (True, 1, 3), (True, 2, 3)])
@pytest.mark.parametrize("chunks", [1, 3, 7, 16])
def test_host_assembly_and_recovery_bitwise(conv, k, s, chunks):
    from paper_1305_1489_gb300 import HDG_DF32, HDG_MIXED_FP32, HDGMesh
    prob = get_problem("cube48_k2_conv" if conv else "cube16_k3").at(s=s, k=k)
    mesh = make_mesh(prob)
    M = HDGMesh(*mesh, k)
    host = _inputs(prob, M, conv)
    dev = _device_run(M, host, conv, HDG_DF32)  # noqa: F841 (the mesh borrows these buffers)
    C0, Cf0 = (t.cpu().numpy() for t in M.condensed())
    u0h, _, _ = M.solve_trace(rtol=1e-11, maxit=20000, precision=HDG_MIXED_FP32)
    q0, u0 = (t.cpu().numpy() for t in M.recover(u0h))
    M2 = HDGMesh(*mesh, k)
    M2.assemble_condense_host(host, HDG_DF32, chunks=chunks)
    C1, Cf1 = (t.cpu().numpy() for t in M2.condensed())
    assert np.array_equal(C1, C0) and np.array_equal(Cf1, Cf0)
    u1h, _, _ = M2.solve_trace(rtol=1e-11, maxit=20000, precision=HDG_MIXED_FP32)
    assert np.array_equal(u1h.cpu().numpy(), u0h.cpu().numpy())
    q1 = torch.empty((M2.nelt, 3, M2.n), dtype=torch.float64).pin_memory()
    u1 = torch.empty((M2.nelt, M2.n), dtype=torch.float64).pin_memory()
    M2.recover_host(u1h, q1, u1, chunks=chunks)
    assert np.array_equal(q1.numpy(), q0) and np.array_equal(u1.numpy(), u0)
    # a second host assembly into the same buffers (the copies wait for the queued work)
    M2.assemble_condense_host(host, HDG_DF32, chunks=chunks)
    assert np.array_equal(M2.condensed()[0].cpu().numpy(), C0)
    M.close()
    M2.close()


def test_host_assembly_fp64_and_errors():
    from paper_1305_1489_gb300 import HDG_FP64, HDGError, HDGMesh
    prob = get_problem("cube16_k3").at(s=2, k=2)
    mesh = make_mesh(prob)
    M = HDGMesh(*mesh, 2)
    host = _inputs(prob, M, False)
    dev = _device_run(M, host, False, HDG_FP64)  # noqa: F841 (the mesh borrows these buffers)
    C0 = M.condensed()[0].cpu().numpy()
    M2 = HDGMesh(*mesh, 2)
    M2.assemble_condense_host(host, HDG_FP64, chunks=4)
    assert np.array_equal(M2.condensed()[0].cpu().numpy(), C0)
    bad = dict(host)
    bad.pop("kappa")
    with pytest.raises((HDGError, KeyError, ValueError, TypeError)):
        M2.assemble_condense_host(bad, HDG_FP64)
    M.close()
    M2.close()
