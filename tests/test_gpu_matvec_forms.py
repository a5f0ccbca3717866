"""The two forms of the trace operator product in the solve loops (eq. 6.5 element by element):
one face-major pass over the faces' rows of C^K, and the element pass (contiguous C^K blocks
times the gathered x_dK into Y) followed by the per-face sum of the owners' rows of Y.

Both forms compute the same sums in a different order, so the solves agree to the solve
tolerance: FP64 PCG to 1e-14 and BiCGStab to 1e-13 agree to 1e-11 with each other and with the
FP64 oracle; mixed FP32/FP64 solves (refined to 1e-12) to 1e-9; one product y = H x agrees to
1e-13.  The element pass is also run on a
capped grid (HDG_FACE_BLOCKS), where each block loops over several element groups, and the
autotuner is checked to report the form it chose and to keep a form that HDG_MATVEC fixed.
"""
import numpy as np
import pytest

from oracle import convection as cv
from oracle import hdg as ohdg
from workloads import get_problem

from hdg_cases import gpu_setup, make_mesh, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1305_1489_gb300 import build
    build()


def _rd_case(k, s):
    prob = get_problem("cube16_k3").at(k=k)
    prob.jitter, prob.seed = 0.18, 5
    c, e, d, n = make_mesh(prob, s=s)
    return prob, (c, e, d, n)


def _conv_mesh(prob, c, e, d, n):
    from paper_1305_1489_gb300 import HDGMesh
    M = HDGMesh(c, e, d, n, prob.k)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()  # noqa: E731
    X, Y, Z = (t.cpu().numpy() for t in M.volume_nodes())
    EX, EY, EZ = (t.cpu().numpy() for t in M.element_face_nodes())
    tau = np.full((len(e), 4), prob.tau)
    M.set_coefficients(dev(prob.kappa(X, Y, Z)), dev(prob.c(X, Y, Z)), dev(prob.f(X, Y, Z)), dev(tau),
                       beta=dev(np.stack(prob.beta(X, Y, Z))), beta_faces=dev(np.stack(prob.beta(EX, EY, EZ))))
    FX, FY, FZ = (t.cpu().numpy() for t in M.face_nodes())
    M.set_boundary_data(dev(prob.uD(FX, FY, FZ)))
    return M


def _solve(form, conv, k, s, precision, monkeypatch, blocks=None):
    from paper_1305_1489_gb300 import HDG_MIXED_FP32
    monkeypatch.setenv("HDG_MATVEC", form)
    if blocks:
        monkeypatch.setenv("HDG_FACE_BLOCKS", blocks)
    else:
        monkeypatch.delenv("HDG_FACE_BLOCKS", raising=False)
    if conv:
        prob = get_problem("cube48_k2_conv").at(s=s, k=k)
        mesh = make_mesh(prob)
        M = _conv_mesh(prob, *mesh)
    else:
        prob, mesh = _rd_case(k, s)
        M = gpu_setup(prob, *mesh)
    M.set_inner_tolerance(1e-6)
    M.assemble_condense()
    # FP64 BiCGStab (convection) checks its true residual with the face-major product; iterated
    # with the element pass it can stall a little above 1e-14 (the two products round
    # differently), so it is asked for 1e-13
    rtol = 1e-12 if precision == HDG_MIXED_FP32 else (1e-13 if conv else 1e-14)
    uhat, it, rr = M.solve_trace(rtol=rtol, maxit=5000, precision=precision)
    assert rr <= rtol
    return prob, mesh, uhat.cpu().numpy(), it


@pytest.mark.parametrize("conv,k,s", [(False, 1, 4), (False, 2, 3), (False, 3, 2), (False, 4, 1),
                                      (True, 1, 3), (True, 2, 2), (True, 3, 1)])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_element_and_face_forms_agree(conv, k, s, prec, monkeypatch):
    from paper_1305_1489_gb300 import HDG_FP64, HDG_MIXED_FP32
    precision = HDG_FP64 if prec == "fp64" else HDG_MIXED_FP32
    bar = 1e-11 if prec == "fp64" else 1e-9
    prob, mesh, u_face, it_face = _solve("face", conv, k, s, precision, monkeypatch)
    _, _, u_elem, it_elem = _solve("element", conv, k, s, precision, monkeypatch)
    assert rel(u_elem, u_face) < bar
    ref = cv.solve_problem_conv(prob, *mesh) if conv else ohdg.solve_problem(prob, *mesh)
    assert rel(u_elem, ref["uhat"]) < bar
    # a different rounding order moves the iteration count by a few: CG's residual falls
    # monotonically in the energy norm, BiCGStab's is not monotone and near 1e-14 the step at
    # which it first passes the tolerance moves with rounding
    slack = max(8, it_face // 5) if conv else max(3, it_face // 20)
    assert abs(it_elem - it_face) <= slack


@pytest.mark.parametrize("conv,k,s", [(False, 1, 4), (False, 2, 3), (False, 3, 2), (False, 4, 1),
                                      (True, 1, 3), (True, 2, 2), (True, 3, 1)])
def test_trace_apply_forms_agree(conv, k, s, monkeypatch):
    # one product y = H x (hdg_trace_apply follows the FP64 form) on a random x, both forms
    ys = {}
    for form in ("face", "element"):
        monkeypatch.setenv("HDG_MATVEC", form)
        if conv:
            prob = get_problem("cube48_k2_conv").at(s=s, k=k)
            M = _conv_mesh(prob, *make_mesh(prob))
        else:
            prob, mesh = _rd_case(k, s)
            M = gpu_setup(prob, *mesh)
        M.assemble_condense()
        x = torch.from_numpy(np.random.default_rng(3).standard_normal((M.nfc, M.d2))).cuda()
        ys[form] = M.apply(x).cpu().numpy()
        M.close()
    assert rel(ys["element"], ys["face"]) < 1e-13


@pytest.mark.parametrize("conv", [False, True])
def test_element_pass_on_capped_grid(conv, monkeypatch):
    from paper_1305_1489_gb300 import HDG_FP64
    k, s = (2, 3) if conv else (3, 3)
    prob, mesh, u3, _ = _solve("element", conv, k, s, HDG_FP64, monkeypatch, blocks="3")
    nelt = len(mesh[1])
    m = 4 * (k + 1) * (k + 2) // 2
    assert nelt > 3 * (240 // m) * 4  # every block of the capped grid takes several element groups
    ref = cv.solve_problem_conv(prob, *mesh) if conv else ohdg.solve_problem(prob, *mesh)
    assert rel(u3, ref["uhat"]) < 1e-11


def test_autotune_reports_and_keeps_forced_form(monkeypatch):
    from paper_1305_1489_gb300 import HDG_FP64
    prob, mesh = _rd_case(2, 3)
    monkeypatch.delenv("HDG_MATVEC", raising=False)
    M = gpu_setup(prob, *mesh)
    M.assemble_condense()
    t = M.autotune()
    assert t["matvec_em64"] in (0, 1) and t["matvec_em32"] in (0, 1)
    uhat, _, rr = M.solve_trace(rtol=1e-14, maxit=5000, precision=HDG_FP64)
    assert rr <= 1e-14
    for form, flag in (("face", 0), ("element", 1)):
        monkeypatch.setenv("HDG_MATVEC", form)
        M2 = gpu_setup(prob, *mesh)
        M2.assemble_condense()
        t2 = M2.autotune()
        assert t2["matvec_em64"] == flag and t2["matvec_em32"] == flag
        u2, _, rr2 = M2.solve_trace(rtol=1e-14, maxit=5000, precision=HDG_FP64)
        assert rr2 <= 1e-14
        assert rel(u2.cpu().numpy(), uhat.cpu().numpy()) < 1e-11
