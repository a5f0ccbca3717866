"""Batched solve of independent problems of mixed degree (one CUDA graph launch) against
the oracle solving each problem on its own."""
import numpy as np
import pytest

from oracle import hdg as ohdg
from workloads import get_problem
from workloads.problems import sinsinsin

from hdg_cases import make_mesh, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1305_1489_gb300 import build
    build()


def _problems():
    probs = [sinsinsin("b0", 2, 1, kappa0=0.3, c0=2.0), sinsinsin("b1", 3, 2, kappa0=4.0, c0=0.0),
             sinsinsin("b2", 2, 1, kappa0=1.5, c0=0.5), get_problem("cube16_k3").at(s=2, k=2),
             sinsinsin("b4", 1, 3, kappa0=0.7, c0=1.0), sinsinsin("b5", 2, 3, kappa0=9.0, c0=3.0)]
    probs[3].jitter, probs[3].seed = 0.1, 5
    return probs


@pytest.mark.parametrize("prec", ["fp64", "df32"])
def test_batch_matches_individual_solves(prec):
    from paper_1305_1489_gb300 import HDG_DF32, HDG_FP64, HDGBatch
    probs = _problems()
    meshes = [make_mesh(p) for p in probs]
    B = HDGBatch([(c, e, d, n, p.k) for (c, e, d, n), p in zip(meshes, probs)])
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()  # noqa: E731
    for G in B.groups:
        M = G["mesh"]
        X, Y, Z = (t.cpu().numpy() for t in M.volume_nodes())
        FX, FY, FZ = (t.cpu().numpy() for t in M.face_nodes())
        kap, cq, fq = (np.zeros_like(X) for _ in range(3))
        uD = np.zeros_like(FX)
        gN = np.zeros((3,) + FX.shape)
        for i, p in enumerate(G["probs"]):
            pr = probs[p]
            es = slice(G["elem_off"][i], G["elem_off"][i + 1])
            fs = slice(G["face_off"][i], G["face_off"][i + 1])
            kap[es], cq[es], fq[es] = pr.kappa(X[es], Y[es], Z[es]), pr.c(X[es], Y[es], Z[es]), pr.f(X[es], Y[es], Z[es])
            uD[fs] = pr.uD(FX[fs], FY[fs], FZ[fs])
            if pr.gN is not None:
                gN[:, fs] = np.stack(pr.gN(FX[fs], FY[fs], FZ[fs]))
        M.set_coefficients(dev(kap), dev(cq), dev(fq))
        M.set_boundary_data(dev(uD), dev(gN))
    relres, iters = B.run(precision=HDG_DF32 if prec == "df32" else HDG_FP64, rtol=1e-12, maxit=5000)
    assert np.all(relres <= 1e-12)
    for g, G in enumerate(B.groups):
        uhat, q, u = (t.cpu().numpy() for t in B.solution(g))
        for i, p in enumerate(G["probs"]):
            c, e, d, n = meshes[p]
            ref = ohdg.solve_problem(probs[p], c, e, d, n)
            es = slice(G["elem_off"][i], G["elem_off"][i + 1])
            fs = slice(G["face_off"][i], G["face_off"][i + 1])
            assert rel(uhat[fs], ref["uhat"]) < 1e-9, (p, rel(uhat[fs], ref["uhat"]))
            assert rel(u[es], ref["u"]) < 1e-9
            assert rel(q[es], ref["q"]) < 1e-9
    # a second launch of the same graph gives the same answer
    relres2, _ = B.run(precision=HDG_DF32 if prec == "df32" else HDG_FP64, rtol=1e-12, maxit=5000)
    assert np.allclose(relres, relres2, rtol=0, atol=1e-15)
    B.close()


def test_batch_two_level_matches_individual_solves():
    """The batch with a two-level preconditioner per group (block-diagonal union of each
    problem's P1 hierarchy, shallow problems padded) reaches the same solutions in fewer
    iterations than block-Jacobi."""
    from paper_1305_1489_gb300 import HDG_FP64, HDGBatch
    from workloads import kuhn_p1_hierarchy
    probs = _problems() + [sinsinsin("b6", 8, 2, kappa0=2.0, c0=1.0), sinsinsin("b7", 7, 2, kappa0=0.5, c0=0.0)]
    meshes = [make_mesh(p) for p in probs]
    B = HDGBatch([(c, e, d, n, p.k) for (c, e, d, n), p in zip(meshes, probs)])
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()  # noqa: E731
    for G in B.groups:
        M = G["mesh"]
        X, Y, Z = (t.cpu().numpy() for t in M.volume_nodes())
        FX, FY, FZ = (t.cpu().numpy() for t in M.face_nodes())
        kap, cq, fq = (np.zeros_like(X) for _ in range(3))
        uD = np.zeros_like(FX)
        gN = np.zeros((3,) + FX.shape)
        for i, p in enumerate(G["probs"]):
            pr = probs[p]
            es = slice(G["elem_off"][i], G["elem_off"][i + 1])
            fs = slice(G["face_off"][i], G["face_off"][i + 1])
            kap[es], cq[es], fq[es] = pr.kappa(X[es], Y[es], Z[es]), pr.c(X[es], Y[es], Z[es]), pr.f(X[es], Y[es], Z[es])
            uD[fs] = pr.uD(FX[fs], FY[fs], FZ[fs])
            if pr.gN is not None:
                gN[:, fs] = np.stack(pr.gN(FX[fs], FY[fs], FZ[fs]))
        M.set_coefficients(dev(kap), dev(cq), dev(fq))
        M.set_boundary_data(dev(uD), dev(gN))
    relres_bj, it_bj = B.run(precision=HDG_FP64, rtol=1e-11, maxit=20000)
    B.set_coarse_spaces([kuhn_p1_hierarchy(p.s, p.dirichlet_planes, max_coarsest=1, strict=False) for p in probs])
    relres, it_tl = B.run(precision=HDG_FP64, rtol=1e-11, maxit=20000)
    assert np.all(relres <= 1e-11)
    assert np.all(it_tl <= it_bj) and it_tl.sum() < it_bj.sum()
    for g, G in enumerate(B.groups):
        uhat, q, u = (t.cpu().numpy() for t in B.solution(g))
        for i, p in enumerate(G["probs"]):
            pr = probs[p]
            c, e, d, n = meshes[p]
            ref = ohdg.solve_problem(pr, c, e, d, n)
            fs = slice(G["face_off"][i], G["face_off"][i + 1])
            es = slice(G["elem_off"][i], G["elem_off"][i + 1])
            assert rel(uhat[fs], ref["uhat"]) < 1e-9, (p, rel(uhat[fs], ref["uhat"]))
            assert rel(u[es], ref["u"]) < 1e-9
    # removing the coarse spaces restores the block-Jacobi iteration counts
    B.set_coarse_spaces(None)
    _, it_again = B.run(precision=HDG_FP64, rtol=1e-11, maxit=20000)
    assert np.all(it_again == it_bj)
    B.close()


@pytest.mark.parametrize("coarse", [False, True])
def test_batch_mixed_precision_matches_individual_solves(coarse):
    """FP32 inner / FP64 outer refinement inside the batch graph (nested device-driven loops),
    with block-Jacobi or two-level preconditioning: every problem reaches rtol and the oracle's
    solution."""
    from paper_1305_1489_gb300 import HDG_DF32, HDG_MIXED_FP32, HDGBatch
    from workloads import kuhn_p1_hierarchy
    probs = _problems() + [sinsinsin("b6", 6, 2, kappa0=2.0, c0=1.0)]
    meshes = [make_mesh(p) for p in probs]
    B = HDGBatch([(c, e, d, n, p.k) for (c, e, d, n), p in zip(meshes, probs)])
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()  # noqa: E731
    for G in B.groups:
        M = G["mesh"]
        X, Y, Z = (t.cpu().numpy() for t in M.volume_nodes())
        FX, FY, FZ = (t.cpu().numpy() for t in M.face_nodes())
        kap, cq, fq = (np.zeros_like(X) for _ in range(3))
        uD = np.zeros_like(FX)
        gN = np.zeros((3,) + FX.shape)
        for i, p in enumerate(G["probs"]):
            pr = probs[p]
            es = slice(G["elem_off"][i], G["elem_off"][i + 1])
            fs = slice(G["face_off"][i], G["face_off"][i + 1])
            kap[es], cq[es], fq[es] = pr.kappa(X[es], Y[es], Z[es]), pr.c(X[es], Y[es], Z[es]), pr.f(X[es], Y[es], Z[es])
            uD[fs] = pr.uD(FX[fs], FY[fs], FZ[fs])
            if pr.gN is not None:
                gN[:, fs] = np.stack(pr.gN(FX[fs], FY[fs], FZ[fs]))
        M.set_coefficients(dev(kap), dev(cq), dev(fq))
        M.set_boundary_data(dev(uD), dev(gN))
    if coarse:
        B.set_coarse_spaces([kuhn_p1_hierarchy(p.s, p.dirichlet_planes, max_coarsest=1, strict=False) for p in probs])
    B.set_inner_tolerance(1e-6)
    B.set_solve_precision(HDG_MIXED_FP32)
    relres, iters = B.run(precision=HDG_DF32, rtol=1e-11, maxit=20000)
    assert np.all(relres <= 1e-11) and np.all(iters > 0)
    for g, G in enumerate(B.groups):
        uhat, q, u = (t.cpu().numpy() for t in B.solution(g))
        for i, p in enumerate(G["probs"]):
            c, e, d, n = meshes[p]
            ref = ohdg.solve_problem(probs[p], c, e, d, n)
            fs = slice(G["face_off"][i], G["face_off"][i + 1])
            es = slice(G["elem_off"][i], G["elem_off"][i + 1])
            assert rel(uhat[fs], ref["uhat"]) < 1e-9, (p, rel(uhat[fs], ref["uhat"]))
            assert rel(u[es], ref["u"]) < 1e-9
    # a second launch reaches the same result
    relres2, iters2 = B.run(precision=HDG_DF32, rtol=1e-11, maxit=20000)
    assert np.array_equal(iters, iters2) and np.allclose(relres, relres2, rtol=0, atol=1e-15)
    B.close()
