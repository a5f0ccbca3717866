"""Pins of the oracle's HDG projection (eq. 9.13), face projection (eq. 9.12) and the
superconvergence diagnostics (eq. 10.2) against what the mathematics fixes.

* eq. 9.13 has a unique solution, so data already in P_k(K)^3 x P_k(K) is reproduced exactly,
  on a jittered mesh with a different tau on every face of every element (a wrong normal
  sign, face permutation or tau factor breaks it: the top-degree coefficients come from the
  face rows only);
* data of degree k + 1 is not reproduced (the reproduction pin is not vacuous), and the
  projection is linear;
* eq. 9.12 reproduces P_k face data;
* the superconvergence the paper reports (Tables 1-3, theory of Cockburn, Gopalakrishnan and
  Sayas 2010): eps^u = ||Pi u - u_h|| / ||u|| and eps^uhat decay like h^(k+2) while e^u decays
  like h^(k+1); a planted sign error in the face rows of eq. 9.13 destroys the h^(k+2) rate.
"""
import numpy as np
import pytest

from oracle import basis, hdg, projection
from oracle.geometry import ExpandedMesh
from workloads import boundary_faces, get_problem, kuhn_cube


def _mesh(s, jitter=0.15, seed=5):
    c, e = kuhn_cube(s, jitter=jitter, seed=seed)
    d, n = boundary_faces(c, e, lambda ax, v: "D")
    return ExpandedMesh(c, e, d, n)


def _poly(k, rng):
    """A random polynomial of total degree k in (x, y, z) as a callable."""
    terms = [(a, b, c) for a in range(k + 1) for b in range(k + 1 - a) for c in range(k + 1 - a - b)]
    coef = rng.standard_normal(len(terms))
    return lambda x, y, z: sum(cf * x ** a * y ** b * z ** c for cf, (a, b, c) in zip(coef, terms))


def _inputs(mesh, tab, qf, uf):
    X, Y, Z = hdg.volume_nodes(mesh, tab)
    pts = projection.element_face_points(mesh, tab)
    FX, FY, FZ = pts[..., 0], pts[..., 1], pts[..., 2]
    q_vol = np.stack([f(X, Y, Z) for f in qf])
    q_face = np.stack([f(FX, FY, FZ) for f in qf])
    return q_vol, uf(X, Y, Z), q_face, uf(FX, FY, FZ)


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_projection_reproduces_polynomials_of_degree_k(k):
    rng = np.random.default_rng(10 + k)
    mesh = _mesh(2)
    tab = hdg.Tables(k)
    qf = [_poly(k, rng) for _ in range(3)]
    uf = _poly(k, rng)
    tau = rng.uniform(0.5, 3.0, size=(mesh.nelt, 4))
    q_vol, u_vol, q_face, u_face = _inputs(mesh, tab, qf, uf)
    Pq, Pu = projection.hdg_projection(mesh, tab, q_vol, u_vol, q_face, u_face, tau=tau)
    scale = np.abs(u_vol).max()
    assert np.abs(Pu @ tab.P.T - u_vol).max() < 1e-11 * scale
    for c in range(3):
        assert np.abs(Pq[:, c] @ tab.P.T - q_vol[c]).max() < 1e-11 * np.abs(q_vol[c]).max()


@pytest.mark.parametrize("k", [1, 2])
def test_projection_of_degree_k_plus_1_data_differs_and_is_linear(k):
    rng = np.random.default_rng(20 + k)
    mesh = _mesh(2)
    tab = hdg.Tables(k)
    qf1 = [_poly(k + 1, rng) for _ in range(3)]
    uf1 = _poly(k + 1, rng)
    qf2 = [_poly(k + 1, rng) for _ in range(3)]
    uf2 = _poly(k + 1, rng)
    a1 = _inputs(mesh, tab, qf1, uf1)
    a2 = _inputs(mesh, tab, qf2, uf2)
    P1 = projection.hdg_projection(mesh, tab, *a1)
    P2 = projection.hdg_projection(mesh, tab, *a2)
    assert np.abs(P1[1] @ tab.P.T - a1[1]).max() > 1e-4 * np.abs(a1[1]).max()
    Pc = projection.hdg_projection(mesh, tab, *(2.0 * x - 3.0 * y for x, y in zip(a1, a2)))
    for i in range(2):
        lin = 2.0 * P1[i] - 3.0 * P2[i]
        assert np.abs(Pc[i] - lin).max() < 1e-11 * np.abs(lin).max()


@pytest.mark.parametrize("k", [1, 2, 3])
def test_face_projection_reproduces_polynomials(k):
    rng = np.random.default_rng(30 + k)
    mesh = _mesh(2)
    tab = hdg.Tables(k)
    uf = _poly(k, rng)
    FX, FY, FZ = hdg.face_nodes(mesh, tab)
    vals = uf(FX, FY, FZ)
    Pu = projection.face_projection(tab, vals)
    assert np.abs(Pu @ tab.D.T - vals).max() < 1e-11 * np.abs(vals).max()


def _eps(prob, s, plant=False, monkeypatch=None):
    r = hdg.solve_problem(prob.at(s=s))
    mesh, tab = r["mesh"], r["tab"]
    if plant:
        orig = hdg.local_blocks

        def flipped(*a, **kw):
            b = orig(*a, **kw)
            b = dict(b)
            b["nDP"] = tuple(-x for x in b["nDP"])  # q.nu with the wrong sign in eq. 9.13
            return b

        monkeypatch.setattr(projection, "local_blocks", flipped)
    q_vol, u_vol, q_face, u_face = _inputs(mesh, tab, [lambda x, y, z, c=c: prob.q(x, y, z)[c] for c in range(3)],
                                           prob.u)
    Pq, Pu = projection.hdg_projection(mesh, tab, q_vol, u_vol, q_face, u_face, tau=prob.tau)
    FX, FY, FZ = hdg.face_nodes(mesh, tab)
    uf = prob.u(FX, FY, FZ)
    Pf = projection.face_projection(tab, uf)
    sc = projection.superconvergence(mesh, prob.k, Pu, r["u"], Pf, r["uhat"], u_vol, uf)
    e_u, ref = projection.norm2_volume(mesh, prob.k, r["u"], u_vol, prob.k)
    sc["e_u"] = float(np.sqrt(e_u / ref))
    return sc


@pytest.mark.parametrize("k", [1, 2])
def test_superconvergence_orders(k):
    prob = get_problem("cube4_k1").at(k=k)
    e4, e8 = _eps(prob, 4), _eps(prob, 8)
    rate = {a: np.log2(e4[a] / e8[a]) for a in e4}
    assert abs(rate["e_u"] - (k + 1)) < 0.3, rate
    assert rate["eps_u"] > k + 2 - 0.35, rate
    assert rate["eps_uhat"] > k + 2 - 0.35, rate


def test_planted_normal_sign_destroys_superconvergence(monkeypatch):
    prob = get_problem("cube4_k1")
    e4 = _eps(prob, 4, plant=True, monkeypatch=monkeypatch)
    e8 = _eps(prob, 8, plant=True, monkeypatch=monkeypatch)
    assert np.log2(e4["eps_u"] / e8["eps_u"]) < 2.5
