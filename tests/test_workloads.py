"""The synthetic inputs: meshes are valid and the manufactured data satisfy eq. 1.1."""
import numpy as np
import pytest

from workloads import boundary_faces, get_problem, kuhn_cube
from workloads.problems import batch_problems, grf_field, grf_sample


@pytest.mark.parametrize("s,jit", [(4, 0.0), (5, 0.2)])
def test_kuhn_cube(s, jit):
    c, e = kuhn_cube(s, jitter=jit, seed=0)
    v = c[e]
    det = np.einsum("ij,ij->i", np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]), v[:, 3] - v[:, 0])
    assert e.shape == (6 * s ** 3, 4) and np.all(det > 0)
    assert abs(det.sum() / 6 - 1) < 1e-12
    d, n = boundary_faces(c, e, lambda ax, val: "D" if ax == 0 else "N")
    assert len(d) == 4 * s * s and len(n) == 8 * s * s


def _div(F, x, y, z, h=1e-5):
    return sum((F(*(p + h * (i == a) for i, p in enumerate((x, y, z))))[a]
                - F(*(p - h * (i == a) for i, p in enumerate((x, y, z))))[a]) / (2 * h) for a in range(3))


def _grad(u, x, y, z, h=1e-5):
    return tuple((u(*(p + h * (i == a) for i, p in enumerate((x, y, z))))
                  - u(*(p - h * (i == a) for i, p in enumerate((x, y, z))))) / (2 * h) for a in range(3))


@pytest.mark.parametrize("name", ["cube4_k1", "cube16_k3", "cube48_k2_conv"])
def test_manufactured_data(name):
    prob = get_problem(name)
    rng = np.random.default_rng(0)
    x, y, z = rng.uniform(0.05, 0.95, size=(3, 40))
    g = _grad(prob.u, x, y, z)
    q = prob.q(x, y, z)
    kap = prob.kappa(x, y, z)
    for a in range(3):  # eq. 1.1a: kappa^-1 q + grad u = 0
        assert np.allclose(q[a] / kap + g[a], 0, atol=1e-6)
    flux = prob.q
    if prob.beta is not None:  # conservative convection: div(q + beta u) + c u = f
        flux = lambda x, y, z: tuple(qa + ba * prob.u(x, y, z) for qa, ba in zip(prob.q(x, y, z), prob.beta(x, y, z)))  # noqa: E731
    lhs = _div(flux, x, y, z) + prob.c(x, y, z) * prob.u(x, y, z)  # eq. 1.1b
    assert np.allclose(lhs, prob.f(x, y, z), rtol=1e-6, atol=1e-5)
    if prob.gN is not None:  # eq. 1.1d: -q.nu = g_N.nu
        gn = prob.gN(x, y, z)
        for a in range(3):
            assert np.allclose(-q[a], gn[a])


def test_grf_statistics():
    # pointwise variance sigma^2 = 1 over many samples
    x = np.array([0.3, 0.7]); y = np.array([0.5, 0.1]); z = np.array([0.2, 0.9])
    vals = np.array([grf_field(grf_sample(i))(x, y, z) for i in range(400)])
    assert abs(vals.var(axis=0).mean() - 1.0) < 0.2


def test_batch_sampler():
    probs = batch_problems()
    assert len(probs) == 64
    assert all(8 <= p.s <= 24 and 1 <= p.k <= 4 for p in probs)


def test_coarse_interpolation_is_nested_p1():
    """The fine-vertex values of a random coarse P1 field, interpolated linearly on each fine
    element, equal the coarse field (Freudenthal interpolation on the coarse Kuhn simplex)."""
    from workloads import kuhn_coarse_interpolation
    s, sc = 6, 3
    c, e = kuhn_cube(s)
    nodes, w, nc = kuhn_coarse_interpolation(s, sc, interior_only=False)
    rng = np.random.default_rng(0)
    cv = rng.normal(size=nc)
    V = (np.where(nodes >= 0, cv[np.maximum(nodes, 0)], 0.0) * w).sum(axis=1)
    bary = rng.dirichlet(np.ones(4), size=len(e))
    pts = np.einsum("ek,ekd->ed", bary, c[e])
    fine = np.einsum("ek,ek->e", bary, V[e])
    m1 = sc + 1
    loc = pts * sc
    base = np.minimum(np.floor(loc).astype(int), sc - 1)
    x = loc - base
    order = np.argsort(-x, axis=1)
    xs = np.take_along_axis(x, order, axis=1)
    vid = lambda b: b[:, 0] + m1 * (b[:, 1] + m1 * b[:, 2])  # noqa: E731
    v0 = base.copy()
    unit = np.eye(3, dtype=int)
    v1 = v0 + unit[order[:, 0]]
    v2 = v1 + unit[order[:, 1]]
    v3 = v2 + unit[order[:, 2]]
    coarse = ((1 - xs[:, 0]) * cv[vid(v0)] + (xs[:, 0] - xs[:, 1]) * cv[vid(v1)]
              + (xs[:, 1] - xs[:, 2]) * cv[vid(v2)] + xs[:, 2] * cv[vid(v3)])
    assert np.abs(fine - coarse).max() < 1e-12


def test_kuhn_interpolation_any_sizes():
    """Linear interpolation between Kuhn grids of any two sizes reproduces linear fields, has
    weights in [0, 1] summing to one, and for s_fine = 2 s_coarse is the nested midpoint rule."""
    from workloads import kuhn_coarse_interpolation, kuhn_interpolation

    def grid(s):
        i = np.arange(s + 1)
        I, J, L = np.meshgrid(i, i, i, indexing="ij")
        return np.stack([a.transpose(2, 1, 0).ravel() for a in (I, J, L)], 1) / s

    g = lambda p: 1.0 + p @ np.array([0.3, -2.0, 1.1])  # noqa: E731
    for sf, sc in [(9, 5), (7, 4), (13, 7), (6, 3), (5, 5)]:
        nd, w = kuhn_interpolation(sf, sc)
        cf = g(grid(sc))
        val = sum(np.where(nd[:, j] >= 0, w[:, j] * cf[np.maximum(nd[:, j], 0)], 0.0) for j in range(4))
        assert np.abs(val - g(grid(sf))).max() < 1e-13
        assert w.min() >= 0.0 and np.abs(w.sum(axis=1) - 1.0).max() < 1e-13
    n1, w1 = kuhn_interpolation(8, 4)
    n2, w2, _ = kuhn_coarse_interpolation(8, 4, interior_only=False)
    D1, D2 = np.zeros((729, 125)), np.zeros((729, 125))
    for j in range(4):
        ok1, ok2 = n1[:, j] >= 0, n2[:, j] >= 0
        np.add.at(D1, (np.nonzero(ok1)[0], n1[ok1, j]), w1[ok1, j])
        np.add.at(D2, (np.nonzero(ok2)[0], n2[ok2, j]), w2[ok2, j])
    assert np.abs(D1 - D2).max() == 0.0
