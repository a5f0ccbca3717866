"""Absolute pin of the oracle's error functionals (eq. 10.1, 10.2): errors() against closed
forms that do not go through it.

With the exact fields u = 1 and q = (1, 0, 0) (constants: their projections onto P_k are
exact, and the first member of each orthonormal basis is the constant 1), a perturbation
eps * P_j of one coefficient on a set S of elements adds exactly eps^2 |K| per element to
int (u - u_h)^2, because int_K P_j^2 = |K| (orthonormality, Section 3), whatever j is.  On the
faces, a perturbation eps * D_j of u_hat on a face set F adds |e| * eps^2 |e| to the
||.||_h^2 of eq. 10.2.  So, on a jittered unit cube (sum |K| = 1),
    e_u = eps sqrt(sum_S |K|),   e_q = sqrt(eps^2 sum_S |K| + delta^2 sum_S2 |K|),
    e_uhat = eps sqrt(sum_F |e|^2 / sum_all |e|^2),
with |K| and |e| computed here from the vertex coordinates.  A dropped |e| weight, a wrong
component, a transposed basis matrix or a missing square root fails one of these.
"""
import numpy as np

from oracle import hdg as ohdg
from oracle.geometry import ExpandedMesh
from workloads import boundary_faces, kuhn_cube


class _Const:
    """Exact fields u = 1, q = (1, 0, 0) (only u and q are read by errors())."""

    @staticmethod
    def u(x, y, z):
        return np.ones_like(x)

    @staticmethod
    def q(x, y, z):
        return (np.ones_like(x), np.zeros_like(x), np.zeros_like(x))


def _volumes(coords, elems):
    v = coords[elems]
    return np.abs(np.linalg.det(v[:, 1:] - v[:, :1])) / 6.0


def _areas(coords, faces):
    v = coords[faces]
    return 0.5 * np.linalg.norm(np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]), axis=1)


def test_errors_absolute_values_of_known_perturbations():
    k, s = 2, 3
    c, e = kuhn_cube(s, 0.2, 5)
    d, n = boundary_faces(c, e, lambda ax, val: "D")
    mesh = ExpandedMesh(c, e, d, n)
    nelt, nfc = len(e), mesh.nfc
    nb = (k + 1) * (k + 2) * (k + 3) // 6
    nb1 = (k + 2) * (k + 3) * (k + 4) // 6
    d2 = (k + 1) * (k + 2) // 2
    vol = _volumes(c, e)
    area = _areas(c, mesh.faces)
    assert abs(vol.sum() - 1.0) < 1e-13
    rng = np.random.default_rng(0)
    eps, delta = 1e-3, 3e-4
    S = rng.random(nelt) < 0.3
    S2 = rng.random(nelt) < 0.2
    F = rng.random(nfc) < 0.25
    # exact projections plus the perturbations (random basis index per element / face)
    u = np.zeros((nelt, nb))
    u[:, 0] = 1.0
    u[np.nonzero(S)[0], rng.integers(0, nb, S.sum())] += eps
    q = np.zeros((nelt, 3, nb))
    q[:, 0, 0] = 1.0
    q[np.nonzero(S)[0], 0, rng.integers(0, nb, S.sum())] += eps
    q[np.nonzero(S2)[0], 1, rng.integers(0, nb, S2.sum())] += delta
    ustar = np.zeros((nelt, nb1))
    ustar[:, 0] = 1.0
    ustar[np.nonzero(S2)[0], rng.integers(0, nb1, S2.sum())] += delta
    uhat = np.zeros((nfc, d2))
    uhat[:, 0] = 1.0
    uhat[np.nonzero(F)[0], rng.integers(0, d2, F.sum())] += eps
    got = ohdg.errors(mesh, k, q, u, uhat, ustar, _Const())
    want = {"e_u": eps * np.sqrt(vol[S].sum()),
            "e_q": np.sqrt(eps ** 2 * vol[S].sum() + delta ** 2 * vol[S2].sum()),
            "e_star": delta * np.sqrt(vol[S2].sum()),
            "e_uhat": eps * np.sqrt((area[F] ** 2).sum() / (area ** 2).sum())}
    for key, w in want.items():
        assert abs(got[key] - w) <= 1e-10 * w, (key, got[key], w)
