"""Pins of the oracle's expanded mesh (Section 2, eq. 2.0-2.5, 3.8) on CPU."""
import numpy as np
import pytest

from oracle import quadrature
from oracle.geometry import LOCAL_FACES, ExpandedMesh, piola_cofactors
from workloads import boundary_faces, kuhn_cube


def _mesh(s, jitter=0.0, mixed=False):
    c, e = kuhn_cube(s, jitter=jitter, seed=3)
    cls = (lambda ax, v: "D" if ax == 0 else "N") if mixed else (lambda ax, v: "D")
    d, n = boundary_faces(c, e, cls)
    return ExpandedMesh(c, e, d, n)


@pytest.mark.parametrize("s,jit", [(2, 0.0), (3, 0.2)])
def test_volumes_areas_normals(s, jit):
    m = _mesh(s, jit)
    assert abs(m.volume.sum() - 1.0) < 1e-13  # unit cube, also after jitter
    assert m.nelt == 6 * s ** 3 and m.nfc == 12 * s ** 3 + 6 * s ** 2
    assert np.allclose(m.normals.sum(axis=1), 0.0, atol=1e-15)  # closed surface
    assert np.allclose(m.elem_area, m.area[m.facebyele])  # |n_l| = |e_l|
    v = m.coordinates[m.elements]
    cK = v.mean(axis=1)
    for l in range(4):
        cf = v[:, LOCAL_FACES[l]].mean(axis=1)
        assert np.all(np.einsum("ij,ij->i", m.normals[:, l], cf - cK) > 0)  # outward
        w = v[:, LOCAL_FACES[l]]
        nloc = 0.5 * np.cross(w[:, 1] - w[:, 0], w[:, 2] - w[:, 0])
        # Section 2: with the order of eq. 2.1, faces 2 and 4 point outwards, 1 and 3 inwards
        sign = 1.0 if l in (1, 3) else -1.0
        assert np.allclose(nloc, sign * m.normals[:, l])


def test_interior_faces_have_opposite_normals():
    m = _mesh(2, 0.2)
    owners = {}
    for K in range(m.nelt):
        for l in range(4):
            owners.setdefault(m.facebyele[K, l], []).append((K, l))
    for e, lst in owners.items():
        if len(lst) == 2:
            (K1, l1), (K2, l2) = lst
            assert np.allclose(m.normals[K1, l1], -m.normals[K2, l2])
            assert m.facetype[e] == 0
        else:
            assert m.facetype[e] in (1, 2)


def test_perm_matches_parametrisations():
    """eq. 2.3: phi_e o F_perm(K,l) = phi_l^K, at random points of K_hat_2."""
    m = _mesh(2, 0.2, mixed=True)
    rng = np.random.default_rng(0)
    st = rng.dirichlet(np.ones(3), size=7)[:, 1:]
    ref = quadrature.face_points_on_reference_tet(st)  # q_hat^l
    for K in range(m.nelt):
        v = m.coordinates[m.elements[K]]
        B = np.stack([v[1] - v[0], v[2] - v[0], v[3] - v[0]], axis=1)
        for l in range(4):
            lhs_local = ref[l] @ B.T + v[0]  # F_K(q_hat^l) = phi_l^K(s,t), eq. 2.5
            w = m.coordinates[m.faces[m.facebyele[K, l]]]
            st2 = quadrature.F_mu(int(m.perm[K, l]), st)
            rhs = st2[:, :1] * (w[1] - w[0]) + st2[:, 1:] * (w[2] - w[0]) + w[0]
            assert np.allclose(lhs_local, rhs)


def test_piola_cofactors():
    m = _mesh(2, 0.2)
    a = piola_cofactors(m.coordinates, m.elements)
    ref = m.detB[:, None, None] * np.linalg.inv(m.B).transpose(0, 2, 1)
    assert np.allclose(a, ref)
    assert np.allclose(m.detB, 6 * m.volume)


def test_mesh_errors():
    c, e = kuhn_cube(1)
    d, n = boundary_faces(c, e, lambda ax, v: "D")
    with pytest.raises(ValueError):
        ExpandedMesh(c, e, d[:-1], n)  # one boundary face missing
    e2 = e.copy()
    e2[0, [2, 3]] = e2[0, [3, 2]]
    with pytest.raises(ValueError):
        ExpandedMesh(c, e2, d, n)  # negative orientation
