"""Expanded tetrahedral data structure (oracle; test infrastructure).

Section 2 of the paper: the affine map F_K (eq. 2.0), face parametrisations phi_e, the local
face order of eq. 2.1, the maps F_mu of eq. 2.2, the permutation matrix perm(K,l) of eq. 2.3,
and the expanded fields T.faces, T.facebyele, T.perm, T.volume, T.area, T.normals.

Readings:
  * global face parametrisation (the paper: "its order will give the intrinsic
    parametrization"): the face's three global vertex numbers sorted ascending;
  * global face numbering: faces sorted lexicographically by that sorted triple (0-based);
  * the Neumann normal n_e of eq. 6.4 is the adjacent element's outward normal.
Indices are 0-based here; perm values keep the paper's 1..6.
"""

import numpy as np

# eq. 2.1: local faces of K as positions in (v1, v2, v3, v4)
LOCAL_FACES = np.array([(0, 1, 2), (0, 1, 3), (0, 2, 3), (3, 1, 2)])

# eq. 2.2, right-hand table: indices of the images of (w1, w2, w3) under F_mu, mu = 1..6
F_MU_TABLE = {1: (1, 2, 3), 2: (1, 3, 2), 3: (3, 1, 2), 4: (3, 2, 1), 5: (2, 3, 1), 6: (2, 1, 3)}


class ExpandedMesh:
    """The paper's T in expanded form, built from the basic fields (Section 2)."""

    def __init__(self, coords, elements, dirichlet, neumann):
        self.coordinates = np.asarray(coords, dtype=np.float64)
        self.elements = np.asarray(elements, dtype=np.int64)
        self.dirichlet = np.asarray(dirichlet, dtype=np.int64).reshape(-1, 3)
        self.neumann = np.asarray(neumann, dtype=np.int64).reshape(-1, 3)
        nelt = self.elements.shape[0]

        tri = self.elements[:, LOCAL_FACES]  # [Nelt, 4, 3] local vertex order of eq. 2.1
        key = np.sort(tri, axis=2).reshape(-1, 3)
        faces, inv, counts = np.unique(key, axis=0, return_inverse=True, return_counts=True)
        self.faces = faces  # [Nfc, 3] sorted vertex triples
        self.facebyele = inv.reshape(nelt, 4)
        nfc = faces.shape[0]

        ftype = np.zeros(nfc, dtype=np.int64)
        lookup = {tuple(f): i for i, f in enumerate(faces)}
        for lst, code in ((self.dirichlet, 1), (self.neumann, 2)):
            for t in lst:
                e = lookup.get(tuple(sorted(int(v) for v in t)))
                if e is None:
                    raise ValueError("boundary face is not a face of the mesh")
                ftype[e] = code
        boundary = counts == 1
        if np.any(boundary & (ftype == 0)):
            raise ValueError("a boundary face is neither Dirichlet nor Neumann")
        if np.any(counts > 2):
            raise ValueError("non-conforming mesh: a face shared by more than two elements")
        self.facetype = ftype
        self.dirfaces = np.nonzero(ftype == 1)[0]
        self.neufaces = np.nonzero(ftype == 2)[0]

        # perm(K, l) of eq. 2.3: phi_e o F_mu = phi_l^K.  phi_e(w_hat_i) = faces[e][i] and
        # phi_l^K(w_hat_i) = local vertex i, so F_mu must send w_hat_i to the position of
        # local vertex i inside the sorted triple.
        fv_sorted = faces[self.facebyele]  # [Nelt, 4, 3]
        pos = np.argmax(fv_sorted[:, :, None, :] == tri[:, :, :, None], axis=3) + 1  # [Nelt,4,3]
        code = pos[..., 0] * 16 + pos[..., 1] * 4 + pos[..., 2]
        perm = np.zeros((nelt, 4), dtype=np.int64)
        for m, (i1, i2, i3) in F_MU_TABLE.items():
            perm[code == i1 * 16 + i2 * 4 + i3] = m
        assert np.all(perm > 0)
        self.perm = perm

        v = self.coordinates[self.elements]  # [Nelt, 4, 3]
        self.B = np.stack([v[:, 1] - v[:, 0], v[:, 2] - v[:, 0], v[:, 3] - v[:, 0]], axis=2)  # eq. 2.0
        self.detB = np.linalg.det(self.B)
        if np.any(self.detB <= 0):
            raise ValueError("element with non-positive orientation")
        self.volume = self.detB / 6.0

        # T.normals: outward, |n_l| = |e_l|.  n_e = (1/2)(w2-w1)x(w3-w1) in the local order,
        # then flipped where it points towards the opposite vertex.
        normals = np.zeros((nelt, 4, 3))
        for l in range(4):
            w = v[:, LOCAL_FACES[l]]
            n = 0.5 * np.cross(w[:, 1] - w[:, 0], w[:, 2] - w[:, 0])
            opp = [i for i in range(4) if i not in LOCAL_FACES[l]][0]
            towards = np.einsum("ij,ij->i", n, v[:, opp] - w[:, 0]) > 0
            n[towards] *= -1
            normals[:, l] = n
        self.normals = normals
        self.elem_area = np.linalg.norm(normals, axis=2)  # |e_l^K|
        fv = self.coordinates[faces]
        self.area = 0.5 * np.linalg.norm(np.cross(fv[:, 1] - fv[:, 0], fv[:, 2] - fv[:, 0]), axis=1)

    @property
    def nelt(self):
        return self.elements.shape[0]

    @property
    def nfc(self):
        return self.faces.shape[0]


def piola_cofactors(coords, elements):
    """a_{*#} = (det B_K B_K^{-T})_{*#}, the nine closed forms of eq. 3.8.  Returns [Nelt,3,3]."""
    v = np.asarray(coords)[np.asarray(elements)]
    x1, x2, x3, x4 = (v[:, i, 0] for i in range(4))
    y1, y2, y3, y4 = (v[:, i, 1] for i in range(4))
    z1, z2, z3, z4 = (v[:, i, 2] for i in range(4))
    a = np.empty((v.shape[0], 3, 3))
    a[:, 0, 0] = (y3 - y1) * (z4 - z1) - (y4 - y1) * (z3 - z1)
    a[:, 0, 1] = (y4 - y1) * (z2 - z1) - (y2 - y1) * (z4 - z1)
    a[:, 0, 2] = (y2 - y1) * (z3 - z1) - (y3 - y1) * (z2 - z1)
    a[:, 1, 0] = (x4 - x1) * (z3 - z1) - (x3 - x1) * (z4 - z1)
    a[:, 1, 1] = (x2 - x1) * (z4 - z1) - (x4 - x1) * (z2 - z1)
    a[:, 1, 2] = (x3 - x1) * (z2 - z1) - (x2 - x1) * (z3 - z1)
    a[:, 2, 0] = (x3 - x1) * (y4 - y1) - (x4 - x1) * (y3 - y1)
    a[:, 2, 1] = (x4 - x1) * (y2 - y1) - (x2 - x1) * (y4 - y1)
    a[:, 2, 2] = (x2 - x1) * (y3 - y1) - (x3 - x1) * (y2 - y1)
    return a
