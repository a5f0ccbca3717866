"""Structured tetrahedral meshes of the unit cube (input generator, no method arithmetic).

The cube [0,1]^3 is cut into s^3 subcubes, each split into the 6 Kuhn tetrahedra that share
the subcube's main diagonal.  All subcubes use the same diagonal direction, so the mesh is
conforming.  Elements are listed with positive orientation (det B_K > 0, Section 2 of the
paper).  Optionally the interior vertices are jittered by a seeded uniform perturbation.
"""

import itertools

import numpy as np

# The 6 Kuhn simplices of the unit cube: walk from corner 000 to 111 along the axes in the
# order of a permutation.
_PERMS = list(itertools.permutations(range(3)))


def _vid(i, j, l, s):
    return i + (s + 1) * (j + (s + 1) * l)


def kuhn_cube(s, jitter=0.0, seed=0):
    """Return (coords [Nver,3] f64, elements [Nelt,4] int32) for an s^3 x 6 Kuhn cube.

    jitter: interior vertices move by U(-jitter*h, jitter*h)^3 with h = 1/s (numpy
    default_rng(seed)).  Element orientation is fixed from the unjittered mesh; callers
    check that jitter keeps it positive.
    """
    n1 = s + 1
    g = np.arange(n1, dtype=np.float64) / s
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")  # vertex id = i + n1*(j + n1*l)
    coords = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)

    # Subcube corners (i, j, l), i fastest, then the 6 Kuhn walks per subcube.
    L, J, I = np.meshgrid(np.arange(s), np.arange(s), np.arange(s), indexing="ij")
    base = np.stack([I.ravel(), J.ravel(), L.ravel()], axis=1)  # [s^3, 3]
    unit = np.eye(3, dtype=np.int64)
    walks = []
    for p in _PERMS:
        c0 = base
        c1 = c0 + unit[p[0]]
        c2 = c1 + unit[p[1]]
        c3 = c2 + unit[p[2]]
        walks.append(np.stack([_vid(c[:, 0], c[:, 1], c[:, 2], s) for c in (c0, c1, c2, c3)], axis=1))
    elems = np.stack(walks, axis=1).reshape(-1, 4).astype(np.int64)  # [s^3*6, 4]

    # Orientation: swap the last two vertices where the signed volume is negative.
    v = coords[elems]
    d = np.einsum("ij,ij->i", np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]), v[:, 3] - v[:, 0])
    neg = d < 0
    elems[neg, 2], elems[neg, 3] = elems[neg, 3].copy(), elems[neg, 2].copy()

    if jitter:
        rng = np.random.default_rng(seed)
        h = 1.0 / s
        interior = np.all((coords > 1e-12) & (coords < 1 - 1e-12), axis=1)
        pert = rng.uniform(-jitter * h, jitter * h, size=coords.shape)
        coords = coords + pert * interior[:, None]
    return coords, elems.astype(np.int32)


def boundary_faces(coords, elems, classify):
    """Boundary faces of a cube mesh as vertex triples, split by `classify`.

    A face lies on the boundary when its three vertices share one of the planes x, y or
    z in {0, 1}.  classify(plane_axis, plane_value) returns "D" or "N".  Returns
    (dirichlet [Ndir,3] int32, neumann [Nneu,3] int32), each triple ordered so that its
    normal (w2-w1)x(w3-w1) points out of the cube (the paper's positive orientation).
    """
    tol = 1e-12
    local = np.array([(0, 1, 2), (0, 1, 3), (0, 2, 3), (3, 1, 2)])
    tri = elems[:, local].reshape(-1, 3).astype(np.int64)  # every element face
    p = coords[tri]  # [F,3,3]
    dirs, neus = [], []
    for ax in range(3):
        for val in (0.0, 1.0):
            on = np.all(np.abs(p[:, :, ax] - val) < tol, axis=1)
            t = tri[on].copy()
            q = p[on]
            nrm = np.cross(q[:, 1] - q[:, 0], q[:, 2] - q[:, 0])
            out = 1.0 if val == 1.0 else -1.0
            flip = nrm[:, ax] * out < 0
            t[flip, 1], t[flip, 2] = t[flip, 2].copy(), t[flip, 1].copy()
            (dirs if classify(ax, val) == "D" else neus).append(t)
    d = np.concatenate(dirs).astype(np.int32).reshape(-1, 3) if dirs else np.zeros((0, 3), np.int32)
    n = np.concatenate(neus).astype(np.int32).reshape(-1, 3) if neus else np.zeros((0, 3), np.int32)
    return d, n
