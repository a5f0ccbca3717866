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


def kuhn_coarse_interpolation(s, s_coarse, interior_only=True):
    """Vertex interpolation from the coarse Kuhn grid (s_coarse^3 cubes) to the fine one.

    The fine grid (s = r s_coarse, r a power of two) refines every coarse Kuhn simplex into
    Kuhn simplices, so a continuous piecewise-linear field on the coarse mesh is linear on
    every fine element and is fixed by its values at the fine vertices.  For r = 2 a fine
    vertex lies at a coarse node or at the midpoint of a coarse Kuhn edge (the cube's main
    diagonal direction (1,1,1) and its face diagonals in the +,+ directions are edges).
    Returns nodes int32 [nver, 4] (-1 = unused) and weights f64 [nver, 4] over the coarse
    nodes numbered i + (s_c+1)(j + (s_c+1) l) -- or, with interior_only, over the interior
    coarse nodes only (boundary coarse values fixed to zero), plus the number of coarse
    unknowns.
    """
    if s == s_coarse:
        r = 1
    elif s == 2 * s_coarse:
        r = 2
    else:
        raise ValueError("only s = s_coarse or s = 2 s_coarse")
    n1, m1 = s + 1, s_coarse + 1
    I, J, L = np.meshgrid(np.arange(n1), np.arange(n1), np.arange(n1), indexing="ij")
    I, J, L = (a.transpose(2, 1, 0).ravel() for a in (I, J, L))  # vertex id = i + n1 (j + n1 l)
    if r == 1:
        ends = [(I, J, L, 1.0)]
    else:
        b0 = np.stack([I // 2, J // 2, L // 2], axis=1)
        odd = np.stack([I % 2, J % 2, L % 2], axis=1)
        # the fine vertex is the midpoint of the coarse edge from b0 to b0 + odd
        ends = [(b0[:, 0], b0[:, 1], b0[:, 2], 0.5), (b0[:, 0] + odd[:, 0], b0[:, 1] + odd[:, 1], b0[:, 2] + odd[:, 2], 0.5)]
        is_node = odd.sum(axis=1) == 0
    nodes = -np.ones((len(I), 4), np.int64)
    weights = np.zeros((len(I), 4))
    if interior_only:
        cid = -np.ones(m1 ** 3, np.int64)
        ii, jj, ll = np.meshgrid(np.arange(m1), np.arange(m1), np.arange(m1), indexing="ij")
        ii, jj, ll = (a.transpose(2, 1, 0).ravel() for a in (ii, jj, ll))
        inner = (ii > 0) & (ii < s_coarse) & (jj > 0) & (jj < s_coarse) & (ll > 0) & (ll < s_coarse)
        cid[inner] = np.arange(inner.sum())
        nc = int(inner.sum())
    else:
        cid = np.arange(m1 ** 3)
        nc = m1 ** 3
    for slot, (a, b, c, w) in enumerate(ends):
        g = cid[a + m1 * (b + m1 * c)]
        wt = np.full(len(I), w)
        if r == 2:
            wt = np.where(is_node, 1.0 if slot == 0 else 0.0, wt)
        ok = (g >= 0) & (wt != 0.0)
        nodes[ok, slot] = g[ok]
        weights[ok, slot] = wt[ok]
    return nodes.astype(np.int32), weights, nc


def _grid_ids(s):
    n1 = s + 1
    I, J, L = np.meshgrid(np.arange(n1), np.arange(n1), np.arange(n1), indexing="ij")
    return tuple(a.transpose(2, 1, 0).ravel() for a in (I, J, L))  # id = i + n1 (j + n1 l)


def _kept(s, fixed_planes):
    """Mask of grid vertices not on a fixed (Dirichlet) plane; planes are (axis, 0.0 or 1.0)."""
    ijk = _grid_ids(s)
    keep = np.ones((s + 1) ** 3, bool)
    for ax, val in fixed_planes:
        keep &= ijk[ax] != (0 if val == 0.0 else s)
    return keep


def kuhn_interpolation(s_fine, s_coarse):
    """Linear interpolation of the P1 field of the s_coarse^3 Kuhn grid at the vertices of the
    s_fine^3 grid (any two sizes): a fine vertex at x lies in the coarse cube c = floor(x s_c)
    and, with xi = x s_c - c sorted so that xi_a >= xi_b >= xi_d, in the Kuhn simplex
    c, c + e_a, c + e_a + e_b, c + 1 whose barycentric weights are 1 - xi_a, xi_a - xi_b,
    xi_b - xi_d, xi_d.  Returns nodes int64 [nver_fine, 4] (coarse vertex ids, -1 where the
    weight is 0) and weights f64 [nver_fine, 4].  For s_fine = 2 s_coarse this is the nested
    midpoint rule of kuhn_coarse_interpolation."""
    i, j, l = _grid_ids(s_fine)
    x = np.stack([i, j, l], axis=1) * (s_coarse / s_fine)
    cell = np.minimum(np.floor(x + 1e-12), s_coarse - 1).astype(np.int64)
    xi = np.clip(x - cell, 0.0, 1.0)
    order = np.argsort(-xi, axis=1, kind="stable")
    xs = np.take_along_axis(xi, order, axis=1)
    w = np.stack([1.0 - xs[:, 0], xs[:, 0] - xs[:, 1], xs[:, 1] - xs[:, 2], xs[:, 2]], axis=1)
    corner = cell.copy()
    nodes = np.empty((len(i), 4), np.int64)
    m1 = s_coarse + 1
    nodes[:, 0] = corner[:, 0] + m1 * (corner[:, 1] + m1 * corner[:, 2])
    for q in range(3):
        corner[np.arange(len(i)), order[:, q]] += 1
        nodes[:, q + 1] = corner[:, 0] + m1 * (corner[:, 1] + m1 * corner[:, 2])
    w = np.where(np.abs(w) < 1e-13, 0.0, w)
    nodes = np.where(w != 0.0, nodes, -1)
    return nodes, w


def kuhn_p1_hierarchy(s, fixed_planes, max_coarsest=64, strict=True):
    """Continuous P1 spaces for the two-level trace preconditioner of an s^3 Kuhn cube.

    Level 0 is the P1 space of the mesh itself (one node per vertex not on a fixed plane);
    level l+1 is the P1 space of the Kuhn grid with ceil(s_l / 2) cells per side, down to the
    first level with at most max_coarsest nodes.  Returns (sizes [nlev], nodes int32 [R, 4],
    weights f64 [R, 4]) with R = nver + sizes[0] + ... + sizes[nlev-2]: first, for every mesh
    vertex, its level-0 node (weight 1; -1 on a fixed plane); then, for every node of level l,
    the level-(l+1) nodes and weights that interpolate it (kuhn_interpolation; values on a
    fixed plane are 0 and drop out).  For even sizes the levels are nested.  With
    strict=False a grid too small to coarsen returns the levels built so far (possibly one
    level, possibly empty) instead of raising.
    """
    keep = _kept(s, fixed_planes)
    ids = -np.ones((s + 1) ** 3, np.int64)
    ids[keep] = np.arange(keep.sum())
    sizes = [int(keep.sum())]
    nodes = [np.stack([ids, -np.ones_like(ids), -np.ones_like(ids), -np.ones_like(ids)], axis=1)]
    weights = [np.stack([np.where(keep, 1.0, 0.0), np.zeros(len(ids)), np.zeros(len(ids)), np.zeros(len(ids))],
                        axis=1)]
    cur = s
    while sizes[-1] > max_coarsest:
        nxt = (cur + 1) // 2
        keep_c = _kept(nxt, fixed_planes)
        if nxt == cur or not keep_c.any():
            if strict:
                raise ValueError("cannot coarsen further")
            break
        nd, wt = kuhn_interpolation(cur, nxt)
        cid = -np.ones((nxt + 1) ** 3, np.int64)
        cid[keep_c] = np.arange(keep_c.sum())
        rows_f = np.nonzero(_kept(cur, fixed_planes))[0]  # level-l nodes in id order
        nd, wt = nd[rows_f], wt[rows_f]
        mapped = np.where(nd >= 0, cid[np.maximum(nd, 0)], -1)
        wt = np.where(mapped >= 0, wt, 0.0)
        nodes.append(mapped)
        weights.append(wt)
        sizes.append(int(keep_c.sum()))
        cur = nxt
    if len(sizes) < 2 and strict:
        raise ValueError("the hierarchy needs at least two levels")
    return sizes, np.concatenate(nodes).astype(np.int32), np.concatenate(weights)


def kuhn_grid_points(s, interior_only=True):
    """Coordinates [n, 3] of the vertices of the s^3 grid in vertex-id order (the numbering of
    kuhn_coarse_interpolation's coarse nodes), interior vertices only if asked."""
    i, j, l = _grid_ids(s)
    pts = np.stack([i, j, l], axis=1) / s
    if interior_only:
        keep = (i > 0) & (i < s) & (j > 0) & (j < s) & (l > 0) & (l < s)
        pts = pts[keep]
    return pts
