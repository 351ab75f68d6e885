"""Seeded tetrahedral meshes: a tensor-product hexahedral grid, each cell split
into the six Kuhn tetrahedra that share the cell diagonal (0,0,0)->(1,1,1).

The Kuhn split is translation invariant, so neighbouring cells produce
conforming faces and a periodic wrap is conforming as well.  Periodic vertices
share one vertex id; per-element coordinates are the *unwrapped* positions, so
a tetrahedron that straddles the wrap keeps its true shape.

Nothing here evaluates the numerical method: the arrays are what the C-ABI
call ``dg_mesh_create`` and the oracle both take as input.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

# Face f of a tetrahedron is the face opposite local vertex f.
FACE_BC_INTERIOR = 0
FACE_BC_FREE_SURFACE = 1
FACE_BC_ABSORBING = 2


@dataclass
class Mesh:
    elem_xyz: np.ndarray          # [E,4,3] float64, unwrapped vertex coordinates
    elem_vid: np.ndarray          # [E,4] int64, global vertex ids (periodic images share ids)
    face_bc: np.ndarray           # [E,4] int8, boundary tag of the face opposite each vertex
    cells: tuple                  # (nx, ny, nz) hexahedral cells
    periodic: tuple               # (px, py, pz) booleans
    extent: np.ndarray            # [3] box size
    meta: dict = field(default_factory=dict)

    @property
    def n_elem(self) -> int:
        return int(self.elem_xyz.shape[0])

    def centroids(self) -> np.ndarray:
        return self.elem_xyz.mean(axis=1)

    def permuted(self, elem_perm=None, vertex_perm=None) -> "Mesh":
        """Relabel elements (elem_perm[new] = old) and/or reorder each element's
        local vertices (vertex_perm[e] is a permutation of 0..3)."""
        xyz, vid, bc = self.elem_xyz, self.elem_vid, self.face_bc
        if elem_perm is not None:
            xyz, vid, bc = xyz[elem_perm], vid[elem_perm], bc[elem_perm]
        if vertex_perm is not None:
            rows = np.arange(xyz.shape[0])[:, None]
            xyz = xyz[rows, vertex_perm]
            vid = vid[rows, vertex_perm]
            bc = bc[rows, vertex_perm]          # face f is opposite vertex f: moves with it
        return Mesh(np.ascontiguousarray(xyz), np.ascontiguousarray(vid),
                    np.ascontiguousarray(bc), self.cells, self.periodic, self.extent.copy(),
                    dict(self.meta))


def _kuhn_offsets():
    """The six Kuhn tetrahedra of the unit cube as lists of 4 corner offsets,
    each listed with positive orientation."""
    tets = []
    for perm in itertools.permutations(range(3)):
        e = np.eye(3, dtype=np.int64)
        p0 = np.zeros(3, dtype=np.int64)
        p1 = e[perm[0]]
        p2 = e[perm[0]] + e[perm[1]]
        p3 = np.ones(3, dtype=np.int64)
        verts = [p0, p1, p2, p3]
        det = np.linalg.det(np.stack([p1 - p0, p2 - p0, p3 - p0], axis=1).astype(float))
        if det < 0:
            verts = [p0, p2, p1, p3]
        tets.append(np.stack(verts))
    return np.stack(tets)  # [6,4,3]


def kuhn_box_mesh(xs, ys, zs, periodic=(True, True, True), jitter=0.0, seed=1,
                  sort_by_vid=False, top_bc=FACE_BC_FREE_SURFACE,
                  side_bc=FACE_BC_ABSORBING) -> Mesh:
    """Tetrahedral mesh of the box spanned by the grid lines xs, ys, zs.

    jitter: each unique vertex moves by U(-jitter*h, jitter*h) per coordinate
    (h = local minimum grid spacing, seeded).  On non-periodic boundaries the
    normal coordinate of boundary vertices is not moved, so the box keeps its
    shape.  sort_by_vid lists each element's vertices by increasing vertex id.
    Non-periodic box faces are tagged: z-max with ``top_bc``, the others with
    ``side_bc``.
    """
    grids = [np.asarray(g, dtype=np.float64) for g in (xs, ys, zs)]
    ncell = tuple(len(g) - 1 for g in grids)
    nvert = tuple(n if p else n + 1 for n, p in zip(ncell, periodic))
    rng = np.random.default_rng(seed)

    # per-unique-vertex jitter, drawn in vid order
    n_unique = nvert[0] * nvert[1] * nvert[2]
    jit = rng.uniform(-1.0, 1.0, size=(n_unique, 3)) * jitter
    spacing = []
    for g, p in zip(grids, periodic):
        d = np.diff(g)
        # local spacing at grid line i = min of adjacent cells
        h = np.empty(len(g))
        h[1:-1] = np.minimum(d[:-1], d[1:])
        h[0] = min(d[0], d[-1]) if p else d[0]
        h[-1] = h[0] if p else d[-1]
        spacing.append(h)

    def vid_of(i, j, k):
        ii = i % nvert[0] if periodic[0] else i
        jj = j % nvert[1] if periodic[1] else j
        kk = k % nvert[2] if periodic[2] else k
        return ii + nvert[0] * (jj + nvert[1] * kk)

    offs = _kuhn_offsets()
    nx, ny, nz = ncell
    ci, cj, ck = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    # x fastest
    cells = np.stack([ci.transpose(2, 1, 0).ravel(), cj.transpose(2, 1, 0).ravel(),
                      ck.transpose(2, 1, 0).ravel()], axis=1)
    lat = cells[:, None, None, :] + offs[None, :, :, :]       # [C,6,4,3] lattice indices
    lat = lat.reshape(-1, 4, 3)
    E = lat.shape[0]
    vid = vid_of(lat[..., 0], lat[..., 1], lat[..., 2]).astype(np.int64)

    xyz = np.empty((E, 4, 3))
    for d in range(3):
        g = grids[d]
        xyz[..., d] = g[lat[..., d]]
        hj = spacing[d][lat[..., d]]
        shift = jit[vid, d] * hj
        if not periodic[d]:
            on_bnd = (lat[..., d] == 0) | (lat[..., d] == ncell[d])
            shift = np.where(on_bnd, 0.0, shift)
        xyz[..., d] += shift

    face_bc = np.zeros((E, 4), dtype=np.int8)
    for d in range(3):
        if periodic[d]:
            continue
        for side, val in ((0, 0), (1, ncell[d])):
            on = lat[..., d] == val                              # [E,4]
            for f in range(4):
                others = [v for v in range(4) if v != f]
                face_on = on[:, others].all(axis=1)
                tag = top_bc if (d == 2 and side == 1) else side_bc
                face_bc[face_on, f] = tag

    if sort_by_vid:
        order = np.argsort(vid, axis=1, kind="stable")
        rows = np.arange(E)[:, None]
        xyz, vid, face_bc = xyz[rows, order], vid[rows, order], face_bc[rows, order]

    extent = np.array([g[-1] - g[0] for g in grids])
    return Mesh(np.ascontiguousarray(xyz), np.ascontiguousarray(vid),
                np.ascontiguousarray(face_bc), ncell, tuple(periodic), extent,
                {"jitter": jitter, "seed": seed})


def periodic_cube_mesh(n, side, jitter=0.0, seed=1, sort_by_vid=False) -> Mesh:
    """n^3 cubes x 6 Kuhn tetrahedra of the periodic cube [0, side]^3."""
    g = np.linspace(0.0, side, n + 1)
    return kuhn_box_mesh(g, g, g, periodic=(True, True, True), jitter=jitter, seed=seed,
                         sort_by_vid=sort_by_vid)
