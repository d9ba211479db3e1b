"""Seeded synthetic inputs: jittered simplicial meshes of the unit square / cube and
initial fields.

This module produces INPUTS only. It holds none of the finite-volume arithmetic
(no face extraction, no geometry, no gradients, no fluxes): the CPU oracle and the
GPU library each derive those on their own from the arrays returned here.

Mesh recipe (stands in for the paper's gmsh meshes G1/G15/G30 and the annex
``cube.msh``, which are not available):

* 2D: unit square, ``n x n`` quads on the ``(n+1)^2`` lattice points, spacing h=1/n.
  Every point moves by an independent uniform offset in [-jitter*h, +jitter*h] per
  coordinate; a point on the boundary keeps the coordinate normal to its side (it
  slides tangentially), corners stay put. Each quad is split into two triangles
  along a diagonal drawn by a second seeded stream. Triangles are counter-clockwise.
* 3D: unit cube, ``k^3`` hexes on the ``(k+1)^3`` lattice, jittered the same way,
  each hex split into the 6 Kuhn tetrahedra that share its main diagonal
  (000)-(111). The split is conforming across hexes. Tetrahedra are positively
  oriented (det[x1-x0, x2-x0, x3-x0] > 0).
* Boundary faces (edges in 2D, triangles in 3D) are listed with a tag per side:
  1: x=0, 2: x=1, 3: y=0, 4: y=1, 5: z=0, 6: z=1.

Random numbers come from numpy's PCG64 stream seeded by the given integer.
"""
from __future__ import annotations

import numpy as np

TAG_X0, TAG_X1, TAG_Y0, TAG_Y1, TAG_Z0, TAG_Z1 = 1, 2, 3, 4, 5, 6


class Mesh:
    """Plain container for a simplicial mesh as handed to a solver."""

    def __init__(self, dim, xyz, cells, bface_vert, bface_tag, h):
        self.dim = int(dim)
        self.xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        self.cells = np.ascontiguousarray(cells, dtype=np.int32)
        self.bface_vert = np.ascontiguousarray(bface_vert, dtype=np.int32)
        self.bface_tag = np.ascontiguousarray(bface_tag, dtype=np.int32)
        self.h = float(h)

    @property
    def n_cell(self):
        return self.cells.shape[0]

    @property
    def n_vert(self):
        return self.xyz.shape[0]

    def vertex_mean(self):
        """Arithmetic mean of each cell's vertices, used only to lay down initial fields."""
        return self.xyz[self.cells].mean(axis=1)


def _jitter_lattice(n, dim, jitter, rng):
    h = 1.0 / n
    axes = np.meshgrid(*([np.arange(n + 1)] * dim), indexing="ij")
    idx = np.stack([a.ravel() for a in axes], axis=1)  # lexicographic, last axis fastest
    xyz = idx * h
    off = rng.uniform(-jitter * h, jitter * h, size=xyz.shape)
    on_bnd = (idx == 0) | (idx == n)
    off[on_bnd] = 0.0
    return xyz + off, idx


def jittered_square(n, seed_jitter=101, seed_diag=102, jitter=0.2):
    """2D jittered triangle mesh of the unit square (2 n^2 cells)."""
    xyz, _ = _jitter_lattice(n, 2, jitter, np.random.default_rng(seed_jitter))

    def vid(i, j):
        return i * (n + 1) + j

    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    i = i.ravel()
    j = j.ravel()
    v00, v10, v01, v11 = vid(i, j), vid(i + 1, j), vid(i, j + 1), vid(i + 1, j + 1)
    diag = np.random.default_rng(seed_diag).integers(0, 2, size=i.size)
    t1 = np.where(diag[:, None] == 0, np.stack([v00, v10, v11], 1), np.stack([v00, v10, v01], 1))
    t2 = np.where(diag[:, None] == 0, np.stack([v00, v11, v01], 1), np.stack([v10, v11, v01], 1))
    cells = np.stack([t1, t2], axis=1).reshape(-1, 3)

    s = np.arange(n)
    bv, bt = [], []
    bv.append(np.stack([vid(0, s), vid(0, s + 1)], 1)); bt.append(np.full(n, TAG_X0))
    bv.append(np.stack([vid(n, s), vid(n, s + 1)], 1)); bt.append(np.full(n, TAG_X1))
    bv.append(np.stack([vid(s, 0), vid(s + 1, 0)], 1)); bt.append(np.full(n, TAG_Y0))
    bv.append(np.stack([vid(s, n), vid(s + 1, n)], 1)); bt.append(np.full(n, TAG_Y1))
    return Mesh(2, xyz, cells, np.concatenate(bv), np.concatenate(bt), 1.0 / n)


# Kuhn subdivision of the unit hex: one tetrahedron per permutation of the axes,
# walking 000 -> e_a -> e_a+e_b -> 111. Odd permutations swap the two middle
# vertices so that every tetrahedron is positively oriented.
_PERMS = [((0, 1, 2), +1), ((1, 2, 0), +1), ((2, 0, 1), +1),
          ((0, 2, 1), -1), ((2, 1, 0), -1), ((1, 0, 2), -1)]


def _kuhn_corners():
    tets = []
    for (a, b, _c), sign in _PERMS:
        p0 = (0, 0, 0)
        p1 = [0, 0, 0]; p1[a] = 1
        p2 = list(p1); p2[b] = 1
        p3 = (1, 1, 1)
        t = [p0, tuple(p1), tuple(p2), p3]
        if sign < 0:
            t = [t[0], t[2], t[1], t[3]]
        tets.append(t)
    return tets


def jittered_cube(k, seed=201, jitter=0.2):
    """3D jittered Kuhn-tetrahedron mesh of the unit cube (6 k^3 cells)."""
    xyz, _ = _jitter_lattice(k, 3, jitter, np.random.default_rng(seed))

    def vid(i, j, l):
        return (i * (k + 1) + j) * (k + 1) + l

    i, j, l = np.meshgrid(np.arange(k), np.arange(k), np.arange(k), indexing="ij")
    i = i.ravel(); j = j.ravel(); l = l.ravel()
    cells = []
    for tet in _kuhn_corners():
        cells.append(np.stack([vid(i + c[0], j + c[1], l + c[2]) for c in tet], 1))
    cells = np.stack(cells, axis=1).reshape(-1, 4)

    # boundary triangles: on each side the Kuhn faces split a lattice square along the
    # diagonal joining its lowest and highest corner in the side's two axes
    s, t = np.meshgrid(np.arange(k), np.arange(k), indexing="ij")
    s = s.ravel(); t = t.ravel()
    bv, bt = [], []
    sides = [(0, 0, TAG_X0), (0, k, TAG_X1), (1, 0, TAG_Y0), (1, k, TAG_Y1), (2, 0, TAG_Z0), (2, k, TAG_Z1)]
    for axis, fixed, tag in sides:
        ax = [a for a in range(3) if a != axis]

        def point(ds, dt):
            c = [None, None, None]
            c[axis] = np.full_like(s, fixed)
            c[ax[0]] = s + ds
            c[ax[1]] = t + dt
            return vid(c[0], c[1], c[2])

        p00, p10, p01, p11 = point(0, 0), point(1, 0), point(0, 1), point(1, 1)
        bv.append(np.stack([p00, p10, p11], 1)); bt.append(np.full(s.size, tag))
        bv.append(np.stack([p00, p11, p01], 1)); bt.append(np.full(s.size, tag))
    return Mesh(3, xyz, cells, np.concatenate(bv), np.concatenate(bt), 1.0 / k)


def ensemble_sizes(n_mesh=64, lo=20_000, hi=1_000_000, seed=5000):
    """Cell-count targets log-uniform in [lo, hi] and the cube resolutions k that
    realise them (6 k^3 cells closest to the target)."""
    rng = np.random.default_rng(seed)
    target = np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_mesh))
    k = np.maximum(2, np.round((target / 6.0) ** (1.0 / 3.0)).astype(int))
    return target, k


def gaussian(points, centre, sigma, peak=1.0, background=0.0):
    """peak * exp(-|x - centre|^2 / sigma^2) + background (the paper's convention,
    Section 4, initial conditions)."""
    r2 = ((points - np.asarray(centre)[None, :]) ** 2).sum(axis=1)
    return peak * np.exp(-r2 / sigma ** 2) + background
