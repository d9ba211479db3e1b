"""Mesh topology and FP64 geometry of a simplicial mesh (oracle; test infrastructure).

Follows Section 2.1 of the paper: unknowns live at cell centres (the centre of
gravity of the cell, i.e. the vertex mean for a simplex); fluxes live on faces with
measure |sigma_ij| and unit normal n_ij (eq. 2-4). The area vector S_f = |sigma_f| n_f
of a face is oriented from its owner cell L towards its other cell R (towards the
outside for a boundary face).
"""
from __future__ import annotations

from math import factorial

import numpy as np


class MeshError(ValueError):
    pass


class Geometry:
    """Faces and geometry of a positively oriented triangle / tetrahedron mesh.

    Attributes (user order, FP64):
      dim, n_cell, n_vert, n_face
      xyz[V, d], cells[N, d+1]
      cen[N, d]   cell centre of gravity (vertex mean)
      vol[N]      cell measure mu_i (area in 2D, volume in 3D)
      face_L[F], face_R[F]   owner cell and other cell (-1 on the boundary)
      face_vert[F, d]        the face's vertex ids in increasing order (A, B[, C])
      face_tag[F]            boundary tag, 0 for interior faces
      S[F, d]                area vector, |S| = face measure, oriented L -> R / outwards
      xf[F, d]               face centroid (vertex mean)
    """

    def __init__(self, dim, xyz, cells, bface_vert, bface_tag):
        d = int(dim)
        if d not in (2, 3):
            raise MeshError("dim must be 2 or 3")
        xyz = np.asarray(xyz, dtype=np.float64)
        cells = np.asarray(cells, dtype=np.int64)
        V, N = xyz.shape[0], cells.shape[0]
        if cells.shape[1] != d + 1 or xyz.shape[1] != d:
            raise MeshError("bad array shapes")
        if cells.size and (cells.min() < 0 or cells.max() >= V):
            raise MeshError("cell vertex index out of range")
        self.dim, self.xyz, self.cells = d, xyz, cells
        self.n_cell, self.n_vert = N, V

        X = xyz[cells]                                   # N, d+1, d
        self.cen = X.mean(axis=1)
        det = np.linalg.det(X[:, 1:, :] - X[:, :1, :])   # N
        if np.any(det <= 0.0):
            raise MeshError("cell with non-positive orientation")
        self.vol = det / factorial(d)

        # every cell has d+1 faces: local face k omits local vertex k
        loc = [[v for v in range(d + 1) if v != k] for k in range(d + 1)]
        fv = np.concatenate([cells[:, lk] for lk in loc], axis=0)
        owner = np.tile(np.arange(N), d + 1)
        key = np.sort(fv, axis=1)
        uniq, inv, cnt = np.unique(key, axis=0, return_inverse=True, return_counts=True)
        inv = inv.ravel()
        if np.any(cnt > 2):
            raise MeshError("face shared by more than two cells")
        F = uniq.shape[0]
        order = np.argsort(inv, kind="stable")
        first = np.zeros(F, dtype=np.int64)
        first[1:] = np.cumsum(cnt)[:-1]
        c0 = owner[order[first]]
        c1 = np.where(cnt == 2, owner[order[np.minimum(first + 1, len(order) - 1)]], -1)
        L = np.where(cnt == 2, np.minimum(c0, c1), c0)
        R = np.where(cnt == 2, np.maximum(c0, c1), -1)
        self.n_face = F
        self.face_vert = uniq
        self.face_L, self.face_R = L, R

        P = xyz[uniq]                                    # F, d, d
        self.xf = P.mean(axis=1)
        if d == 3:
            S = 0.5 * np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
        else:
            t = P[:, 1] - P[:, 0]
            S = np.stack([t[:, 1], -t[:, 0]], axis=1)
        xR = np.where((R >= 0)[:, None], self.cen[np.maximum(R, 0)], self.xf)
        flip = np.einsum("fi,fi->f", S, xR - self.cen[L]) < 0.0
        S[flip] *= -1.0
        self.S = S

        # boundary tags: every boundary face gets exactly one tag from the list
        bkey = np.sort(np.asarray(bface_vert, dtype=np.int64), axis=1)
        btag = np.asarray(bface_tag, dtype=np.int64)
        is_b = R < 0
        self.face_tag = np.zeros(F, dtype=np.int64)
        if bkey.shape[0] != int(is_b.sum()):
            raise MeshError("boundary face list does not match the mesh boundary")
        allk = np.concatenate([uniq[is_b], bkey])
        u2, inv2, c2 = np.unique(allk, axis=0, return_inverse=True, return_counts=True)
        if np.any(c2 != 2):
            raise MeshError("boundary face list does not match the mesh boundary")
        inv2 = inv2.ravel()
        tag_of_key = np.zeros(u2.shape[0], dtype=np.int64)
        tag_of_key[inv2[is_b.sum():]] = btag
        self.face_tag[np.nonzero(is_b)[0]] = tag_of_key[inv2[: is_b.sum()]]
        if np.any(self.face_tag[is_b] <= 0):
            raise MeshError("boundary tags must be positive")

    # convenience views -------------------------------------------------------
    @property
    def interior(self):
        return self.face_R >= 0

    def faces_with_kind(self, bc, kind):
        """Boundary faces whose tag has boundary-condition kind ``kind``."""
        tags = [t for t, (k, _v) in bc.items() if k == kind]
        return np.nonzero((self.face_R < 0) & np.isin(self.face_tag, tags))[0]

    def check_bc(self, bc):
        tags = set(np.unique(self.face_tag[self.face_R < 0]).tolist())
        missing = tags - set(bc.keys())
        if missing:
            raise MeshError(f"no boundary condition for tags {sorted(missing)}")
        for t, (k, _v) in bc.items():
            if k not in ("wall", "neumann", "dirichlet"):
                raise MeshError(f"unknown boundary kind {k!r}")
