"""Sub-mesh around sampled cells, for checking full-size GPU results cell by cell.

A cell's transport update depends on the cells that share a vertex with it (its
least-squares gradient and the vertex values of its faces) and, through the field
E = -grad phi of its face neighbours, on their node neighbours too. ``patch`` keeps the
cells within ``rings`` node-neighbour rings of the sample, renumbers their vertices,
keeps each original boundary face with its tag and gives every face that the cut opens
the tag ``cut_tag``. Evaluated on the patch, the oracle then gives the sampled cells'
values exactly as on the whole mesh, provided the boundary conditions of ``cut_tag``
are not Dirichlet (wall and Neumann faces add nothing to the gradients or the vertex
values, and the cut faces touch no sampled cell).

Topology only: no geometry and none of the method's arithmetic.
"""
from __future__ import annotations

import numpy as np

from synth.meshgen import Mesh


def vertex_cells(cells, n_vert):
    """CSR (ptr, idx) of the cells around each vertex."""
    v = cells.ravel()
    c = np.repeat(np.arange(cells.shape[0]), cells.shape[1])
    order = np.argsort(v, kind="stable")
    ptr = np.zeros(n_vert + 1, dtype=np.int64)
    np.add.at(ptr, v + 1, 1)
    return np.cumsum(ptr), c[order]


def node_closure(cells, ptr, idx, sel):
    """The cells sharing a vertex with a cell of ``sel`` (``sel`` included)."""
    verts = np.unique(cells[sel].ravel())
    parts = [idx[ptr[a]:ptr[a + 1]] for a in verts]
    return np.unique(np.concatenate(parts + [np.asarray(sel)]))


def patch(mesh, sample, rings=2, cut_tag=1):
    """(sub-mesh, ids of its cells in ``mesh``, positions of ``sample`` in the sub-mesh)."""
    ptr, idx = vertex_cells(mesh.cells, mesh.n_vert)
    keep = np.unique(np.asarray(sample))
    for _ in range(rings):
        keep = node_closure(mesh.cells, ptr, idx, keep)
    cells = mesh.cells[keep]
    verts, local = np.unique(cells.ravel(), return_inverse=True)
    lcells = local.reshape(cells.shape).astype(np.int32)
    nv = mesh.cells.shape[1]
    # faces of the kept cells: a face seen once is on the patch boundary
    faces = np.concatenate([np.delete(lcells, j, axis=1) for j in range(nv)])
    key = np.sort(faces, axis=1)
    uniq, inv, cnt = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    once = np.flatnonzero(cnt[inv.ravel()] == 1)
    bfaces = faces[once]
    # original boundary faces (in the sub-mesh's vertex numbers) keep their tags
    g2l = -np.ones(mesh.n_vert, dtype=np.int64)
    g2l[verts] = np.arange(verts.size)
    ob = g2l[mesh.bface_vert]
    inside = (ob >= 0).all(axis=1)
    tag_of = {tuple(k): t for k, t in zip(np.sort(ob[inside], axis=1), mesh.bface_tag[inside])}
    tags = np.array([tag_of.get(tuple(k), cut_tag) for k in np.sort(bfaces, axis=1)], dtype=np.int32)
    sub = Mesh(mesh.dim, mesh.xyz[verts], lcells, bfaces.astype(np.int32), tags, mesh.h)
    pos = np.searchsorted(keep, np.asarray(sample))
    return sub, keep, pos
