"""Least-squares cell gradient (Algorithm "grad") and least-squares vertex
interpolation (Algorithm "ls") - oracle, test infrastructure only.

Readings where the paper is silent (the same readings are used by the GPU library,
which implements them independently):

* Node neighbours of cell i: the SET of cells that share at least one vertex with
  T_i, without T_i itself (each cell counted once).
* Ghost cells "neighbour by node": for a Dirichlet boundary face that shares a
  vertex with T_i, one extra least-squares point at the face centroid x_f with the
  boundary value g. Wall and Neumann faces add nothing (one-sided fit), which keeps
  the reconstruction exact for linear fields.
* The elided f(A_x, A_y, A_z, D) of Algorithm "grad" is the solution of the normal
  equations M_i grad = J_i with M_i = sum d d^T, J_i = sum d (u_j - u_i),
  d = x_j - x_i (A = components of d, D = det M_i).
* The weights alpha of Algorithm "ls", which the paper attributes to a least-squares
  method without giving it: the weights of an unweighted linear least-squares fit u ~ a + b.(x - x_A) over the
  cells around vertex A, u_A = a. When the fit is degenerate (fewer than d+1 cells,
  or the centred scatter matrix C of the cell centres has det C / (tr C / d)^d below
  1e-10) the weights are the plain mean 1/n. A vertex on a Dirichlet face takes the
  boundary value; with several Dirichlet tags at one vertex the smallest tag wins.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

DEGENERATE_RATIO = 1e-10


def _cell_vertex_incidence(geo):
    N, k = geo.cells.shape
    rows = np.repeat(np.arange(N), k)
    return sp.csr_matrix((np.ones(N * k), (rows, geo.cells.ravel())), shape=(N, geo.n_vert))


def node_neighbour_pairs(geo, with_counts=False):
    """(i, j) for every cell j != i sharing >= 1 vertex with cell i (a set); with_counts
    also returns the number of vertices they share."""
    C2V = _cell_vertex_incidence(geo)
    P = (C2V @ C2V.T).tocoo()
    keep = P.row != P.col
    i, j = P.row[keep].astype(np.int64), P.col[keep].astype(np.int64)
    w = np.rint(P.data[keep]).astype(np.int64)
    o = np.lexsort((j, i))
    return (i[o], j[o], w[o]) if with_counts else (i[o], j[o])


def dirichlet_values(geo, bc):
    """Boundary value g_f of every face (NaN where the face is not Dirichlet)."""
    g = np.full(geo.n_face, np.nan)
    for t, (kind, val) in bc.items():
        if kind == "dirichlet":
            g[(geo.face_R < 0) & (geo.face_tag == t)] = float(val)
    return g


def ghost_point_pairs(geo, bc, with_counts=False):
    """(i, f) for every Dirichlet boundary face f sharing >= 1 vertex with cell i;
    with_counts also returns the number of vertices they share."""
    fd = geo.faces_with_kind(bc, "dirichlet")
    if fd.size == 0:
        z = np.zeros(0, np.int64)
        return (z, z, z) if with_counts else (z, z)
    C2V = _cell_vertex_incidence(geo)
    nv = geo.face_vert.shape[1]
    F2V = sp.csr_matrix((np.ones(fd.size * nv), (np.repeat(np.arange(fd.size), nv),
                                                 geo.face_vert[fd].ravel())),
                        shape=(fd.size, geo.n_vert))
    Q = (C2V @ F2V.T).tocoo()
    i, f = Q.row.astype(np.int64), fd[Q.col]
    w = np.rint(Q.data).astype(np.int64)
    o = np.lexsort((f, i))
    return (i[o], f[o], w[o]) if with_counts else (i[o], f[o])


def ls_gradient(geo, bc, u):
    """Cell gradient of Algorithm "grad": grad u_i = M_i^{-1} J_i (FP64)."""
    geo.check_bc(bc)
    u = np.asarray(u, dtype=np.float64)
    d = geo.dim
    i, j = node_neighbour_pairs(geo)
    dx = geo.cen[j] - geo.cen[i]
    du = u[j] - u[i]
    gi, gf = ghost_point_pairs(geo, bc)
    if gi.size:
        g = dirichlet_values(geo, bc)
        dx = np.concatenate([dx, geo.xf[gf] - geo.cen[gi]])
        du = np.concatenate([du, g[gf] - u[gi]])
        i = np.concatenate([i, gi])
    N = geo.n_cell
    M = np.zeros((N, d, d))
    J = np.zeros((N, d))
    for a in range(d):
        J[:, a] = np.bincount(i, weights=dx[:, a] * du, minlength=N)
        for b in range(d):
            M[:, a, b] = np.bincount(i, weights=dx[:, a] * dx[:, b], minlength=N)
    return np.linalg.solve(M, J[:, :, None])[:, :, 0]


def ls_gradient_vertex(geo, bc, u):
    """Multiplicity-weighted variant of Algorithm "grad" (not in the paper; the
    vertex-factorised gradient): every node neighbour j of T_i, and every Dirichlet ghost
    point of Algorithm "grad", counts once per vertex it shares with T_i -
    grad u_i = M_i^{-1} J_i with M_i = sum m d d^T, J_i = sum m d (u_j - u_i). This is the
    sum over the vertices A of T_i of the stencil of the cells (and Dirichlet faces) around
    A; it is exact for linear fields like Algorithm "grad"."""
    geo.check_bc(bc)
    u = np.asarray(u, dtype=np.float64)
    d = geo.dim
    i, j, w = node_neighbour_pairs(geo, with_counts=True)
    dx = geo.cen[j] - geo.cen[i]
    du = u[j] - u[i]
    gi, gf, gw = ghost_point_pairs(geo, bc, with_counts=True)
    if gi.size:
        g = dirichlet_values(geo, bc)
        dx = np.concatenate([dx, geo.xf[gf] - geo.cen[gi]])
        du = np.concatenate([du, g[gf] - u[gi]])
        i = np.concatenate([i, gi])
        w = np.concatenate([w, gw])
    N = geo.n_cell
    M = np.zeros((N, d, d))
    J = np.zeros((N, d))
    for a in range(d):
        J[:, a] = np.bincount(i, weights=w * dx[:, a] * du, minlength=N)
        for b in range(d):
            M[:, a, b] = np.bincount(i, weights=w * dx[:, a] * dx[:, b], minlength=N)
    return np.linalg.solve(M, J[:, :, None])[:, :, 0]


def vertex_weights(geo):
    """Least-squares interpolation weights alpha_{A,c} (Algorithm "ls") for every
    (vertex A, cell c around A) pair, ignoring boundary conditions.

    Returns (A, c, alpha) sorted by (A, c).
    """
    d = geo.dim
    A = geo.cells.ravel().astype(np.int64)
    c = np.repeat(np.arange(geo.n_cell), d + 1)
    o = np.lexsort((c, A))
    A, c = A[o], c[o]
    V = geo.n_vert
    n = np.bincount(A, minlength=V).astype(np.float64)
    dx = geo.cen[c] - geo.xyz[A]
    r = np.concatenate([np.ones((A.size, 1)), dx], axis=1)          # rows [1, x_c - x_A]
    XtX = np.zeros((V, d + 1, d + 1))
    for a in range(d + 1):
        for b in range(d + 1):
            XtX[:, a, b] = np.bincount(A, weights=r[:, a] * r[:, b], minlength=V)
    # centred scatter of the cell centres around A: sum dx dx^T - n xbar xbar^T
    s1 = XtX[:, 0, 1:]
    C = XtX[:, 1:, 1:] - s1[:, :, None] * s1[:, None, :] / np.maximum(n, 1.0)[:, None, None]
    tr = np.trace(C, axis1=1, axis2=2)
    with np.errstate(divide="ignore", invalid="ignore"):
        ratio = np.linalg.det(C) / (tr / d) ** d
    degenerate = (n < d + 1) | ~(ratio >= DEGENERATE_RATIO)
    XtX[degenerate] = np.eye(d + 1)                                   # placeholder, unused
    e1 = np.zeros((V, d + 1, 1)); e1[:, 0, 0] = 1.0
    y = np.linalg.solve(XtX, e1)[:, :, 0]                             # (X^T X)^{-1} e1
    alpha = np.einsum("pk,pk->p", r, y[A])
    alpha = np.where(degenerate[A], 1.0 / n[A], alpha)
    return A, c, alpha


def dirichlet_vertices(geo, bc):
    """(mask[V], value[V]): vertices on a Dirichlet face and their boundary value
    (smallest Dirichlet tag wins at a shared vertex)."""
    mask = np.zeros(geo.n_vert, dtype=bool)
    val = np.zeros(geo.n_vert)
    for t in sorted(bc.keys(), reverse=True):
        kind, v = bc[t]
        if kind != "dirichlet":
            continue
        f = (geo.face_R < 0) & (geo.face_tag == t)
        vv = np.unique(geo.face_vert[f].ravel())
        mask[vv] = True
        val[vv] = float(v)
    return mask, val


def vertex_values(geo, bc, u, weights=None):
    """u_A of Algorithm "ls" at every vertex; Dirichlet vertices take g."""
    A, c, alpha = weights if weights is not None else vertex_weights(geo)
    uv = np.bincount(A, weights=alpha * np.asarray(u, dtype=np.float64)[c], minlength=geo.n_vert)
    mask, val = dirichlet_vertices(geo, bc)
    uv[mask] = val[mask]
    return uv
