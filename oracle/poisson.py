"""The diamond-scheme Poisson operator (eq. 7 / eq. "laplace") and a direct solve
(oracle; test infrastructure only).

Row i of the discrete Laplacian integrates the diamond face gradient over the cell
boundary: mu_i (Lap_h P)_i = sum over faces of grad P_f . n |sigma| taken outwards
(eq. 7 multiplied by mu_i). Readings:

* The system is written in integrated form with a positive operator,
  A x = -mu Lap_h(x; g = 0), and Lap P = f becomes A P = b with
  b = -mu f + mu Lap_h(0; g) (the Dirichlet lift). Homogeneous Neumann and wall
  faces carry no flux.
* The relative residual is ||b - A x||_2 / ||b||_2 (relative to the right-hand side
  including the lift, not to the initial residual).
* The paper solves A P = b with MUMPS or FGMRES; the oracle takes the plain
  definition P = A^{-1} b by a sparse direct factorisation (SuperLU), dense LU on
  tiny meshes.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fv, ls


def _zero_bc(bc):
    return {t: (k, 0.0) for t, (k, _v) in bc.items()}


def outward_flux_sum(geo, q):
    """sum_{f: L(f)=i} q_f - sum_{f: R(f)=i} q_f (q oriented L -> R)."""
    N = geo.n_cell
    inr = geo.face_R >= 0
    out = np.bincount(geo.face_L, weights=q, minlength=N)
    out -= np.bincount(geo.face_R[inr], weights=q[inr], minlength=N)
    return out


def apply(geo, bc, x, coef=None, weights=None):
    """A x = -mu Lap_h(x) with homogeneous boundary values (matrix-free)."""
    q = fv.face_gradient_flux(geo, _zero_bc(bc), np.asarray(x, dtype=np.float64), coef, weights)
    return -outward_flux_sum(geo, q)


def rhs(geo, bc, f, coef=None, weights=None):
    """b = -mu f + mu Lap_h(0; g)."""
    q = fv.face_gradient_flux(geo, bc, np.zeros(geo.n_cell), coef, weights)
    return -geo.vol * np.asarray(f, dtype=np.float64) + outward_flux_sum(geo, q)


def assemble(geo, bc, coef=None, weights=None):
    """The sparse matrix of ``apply`` built from its definition by linearity:
    A = (B_R - B_L) Q with Q = c1 (E_R - E_L) + c2 (P_A - P_C) W + c3 (P_B - P_C) W."""
    geo.check_bc(bc)
    coef = fv.diamond_coefficients(geo) if coef is None else coef
    A_v, c_v, alpha = weights if weights is not None else ls.vertex_weights(geo)
    N, V, F, d = geo.n_cell, geo.n_vert, geo.n_face, geo.dim
    dmask, _ = ls.dirichlet_vertices(geo, bc)
    keep = ~dmask[A_v]
    W = sp.csr_matrix((alpha[keep], (A_v[keep], c_v[keep])), shape=(V, N))
    fidx = np.arange(F)
    L, R = geo.face_L, geo.face_R
    inr = R >= 0
    E_L = sp.csr_matrix((np.ones(F), (fidx, L)), shape=(F, N))
    E_R = sp.csr_matrix((np.ones(inr.sum()), (fidx[inr], R[inr])), shape=(F, N))

    def pick(col):
        return sp.csr_matrix((np.ones(F), (fidx, geo.face_vert[:, col])), shape=(F, V))

    if d == 3:
        Q = (sp.diags(coef[:, 0]) @ (E_R - E_L)
             + sp.diags(coef[:, 1]) @ (pick(0) - pick(2)) @ W
             + sp.diags(coef[:, 2]) @ (pick(1) - pick(2)) @ W)
    else:
        Q = (sp.diags(coef[:, 0]) @ (E_R - E_L)
             + sp.diags(coef[:, 1]) @ (pick(1) - pick(0)) @ W)
    dir_tags = [t for t, (k, _v) in bc.items() if k == "dirichlet"]
    live = inr | np.isin(geo.face_tag, dir_tags)
    Q = sp.diags(live.astype(np.float64)) @ Q
    B_L = sp.csr_matrix((np.ones(F), (L, fidx)), shape=(N, F))
    B_R = sp.csr_matrix((np.ones(inr.sum()), (R[inr], fidx[inr])), shape=(N, F))
    return ((B_R - B_L) @ Q).tocsr()


def solve(geo, bc, f, dense=False):
    """P = A^{-1} b, the plain definition of the discrete solution."""
    A = assemble(geo, bc)
    b = rhs(geo, bc, f)
    if dense:
        return np.linalg.solve(A.toarray(), b)
    return spla.spsolve(A.tocsc(), b)


def relative_residual(geo, bc, f, x):
    """||b - A x||_2 / ||b||_2 evaluated in FP64 with the matrix-free operator."""
    b = rhs(geo, bc, f)
    r = b - apply(geo, bc, x)
    return float(np.linalg.norm(r) / np.linalg.norm(b))
