"""Face fluxes, the semi-discrete residual of eq. 4 and explicit time stepping
(oracle; test infrastructure only).

Readings (shared with the GPU library, which implements them on its own):

* Diamond face gradient (eq. "diamond", D = C for a tetrahedron): with
  e1 = x_R - x_L, e2 = x_A - x_C, e3 = x_B - x_C, grad u_f is the vector with
  grad.e1 = u_R - u_L, grad.e2 = u_A - u_C, grad.e3 = u_B - u_C (the exact-for-linear
  dual-basis form of eq. "diamond"). In 2D, e1 = x_R - x_L, e2 = x_B - x_A. At a
  Dirichlet boundary face R is the face centroid and u_R = g.
* Upwind (eq. 15 with psi = 0): u_f = u_L when V_f.S_f >= 0, else u_R, with
  V_f = (V_L + V_R) / 2 for a cell-centred velocity.
* MUSCL (eq. 15, recon = 1): the upwind side's value is reconstructed,
  u_f = u_c + psi_c grad u_c . (x_f - x_c), with the least-squares gradient of
  Algorithm "grad" (same boundary conditions) and the Barth-Jespersen limiter psi_c
  (see ``bj_limiter``). A boundary ghost on the upwind side keeps its first-order
  value (g on Dirichlet faces, u_L on Neumann faces).
* Boundary kinds: "wall" - no flux at all; "neumann" (homogeneous) - the ghost
  copies the interior (u_R = u_L, V_R = V_L), no diffusive flux; "dirichlet" - the
  ghost value is g, V_R = V_L.
* The face flux F_f = (V_f.S_f) u_f - D grad u_f.S_f leaves L and enters R; eq. 4
  gives R_i = (sum_{f: R(f)=i} F_f - sum_{f: L(f)=i} F_f) / mu_i + S_i.
* Eq. 6 prints u^{n+1} = u^n; the reading is u^(k) = u^n + alpha_k dt Res(u^(k-1)),
  k = 1..3, alpha = (0.5, 0.5, 1), u^{n+1} = u^(3). One stage with alpha = 1 is
  explicit Euler.
"""
from __future__ import annotations

import numpy as np

from . import ls


def diamond_coefficients(geo):
    """c[F, d] with grad u_f . S_f = c1 du1 + c2 du2 (+ c3 du3) for the differences
    du1 = u_R - u_L, du2 = u_A - u_C, du3 = u_B - u_C (2D: du2 = u_B - u_A)."""
    d = geo.dim
    L, R = geo.face_L, geo.face_R
    xR = np.where((R >= 0)[:, None], geo.cen[np.maximum(R, 0)], geo.xf)
    e1 = xR - geo.cen[L]
    P = geo.xyz[geo.face_vert]
    if d == 3:
        G = np.stack([e1, P[:, 0] - P[:, 2], P[:, 1] - P[:, 2]], axis=1)
    else:
        G = np.stack([e1, P[:, 1] - P[:, 0]], axis=1)
    # G grad = du  =>  grad . S = (G^{-T} S) . du
    return np.linalg.solve(np.transpose(G, (0, 2, 1)), geo.S[:, :, None])[:, :, 0]


def _face_value_differences(geo, bc, u, uv):
    """du[F, d] entering diamond_coefficients, with Dirichlet ghosts at boundary faces."""
    d = geo.dim
    L, R = geo.face_L, geo.face_R
    g = ls.dirichlet_values(geo, bc)
    uR = np.where(R >= 0, u[np.maximum(R, 0)], g)
    fvv = uv[geo.face_vert]
    if d == 3:
        return np.stack([uR - u[L], fvv[:, 0] - fvv[:, 2], fvv[:, 1] - fvv[:, 2]], axis=1)
    return np.stack([uR - u[L], fvv[:, 1] - fvv[:, 0]], axis=1)


def face_gradient_flux(geo, bc, u, coef=None, weights=None):
    """q_f = grad u_f . S_f (eq. "diamond") on every face; 0 on wall/Neumann faces."""
    coef = diamond_coefficients(geo) if coef is None else coef
    uv = ls.vertex_values(geo, bc, u, weights)
    du = _face_value_differences(geo, bc, np.asarray(u, dtype=np.float64), uv)
    q = np.einsum("fk,fk->f", coef, du)
    bnd = geo.face_R < 0
    dir_ = np.isin(geo.face_tag, [t for t, (k, _v) in bc.items() if k == "dirichlet"])
    q[bnd & ~dir_] = 0.0
    return q


def face_velocity(geo, vel):
    """V_f: mean of the two cell velocities; the ghost copies the interior."""
    vel = np.asarray(vel, dtype=np.float64)
    if vel.ndim == 1:
        return np.broadcast_to(vel, (geo.n_face, geo.dim))
    L, R = geo.face_L, geo.face_R
    VR = np.where((R >= 0)[:, None], vel[np.maximum(R, 0)], vel[L])
    return 0.5 * (vel[L] + VR)


def bj_limiter(geo, bc, u, grad):
    """Barth-Jespersen limiter psi_i of eq. 15 (the paper names the limiter; this is its
    standard definition, Barth and Jespersen 1989), with these readings of its stencil:

    * bounds u_min_i, u_max_i: over u_i, the values of the cells sharing a face with T_i
      and the boundary values g of T_i's Dirichlet faces (a wall or Neumann face adds
      nothing: its ghost is absent or equals u_i);
    * every face f of T_i (boundary faces included) has the unlimited increment
      d_f = grad u_i . (x_f - x_i) and the ratio phi_f = min(1, (u_max_i - u_i) / d_f)
      if d_f > 0, min(1, (u_min_i - u_i) / d_f) if d_f < 0, and 1 if d_f = 0;
    * psi_i = min over the faces of T_i of phi_f.
    """
    u = np.asarray(u, dtype=np.float64)
    grad = np.asarray(grad, dtype=np.float64)
    L, R = geo.face_L, geo.face_R
    inr = R >= 0
    g = ls.dirichlet_values(geo, bc)
    dirf = np.isfinite(g)
    umax, umin = u.copy(), u.copy()
    for a, b in ((L[inr], u[R[inr]]), (R[inr], u[L[inr]]), (L[dirf], g[dirf])):
        np.maximum.at(umax, a, b)
        np.minimum.at(umin, a, b)
    psi = np.ones(geo.n_cell)
    for cells, keep in ((L, np.ones(geo.n_face, dtype=bool)), (R, inr)):
        c = cells[keep]
        d = np.einsum("fi,fi->f", grad[c], geo.xf[keep] - geo.cen[c])
        phi = np.ones(c.size)
        pos, neg = d > 0.0, d < 0.0
        phi[pos] = np.minimum(1.0, (umax[c[pos]] - u[c[pos]]) / d[pos])
        phi[neg] = np.minimum(1.0, (umin[c[neg]] - u[c[neg]]) / d[neg])
        np.minimum.at(psi, c, phi)
    return psi


def muscl_states(geo, bc, u, grad=None):
    """(u_Lf, u_Rf, psi): the reconstructed values of the two cells of every face,
    u_c + psi_c grad u_c . (x_f - x_c); u_Rf is NaN on boundary faces."""
    u = np.asarray(u, dtype=np.float64)
    grad = ls.ls_gradient(geo, bc, u) if grad is None else np.asarray(grad, dtype=np.float64)
    psi = bj_limiter(geo, bc, u, grad)
    L, R = geo.face_L, geo.face_R
    Rs = np.maximum(R, 0)
    uLf = u[L] + psi[L] * np.einsum("fi,fi->f", grad[L], geo.xf - geo.cen[L])
    uRf = u[Rs] + psi[Rs] * np.einsum("fi,fi->f", grad[Rs], geo.xf - geo.cen[Rs])
    return uLf, np.where(R >= 0, uRf, np.nan), psi


def face_flux(geo, bc, u, vel, D, coef=None, weights=None, recon=0):
    """F_f = (V_f.S_f) u_f - D grad u_f.S_f, oriented L -> R (eq. 4, eq. 15); recon = 1
    takes u_f from the limited MUSCL reconstruction."""
    geo.check_bc(bc)
    u = np.asarray(u, dtype=np.float64)
    L, R = geo.face_L, geo.face_R
    vn = np.einsum("fi,fi->f", face_velocity(geo, vel), geo.S)
    g = ls.dirichlet_values(geo, bc)
    kind = np.array(["interior"] * geo.n_face, dtype=object)
    for t, (k, _v) in bc.items():
        kind[(R < 0) & (geo.face_tag == t)] = k
    ghost = np.where(kind == "dirichlet", g, u[L])
    if recon:
        uLf, uRf, _ = muscl_states(geo, bc, u)
        u_up = np.where(vn >= 0.0, uLf, np.where(R >= 0, uRf, ghost))
    else:
        uR = np.where(R >= 0, u[np.maximum(R, 0)], ghost)
        u_up = np.where(vn >= 0.0, u[L], uR)
    F = vn * u_up
    if D != 0.0:
        F = F - D * face_gradient_flux(geo, bc, u, coef, weights)
    F[kind == "wall"] = 0.0
    return F


def residual(geo, bc, u, vel, D, src=None, coef=None, weights=None, recon=0):
    """R_i of eq. 4: (sum_{R(f)=i} F_f - sum_{L(f)=i} F_f) / mu_i + S_i."""
    F = face_flux(geo, bc, u, vel, D, coef, weights, recon)
    N = geo.n_cell
    inr = geo.face_R >= 0
    acc = np.bincount(geo.face_R[inr], weights=F[inr], minlength=N).astype(np.float64)
    acc -= np.bincount(geo.face_L, weights=F, minlength=N)
    res = acc / geo.vol
    if src is not None:
        res = res + np.asarray(src, dtype=np.float64)
    return res


def rk_step(geo, bc, u, vel, D, dt, alphas=(1.0,), src=None, coef=None, weights=None,
            recon=0):
    """One time step of eq. 6 with stage coefficients ``alphas`` ((1,) = Euler)."""
    un = np.asarray(u, dtype=np.float64)
    uk = un
    for a in alphas:
        uk = un + a * dt * residual(geo, bc, uk, vel, D, src, coef, weights, recon)
    return uk


def cfl_dt(geo, bc, vel, D, cfl, coef=None):
    """dt = cfl * min_i mu_i / sum_{f in i} [max(V_f.S_f out of i, 0) + D |c1_f|]
    (reading of "explicit Euler at CFL 0.4": outflow plus two-point diffusion rate)."""
    coef = diamond_coefficients(geo) if coef is None else coef
    vn = np.einsum("fi,fi->f", face_velocity(geo, vel), geo.S)
    wall = np.isin(geo.face_tag, [t for t, (k, _v) in bc.items() if k == "wall"]) & (geo.face_R < 0)
    dif = D * np.abs(coef[:, 0])
    dif = np.where(wall, 0.0, dif)
    outL = np.where(wall, 0.0, np.maximum(vn, 0.0))
    outR = np.maximum(-vn, 0.0)
    N = geo.n_cell
    inr = geo.face_R >= 0
    rate = np.bincount(geo.face_L, weights=outL + dif, minlength=N)
    rate += np.bincount(geo.face_R[inr], weights=(outR + dif)[inr], minlength=N)
    return cfl * float(np.min(geo.vol / rate))


def mass(geo, u):
    """sum_i mu_i u_i."""
    return float(np.dot(geo.vol, u))
