"""Pins of the oracle's MUSCL reconstruction with the Barth-Jespersen limiter (eq. 15),
checked against properties that do not reuse its formulas:

* the limiter is the largest scaling psi in [0, 1] of the gradient increment that keeps
  every face value of the cell inside the bounds of its face neighbours (found here by
  bisection, with the bounds collected face by face in a plain loop);
* at a strict local extremum the reconstruction is switched off (psi = 0);
* for a linear field, wherever the limiter is inactive, the convective residual is the
  exact divergence -V . b (the reconstruction is exact at the face centroids) - which
  first-order upwind is not;
* conservation with walls and a steady constant state;
* second-order convergence on a translating, spreading Gaussian, where first-order
  upwind converges at order < 1.
"""
import numpy as np
import pytest

from oracle import fv, ls
from synth.meshgen import gaussian, jittered_cube, jittered_square
from tests.conftest import geometry_of

MIXED3 = {1: ("wall", 0.0), 2: ("neumann", 0.0), 3: ("neumann", 0.0), 4: ("wall", 0.0),
          5: ("dirichlet", 0.25), 6: ("dirichlet", 1.5)}
MIXED2 = {1: ("dirichlet", 0.3), 2: ("neumann", 0.0), 3: ("wall", 0.0), 4: ("dirichlet", 1.0)}
WALLS2 = {t: ("wall", 0.0) for t in range(1, 5)}


def _faces_of(g):
    faces = [[] for _ in range(g.n_cell)]
    for f in range(g.n_face):
        faces[g.face_L[f]].append(f)
        if g.face_R[f] >= 0:
            faces[g.face_R[f]].append(f)
    return faces


def _bounds(g, bc, u, faces):
    """(umin, umax) per cell, face by face: the cell, its face neighbours, the Dirichlet
    values of its boundary faces."""
    gval = {t: v for t, (k, v) in bc.items() if k == "dirichlet"}
    lo, hi = u.copy(), u.copy()
    for i, fl in enumerate(faces):
        vals = [u[i]]
        for f in fl:
            if g.face_R[f] >= 0:
                vals.append(u[g.face_R[f]] if g.face_L[f] == i else u[g.face_L[f]])
            elif g.face_tag[f] in gval:
                vals.append(gval[g.face_tag[f]])
        lo[i], hi[i] = min(vals), max(vals)
    return lo, hi


@pytest.mark.parametrize("dim", [2, 3])
def test_limiter_is_the_largest_bounded_scaling(dim):
    m = jittered_cube(4, seed=11) if dim == 3 else jittered_square(12, 5, 6)
    bc = MIXED3 if dim == 3 else MIXED2
    g = geometry_of(m)
    rng = np.random.default_rng(dim)
    u = np.sin(3.0 * g.cen @ rng.uniform(1, 2, size=dim)) + 0.4 * rng.normal(size=g.n_cell)
    grad = ls.ls_gradient(g, bc, u)
    psi = fv.bj_limiter(g, bc, u, grad)
    faces = _faces_of(g)
    lo, hi = _bounds(g, bc, u, faces)
    for i in range(g.n_cell):
        d = np.array([grad[i] @ (g.xf[f] - g.cen[i]) for f in faces[i]])

        def ok(p):
            v = u[i] + p * d
            return bool(np.all(v <= hi[i]) and np.all(v >= lo[i]))

        if ok(1.0):
            want = 1.0
        else:
            a, b = 0.0, 1.0
            for _ in range(60):
                c = 0.5 * (a + b)
                a, b = (c, b) if ok(c) else (a, c)
            want = a
        # equal up to the rounding of u_i + psi d_f at the active bound
        assert abs(psi[i] - want) <= 1e-11, (i, psi[i], want)
    assert 0.0 <= psi.min() and psi.max() <= 1.0
    assert (psi < 1.0).mean() > 0.2            # the test exercises the limiter
    # the reconstructed face states stay inside their cell's bounds
    uLf, uRf, _ = fv.muscl_states(g, bc, u, grad)
    tol = 1e-13 * np.abs(u).max()
    assert np.all(uLf <= hi[g.face_L] + tol) and np.all(uLf >= lo[g.face_L] - tol)
    inr = g.face_R >= 0
    assert np.all(uRf[inr] <= hi[g.face_R[inr]] + tol) and np.all(uRf[inr] >= lo[g.face_R[inr]] - tol)


def test_limiter_switches_off_at_a_strict_extremum():
    g = geometry_of(jittered_cube(4, seed=12))
    bc = {t: ("neumann", 0.0) for t in range(1, 7)}
    u = np.zeros(g.n_cell)
    k = int(np.argmin(np.linalg.norm(g.cen - 0.5, axis=1)))
    u[k] = 1.0
    grad = ls.ls_gradient(g, bc, u)
    assert np.linalg.norm(grad[k]) > 0.0
    assert fv.bj_limiter(g, bc, u, grad)[k] == 0.0


@pytest.mark.parametrize("dim", [2, 3])
def test_linear_field_divergence_is_exact_where_unlimited(dim):
    m = jittered_cube(6, seed=3) if dim == 3 else jittered_square(20, 1, 2)
    g = geometry_of(m)
    bc = {t: ("neumann", 0.0) for t in range(1, 2 * dim + 1)}
    b = np.arange(1, dim + 1) * 0.7
    u = 0.5 + g.cen @ b
    V = np.linspace(0.3, 0.9, dim)
    psi = fv.bj_limiter(g, bc, u, ls.ls_gradient(g, bc, u))
    L, R = g.face_L, g.face_R
    inr = R >= 0
    on_boundary = np.zeros(g.n_cell, dtype=bool)
    on_boundary[L[~inr]] = True
    unlimited = psi == 1.0
    nb = unlimited.copy()
    np.logical_and.at(nb, L[inr], unlimited[R[inr]])
    np.logical_and.at(nb, R[inr], unlimited[L[inr]])
    sel = ~on_boundary & nb
    assert sel.mean() > 0.3
    res = fv.residual(g, bc, u, V, 0.0, recon=1)
    assert np.abs(res[sel] + V @ b).max() <= 1e-12 * abs(V @ b)
    up = fv.residual(g, bc, u, V, 0.0, recon=0)
    assert np.abs(up[sel] + V @ b).max() > 1e-2 * abs(V @ b)


def test_conservation_with_walls_and_constant_state():
    g = geometry_of(jittered_square(16, 7, 8))
    rng = np.random.default_rng(5)
    u0 = 1.0 + rng.random(g.n_cell)
    vel = rng.normal(size=(g.n_cell, 2))
    u = u0.copy()
    for _ in range(20):
        u = fv.rk_step(g, WALLS2, u, vel, 0.01, 2e-3, recon=1)
    assert abs(fv.mass(g, u) - fv.mass(g, u0)) <= 1e-13 * fv.mass(g, u0)
    # a constant state under a constant velocity with open (Neumann) sides is steady
    neu = {t: ("neumann", 0.0) for t in range(1, 5)}
    const = np.full(g.n_cell, 2.5)
    assert np.abs(fv.residual(g, neu, const, np.array([0.4, -0.2]), 0.03, recon=1)).max() < 1e-12


def _gauss_error(n, recon):
    g = geometry_of(jittered_square(n, 101, 102))
    vel = np.array([1.0, 0.5]); D = 0.01; sig = 0.05; x0 = np.array([0.3, 0.3])
    u = gaussian(g.cen, x0, sig)
    dt = fv.cfl_dt(g, WALLS2, vel, D, 0.4)
    coef = fv.diamond_coefficients(g); w = ls.vertex_weights(g)
    T = 0.12
    nsteps = int(round(T / dt)); dt = T / nsteps
    for _ in range(nsteps):
        u = fv.rk_step(g, WALLS2, u, vel, D, dt, coef=coef, weights=w, recon=recon)
    s2 = sig ** 2 + 4 * D * T
    exact = (sig ** 2 / s2) * np.exp(-((g.cen - x0 - vel * T) ** 2).sum(1) / s2)
    return np.sqrt((g.vol * (u - exact) ** 2).sum() / (g.vol * exact ** 2).sum())


@pytest.mark.slow
def test_second_order_on_a_translating_gaussian():
    e = [_gauss_error(n, 1) for n in (25, 50)]
    e_up = _gauss_error(50, 0)
    order = np.log2(e[0] / e[1])
    assert order > 1.7, (e, order)
    assert e[1] < 0.3 * e_up, (e, e_up)
