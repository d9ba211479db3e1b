"""Pins for the oracle's diamond gradient, fluxes, residual and time stepping (CPU)."""
import numpy as np
import pytest

from synth.meshgen import jittered_cube, jittered_square, gaussian
from oracle import fv, ls
from tests.conftest import geometry_of

WALLS_2D = {t: ("wall", 0.0) for t in range(1, 5)}
NEU_3D = {t: ("neumann", 0.0) for t in range(1, 7)}


@pytest.mark.parametrize("dim", [2, 3])
def test_diamond_exact_for_linear(dim):
    """With exact vertex values a linear field gives grad u_f . S_f exactly."""
    m = jittered_cube(4, seed=8) if dim == 3 else jittered_square(8, 3, 4)
    g = geometry_of(m)
    rng = np.random.default_rng(2)
    b = rng.normal(size=dim)
    u = 1.0 + g.cen @ b
    uv = 1.0 + g.xyz @ b
    c = fv.diamond_coefficients(g)
    inr = g.face_R >= 0
    du = fv._face_value_differences(g, NEU_3D if dim == 3 else WALLS_2D, u, uv)
    q = np.einsum("fk,fk->f", c, du)
    assert np.abs(q[inr] - g.S[inr] @ b).max() < 1e-12 * np.abs(b).max()
    # the coefficient of u_R - u_L is |S|^2 / (e1 . S) > 0
    e1 = g.cen[g.face_R[inr]] - g.cen[g.face_L[inr]]
    c1 = (g.S[inr] ** 2).sum(1) / np.einsum("fi,fi->f", e1, g.S[inr])
    assert np.allclose(c[inr, 0], c1, rtol=1e-12)


def test_laplacian_of_linear_vanishes_inside():
    m = jittered_cube(5, seed=4)
    g = geometry_of(m)
    b = np.array([0.4, -1.1, 2.0])
    bc = {1: ("dirichlet", 0.0), 2: ("dirichlet", 0.4)}
    bc.update({t: ("neumann", 0.0) for t in (3, 4, 5, 6)})
    # diffusion-only residual of u = 0.4 x: exact zero flux divergence in cells away
    # from the Neumann sides (where grad u . n = 0 holds for this field too)
    u = 0.4 * g.cen[:, 0]
    r = fv.residual(g, bc, u, np.zeros(3), 1.0)
    assert np.abs(r).max() < 1e-11
    u = g.cen @ b
    r = fv.residual(g, NEU_3D, u, np.zeros(3), 1.0)
    touches_bnd = np.zeros(g.n_cell, bool)
    touches_bnd[g.face_L[g.face_R < 0]] = True
    vb = np.zeros(g.n_vert, bool); vb[g.face_vert[g.face_R < 0].ravel()] = True
    far = ~vb[g.cells].any(axis=1)
    assert far.sum() > 0
    assert np.abs(r[far]).max() < 1e-10


def _config1_like(n=20):
    m = jittered_square(n, 101, 102)
    g = geometry_of(m)
    u0 = gaussian(g.cen, (0.3, 0.3), 0.05)
    return m, g, u0


def test_mass_conserved_with_walls():
    m, g, u0 = _config1_like(20)
    vel = np.array([1.0, 0.5])
    dt = fv.cfl_dt(g, WALLS_2D, vel, 0.01, 0.4)
    u = u0.copy()
    coef = fv.diamond_coefficients(g)
    w = ls.vertex_weights(g)
    for _ in range(50):
        u = fv.rk_step(g, WALLS_2D, u, vel, 0.01, dt, coef=coef, weights=w)
    assert abs(fv.mass(g, u) - fv.mass(g, u0)) <= 1e-13 * abs(fv.mass(g, u0))


def test_constant_state_is_steady():
    m, g, _ = _config1_like(10)
    r = fv.residual(g, WALLS_2D, np.full(g.n_cell, 3.0), np.zeros(2), 0.5)
    assert np.abs(r).max() < 1e-12
    gc = geometry_of(jittered_cube(3, seed=1))
    vel = np.array([0.3, -0.2, 0.1])
    r = fv.residual(gc, NEU_3D, np.full(gc.n_cell, 3.0), vel, 0.5)
    # scale of the flux divergence: convective and diffusive face rates over the volume
    c = fv.diamond_coefficients(gc)
    scale = 3.0 * (np.linalg.norm(vel) * np.linalg.norm(gc.S, axis=1).max()
                   + 0.5 * np.abs(c).max()) / gc.vol.min()
    assert np.abs(r).max() < 1e-12 * scale   # Neumann ghosts carry the same value out and in


def test_upwind_maximum_principle():
    """Pure first-order upwind at CFL <= 1 keeps u within its initial range (each
    update is a convex combination when the ghosts copy the interior); a downwind
    choice (the flipped comparison of eq. 15) breaks this at once."""
    m, g, _ = _config1_like(16)
    neu = {t: ("neumann", 0.0) for t in range(1, 5)}
    rng = np.random.default_rng(0)
    u = rng.uniform(0.0, 1.0, size=g.n_cell)
    vel = np.array([1.0, 0.5])
    dt = fv.cfl_dt(g, neu, vel, 0.0, 0.9)
    for _ in range(20):
        u = fv.rk_step(g, neu, u, vel, 0.0, dt)
        assert u.min() >= -1e-14 and u.max() <= 1.0 + 1e-14


def test_rk3_stage_combination():
    """For a linear operator, the reading of eq. 6 gives
    u^{n+1} = (I + dt L + dt^2 L^2 / 2 + dt^3 L^3 / 4) u^n."""
    gc = geometry_of(jittered_cube(3, seed=2))
    bc = {t: ("dirichlet", 0.0) for t in range(1, 7)}
    rng = np.random.default_rng(4)
    u = rng.normal(size=gc.n_cell)
    dt = 1e-3

    def Lop(x):
        return fv.residual(gc, bc, x, np.zeros(3), 1.0)

    got = fv.rk_step(gc, bc, u, np.zeros(3), 1.0, dt, alphas=(0.5, 0.5, 1.0))
    L1 = Lop(u); L2 = Lop(L1); L3 = Lop(L2)
    want = u + dt * L1 + dt ** 2 / 2 * L2 + dt ** 3 / 4 * L3
    assert np.abs(got - want).max() < 1e-12 * np.abs(u).max()


def _gauss_error(n):
    m = jittered_square(n, 101, 102)
    g = geometry_of(m)
    vel = np.array([1.0, 0.5]); D = 0.01; sig = 0.05; x0 = np.array([0.3, 0.3])
    u = gaussian(g.cen, x0, sig)
    dt = fv.cfl_dt(g, WALLS_2D, vel, D, 0.4)
    coef = fv.diamond_coefficients(g); w = ls.vertex_weights(g)
    T = 0.12                      # bump stays >= 3 sigma_t from the walls
    nsteps = int(round(T / dt)); dt = T / nsteps
    for _ in range(nsteps):
        u = fv.rk_step(g, WALLS_2D, u, vel, D, dt, coef=coef, weights=w)
    s2 = sig ** 2 + 4 * D * T
    exact = (sig ** 2 / s2) * np.exp(-((g.cen - x0 - vel * T) ** 2).sum(1) / s2)
    return np.sqrt((g.vol * (u - exact) ** 2).sum() / (g.vol * exact ** 2).sum())


@pytest.mark.slow
def test_gaussian_advection_diffusion_converges():
    """Translating, spreading Gaussian of constant-coefficient advection-diffusion
    (free-space closed form); first-order upwind -> error falls at >= order ~0.8."""
    e = [_gauss_error(n) for n in (25, 50, 100)]
    assert e[0] > e[1] > e[2]
    orders = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert orders.min() > 0.6, (e, orders)
    assert e[2] < 0.15


def _two_triangles():
    """Unit square cut along its diagonal (0,0)-(1,1): cell 0 = (0,0),(1,0),(1,1) with
    centre (2/3, 1/3), cell 1 = (0,0),(1,1),(0,1) with centre (1/3, 2/3); both have area
    1/2. The interior face has S = (-1, 1) (length sqrt 2, pointing from cell 0 to cell 1);
    the boundary edges have outward area vectors (0,-1) and (1,0) for cell 0, (-1,0) and
    (0,1) for cell 1."""
    from synth.meshgen import Mesh
    xyz = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0]])
    cells = np.array([[0, 1, 3], [0, 3, 2]])
    bf = np.array([[0, 1], [1, 3], [3, 2], [2, 0]])
    tags = np.array([3, 2, 4, 1])
    return geometry_of(Mesh(2, xyz, cells, bf, tags, 1.0))


NEU_2D = {t: ("neumann", 0.0) for t in range(1, 5)}


def test_face_velocity_mean_of_cells_hand_checked():
    """V_f of eq. 4 for a cell-centred velocity (reading R8): the mean of the two cells'
    velocities on interior faces, the interior cell's own velocity on boundary faces.
    The residual is checked against values worked out by hand, so that V_f = V_L,
    V_f = the upwind cell's velocity, or a zero ghost velocity all fail."""
    g = _two_triangles()
    inner = np.nonzero(g.face_R >= 0)[0]
    assert inner.size == 1
    f = inner[0]
    assert (g.face_L[f], g.face_R[f]) == (0, 1)
    assert np.allclose(g.S[f], [-1.0, 1.0])
    vel = np.array([[3.0, 0.0], [0.0, 1.0]])
    Vf = fv.face_velocity(g, vel)
    assert np.allclose(Vf[f], [1.5, 0.5])
    bnd = g.face_R < 0
    assert np.array_equal(Vf[bnd], vel[g.face_L[bnd]])
    # V_f . S = -1 on the interior face: upwind is cell 1 and F = -u_1; cell 0's boundary
    # fluxes are 0 (y = 0) and 3 u_0 (x = 1); cell 1's are 0 (x = 0) and u_1 (y = 1).
    # R_0 = (-F_int - 3 u_0) / (1/2) = 2 u_1 - 6 u_0, R_1 = (F_int - u_1) / (1/2) = -4 u_1.
    u = np.array([2.0, 5.0])
    r = fv.residual(g, NEU_2D, u, vel, 0.0)
    assert np.allclose(r, [2 * 5.0 - 6 * 2.0, -4 * 5.0], rtol=0, atol=1e-13)
    # the misreadings give other numbers: V_f = V_L makes F_int = -3 u_1 (R_0 = 18), V_f =
    # V_upwind (cell 1: V . S = +1, upwind then L) makes F_int = u_0 (R_0 = -16), a zero
    # ghost velocity halves the boundary outflow 3 u_0 (R_0 = 4)
    assert not np.isclose(r[0], 18.0) and not np.isclose(r[0], -16.0) and not np.isclose(r[0], 4.0)


def test_face_velocity_tie_takes_left_and_carries_no_flux():
    """With (V_L + V_R) . S = 0 the interior face carries no convective flux (the tie
    V_f . S >= 0 takes u_L, times zero); V_f = V_L would give -u_1 there instead."""
    g = _two_triangles()
    f = np.nonzero(g.face_R >= 0)[0][0]
    vel = np.array([[1.0, 0.0], [1.0, 2.0]])
    Vf = fv.face_velocity(g, vel)
    assert np.dot(Vf[f], g.S[f]) == 0.0
    u = np.array([2.0, 5.0])
    F = fv.face_flux(g, NEU_2D, u, vel, 0.0)
    assert F[f] == 0.0
    # boundary: cell 0 (V = (1, 0)) has outflow 1 * u_0 at x = 1; cell 1 (V = (1, 2)) has
    # -1 * u_1 at x = 0 and 2 * u_1 at y = 1
    r = fv.residual(g, NEU_2D, u, vel, 0.0)
    assert np.allclose(r, [-2.0 * 2.0, -2.0 * (2.0 * 5.0 - 5.0)], rtol=0, atol=1e-13)
