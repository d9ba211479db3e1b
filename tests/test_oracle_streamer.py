"""Pins for the oracle's streamer step (eq. 10) (CPU)."""
import numpy as np

from synth.meshgen import jittered_cube, gaussian
from oracle import streamer, poisson, fv
from tests.conftest import geometry_of


def _setup(k=5):
    g = geometry_of(jittered_cube(k, seed=201))
    p = streamer.Params(sigma=0.15, peak=1e12, background=1e9)
    ne = gaussian(g.cen, p.centre, p.sigma, p.peak, p.background)
    return g, p, ne


def test_charge_balance():
    """Sources cancel in n_i - n_e, so the total charge changes by exactly dt times
    the net n_e outflow through the (Neumann) boundary."""
    g, p, ne = _setup()
    ni = ne * 1.01
    dt = 1e-9
    ne1, ni1, phi, E, S = streamer.step(g, p, ne, ni, dt)
    v = -p.mu * E
    dq = fv.mass(g, ni1 - ne1) - fv.mass(g, ni - ne)
    want = dt * streamer.boundary_outflow(g, p, ne, v)
    assert abs(dq - want) <= 1e-12 * fv.mass(g, ne)
    assert np.all(S >= 0.0)


def test_neutral_start_gives_applied_field():
    """With n_i = n_e the potential is the linear V z and E = (0, 0, -V)."""
    g, p, ne = _setup(4)
    phi = poisson.solve(g, streamer.bc_phi(p), streamer.poisson_source(ne, ne))
    assert np.abs(phi - p.V * g.cen[:, 2]).max() < 1e-9 * p.V
    _, _, _, E, S = streamer.step(g, p, ne, ne.copy(), 1e-10)
    assert np.abs(E - np.array([0.0, 0.0, -p.V])).max() < 1e-8 * p.V
    alpha = p.A * np.exp(-p.B / p.V)
    assert np.allclose(S, alpha * p.mu * p.V * ne, rtol=1e-9)


def test_no_field_reduces_to_diffusion():
    g, p, ne = _setup(4)
    p.V = 0.0
    ne1, ni1, phi, E, S = streamer.step(g, p, ne, ne.copy(), 1e-7)
    assert np.abs(E).max() < 1e-20 and np.all(S == 0.0)
    want = ne + 1e-7 * fv.residual(g, streamer.bc_ne(), ne, np.zeros(3), p.De)
    assert np.allclose(ne1, want, rtol=1e-14)


RK3 = (0.5, 0.5, 1.0)


def test_three_stage_step_without_field_is_the_transport_rk3():
    """With zero mobility (no drift, no ionisation source) the eq. 6 stages of the streamer
    step are those of the transport step, pinned against its stage polynomial."""
    g, p, ne = _setup(4)
    p.V, p.mu = 0.0, 0.0
    ne1, ni1, phi, E, S = streamer.step(g, p, ne, ne.copy(), 1e-7, alphas=RK3)
    want = fv.rk_step(g, streamer.bc_ne(), ne, np.zeros(3), p.De, 1e-7, alphas=RK3)
    assert np.allclose(ne1, want, rtol=1e-14) and np.array_equal(ni1, ne)


def test_three_stage_charge_balance():
    """The last stage updates from the step's start with alpha = 1 and the field solved from
    the stage-2 densities, so the total charge changes by exactly dt times the n_e outflow
    of the stage-2 state under that field."""
    g, p, ne = _setup()
    ni = ne * 1.01
    dt = 1e-9
    ne2, ni2, _, _, _ = streamer.step(g, p, ne, ni, dt, alphas=RK3[:2])
    ne3, ni3, phi3, E3, S3 = streamer.step(g, p, ne, ni, dt, alphas=RK3)
    dq = fv.mass(g, ni3 - ne3) - fv.mass(g, ni - ne)
    want = dt * streamer.boundary_outflow(g, p, ne2, -p.mu * E3)
    assert abs(dq - want) <= 1e-12 * fv.mass(g, ne)
    # and phi3 solves Poisson for the stage-2 charge (one solve per stage)
    assert poisson.relative_residual(g, streamer.bc_phi(p), streamer.poisson_source(ne2, ni2), phi3) < 1e-10
    # the stages differ from one Euler step
    ne_e, _, _, _, _ = streamer.step(g, p, ne, ni, dt)
    assert np.abs(ne_e - ne3).max() > 1e-6 * np.abs(ne3 - ne).max()


# ---- plasma spots (Section 4, "Streamer Branching") -------------------------------------

def test_spot_gaussian_matches_its_closed_form_integral():
    """Summed over the cells, mu_i exp(-|x_i - c|^2 / sigma^2) is the Gaussian's integral
    pi^(3/2) sigma^3 (resolved spot well inside the cube); exp(-r^2 / (2 sigma^2)) or a
    positive exponent would be far off."""
    g = geometry_of(jittered_cube(16, seed=203))
    sp = streamer.Spot((0.5, 0.5, 0.5), amplitude=3.0, sigma=0.15, t_on=0.0, duration=1.0)
    S = streamer.spot_source(g, [sp], 0.25, 0.5)
    total = fv.mass(g, S)
    assert abs(total / (3.0 * np.pi ** 1.5 * 0.15 ** 3) - 1.0) < 2e-3


def test_spot_window_deposits_its_exact_total():
    """Without ionisation (A = 0) the ion total grows only by the spots: after a run of
    unevenly long steps that covers both windows, by exactly sum_k S_k duration_k
    sum_i mu_i g_k(x_i) (to round-off), and steps outside the windows add nothing."""
    g, p, ne = _setup(5)
    p.A = 0.0
    spots = [streamer.Spot((0.55, 0.5, 0.8), amplitude=2e20, sigma=0.2, t_on=3e-10, duration=4e-10),
             streamer.Spot((0.45, 0.5, 0.78), amplitude=1e20, sigma=0.25, t_on=5e-10, duration=1e-10)]
    ni = ne.copy()
    ni0 = ni.copy()
    t = 0.0
    dts = [1e-10, 2.5e-10, 0.7e-10, 3e-10, 1.3e-10, 2e-10]
    phi = None
    for dt in dts:
        before = ni.copy()
        ne, ni, phi, E, S = streamer.step(g, p, ne, ni, dt, spots=spots, t=t)
        if t + dt <= 3e-10 or t >= 8e-10:
            assert np.array_equal(ni, before)
        t += dt
    assert t > 8e-10
    want = sum(s.amplitude * s.duration * fv.mass(g, np.exp(-((g.cen - s.centre) ** 2).sum(1) / s.sigma ** 2))
               for s in spots)
    got = fv.mass(g, ni) - fv.mass(g, ni0)
    assert abs(got - want) <= 1e-12 * want


def test_spot_keeps_charge_balance():
    """The spot adds electron-ion pairs: n_i - n_e still changes by exactly dt times the
    n_e outflow through the boundary."""
    g, p, ne = _setup()
    ni = ne * 1.01
    dt = 1e-9
    sp = streamer.Spot((0.5, 0.5, 0.7), amplitude=1e22, sigma=0.1, t_on=0.0, duration=1.0)
    ne1, ni1, phi, E, S = streamer.step(g, p, ne, ni, dt, spots=[sp], t=0.0)
    dq = fv.mass(g, ni1 - ne1) - fv.mass(g, ni - ne)
    want = dt * streamer.boundary_outflow(g, p, ne, -p.mu * E)
    assert abs(dq - want) <= 1e-12 * fv.mass(g, ne1)
    assert fv.mass(g, ni1) - fv.mass(g, ni) > 0.5 * dt * 1e22 * np.pi ** 1.5 * 0.1 ** 3
