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
