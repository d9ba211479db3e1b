"""The sub-mesh helper used by the full-size GPU checks: the oracle evaluated on the
patch around sampled cells gives those cells' streamer update, field and gradient as
on the whole mesh (CPU only)."""
import numpy as np

from oracle import ls, streamer
from synth.meshgen import gaussian, jittered_cube
from tests.conftest import geometry_of
from tests.patch import patch


def test_patch_reproduces_whole_mesh_values():
    m = jittered_cube(8, seed=201)
    g = geometry_of(m)
    p = streamer.Params(sigma=0.15, peak=1e13)
    rng = np.random.default_rng(9)
    ne = gaussian(g.cen, p.centre, p.sigma, p.peak, p.background)
    ni = ne * (1.0 + 0.1 * rng.random(g.n_cell))
    phi = p.V * g.cen[:, 2] + 300.0 * np.sin(5.0 * g.cen[:, 0]) * np.cos(4.0 * g.cen[:, 1])
    dt = 1e-9
    one, oni, _, oE, _ = streamer.step(g, p, ne, ni, dt, phi=phi)
    # sample: random cells plus cells on the Dirichlet planes and a corner
    z = g.cen[:, 2]
    sample = np.unique(np.concatenate([rng.choice(g.n_cell, 40, replace=False),
                                       [int(np.argmin(z)), int(np.argmax(z)),
                                        int(np.argmin(g.cen.sum(axis=1)))]]))
    sub, ids, pos = patch(m, sample)
    assert sub.n_cell < g.n_cell
    # the cut faces carry tag 1: Neumann for phi and for n_e, so they add no ghost point
    assert streamer.bc_phi(p)[1][0] == "neumann" and streamer.bc_ne()[1][0] == "neumann"
    gs = geometry_of(sub)
    sne, sni, _, sE, _ = streamer.step(gs, p, ne[ids], ni[ids], dt, phi=phi[ids])
    np.testing.assert_allclose(sne[pos], one[sample], rtol=1e-13)
    np.testing.assert_allclose(sni[pos], oni[sample], rtol=1e-13)
    np.testing.assert_allclose(sE[pos], oE[sample], rtol=1e-11, atol=1e-9 * np.abs(oE).max())
    # the gradient is exact on the first ring too (it feeds the face velocities)
    ring = np.unique(np.concatenate([ids[pos]]))
    gfull = ls.ls_gradient(g, streamer.bc_phi(p), phi)
    gsub = ls.ls_gradient(gs, streamer.bc_phi(p), phi[ids])
    np.testing.assert_allclose(gsub[pos], gfull[ring], rtol=1e-11, atol=1e-9 * np.abs(gfull).max())
    # and a cut that is too small is seen: one ring loses the neighbours' fields
    sub1, ids1, pos1 = patch(m, sample, rings=1)
    g1 = geometry_of(sub1)
    s1, _, _, _, _ = streamer.step(g1, p, ne[ids1], ni[ids1], dt, phi=phi[ids1])
    assert np.abs(s1[pos1] - one[sample]).max() > 1e-9 * np.abs(one[sample] - ne[sample]).max()
