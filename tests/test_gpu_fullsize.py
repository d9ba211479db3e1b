"""Parity at the full workload sizes, in the launch configurations the benchmark times.

* 750,000 cells (50^3 x 6 tets, FP64 plain method): every cell against the oracle for
  the LS gradient, the vertex values, the transport residual and the Poisson operator
  and right-hand side (relative L2 <= 1e-12); then one streamer step after three
  warm-up steps: the oracle's FP64 residual of the GPU potential <= 1e-8, and the
  oracle's transport driven by that potential gives n_e, n_i and E within 1e-12.
* 6,000,000 cells (100^3 x 6 tets, mixed precision, autotuned launch shapes): the
  oracle's residual of the GPU potential over the whole mesh <= 1e-8, and n_e, n_i and
  E on 256 sampled cells, each from the oracle on the patch of cells it depends on,
  within 1e-5.
* the MUSCL + Barth-Jespersen residual: every cell at 750k (FP64), 256 sampled cells at
  6M (FP32).
* the 64-mesh ensemble (about 15.4M cells, mixed precision, graph mode, extrapolated
  start): the same two checks on its smallest, a middle and its largest mesh.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import fv, ls, poisson, streamer  # noqa: E402
from synth.workloads import StreamerCase, streamer_mesh  # noqa: E402
from tests.conftest import geometry_of  # noqa: E402
from tests.patch import patch  # noqa: E402

TOL64, TOL32 = 1e-12, 1e-5


def rel(a, b):
    a, b = np.ravel(np.asarray(a, dtype=np.float64)), np.ravel(np.asarray(b, dtype=np.float64))
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_00925_gb300 import build
    build.build()
    from paper_2203_00925_gb300 import capi, device
    return capi, device


@pytest.fixture(scope="module")
def w750():
    mesh = streamer_mesh(50, 201)
    return mesh, geometry_of(mesh)


def oracle_params(case):
    return streamer.Params(V=case.V, mu=case.mu, A=case.A, B=case.B, De=case.De,
                           centre=case.centre, sigma=case.sigma, peak=case.peak,
                           background=case.background)


def bench_solve(capi, prec):
    return capi.solve_opts(rtol=1e-8, inner_rtol=0.2,
                           prec=capi.FVGB_FP64 if prec == "fp64" else capi.FVGB_FP32)


def test_operators_750k(dev, w750):
    capi, device = dev
    mesh, g = w750
    case = StreamerCase()
    bcs = [case.bc_ne(), case.bc_phi()]
    dm = device.DeviceMesh(mesh, bcs, prec="fp64")
    rng = np.random.default_rng(750)
    u = np.sin(g.cen @ np.array([2.1, 1.3, 2.9])) + 0.3 * rng.normal(size=g.n_cell)
    ud = dm.to_device(u)
    gd = dm.empty(3, dm.n_cell)
    capi.fvgb_gradient(dm.handle, 1, ud, gd)
    uvd = dm.empty(dm.n_vert)
    capi.fvgb_vertex_values(dm.handle, 1, ud, uvd)
    torch.cuda.synchronize()
    w = ls.vertex_weights(g)
    assert rel(dm.to_host(gd).T, ls.ls_gradient(g, bcs[1], u)) < TOL64
    capi.fvgb_gradient_vertex(dm.handle, 1, ud, gd)
    torch.cuda.synchronize()
    assert rel(dm.to_host(gd).T, ls.ls_gradient_vertex(g, bcs[1], u)) < TOL64
    assert rel(dm.vert_to_host(uvd), ls.vertex_values(g, bcs[1], u, weights=w)) < TOL64
    coef = fv.diamond_coefficients(g)
    vel = rng.normal(size=(g.n_cell, 3))
    src = rng.normal(size=g.n_cell)
    res = dm.empty(dm.n_cell)
    capi.fvgb_fv_residual(dm.handle, capi.tcoef(vel=dm.to_device(vel.T), diff=0.1,
                                                 src=dm.to_device(src), bcset=0), ud, res)
    torch.cuda.synchronize()
    want = fv.residual(g, bcs[0], u, vel, 0.1, src=src, coef=coef, weights=w)
    assert rel(dm.to_host(res), want) < TOL64
    # MUSCL + Barth-Jespersen (eq. 15)
    capi.fvgb_fv_residual(dm.handle, capi.tcoef(vel=dm.to_device(vel.T), diff=0.1,
                                                src=dm.to_device(src), bcset=0, recon=1), ud, res)
    torch.cuda.synchronize()
    want = fv.residual(g, bcs[0], u, vel, 0.1, src=src, coef=coef, weights=w, recon=1)
    assert rel(dm.to_host(res), want) < TOL64
    y = dm.empty(dm.n_cell, dtype=torch.float64)
    b = dm.empty(dm.n_cell, dtype=torch.float64)
    capi.fvgb_poisson_apply(dm.handle, 1, dm.to_device(u, torch.float64), y)
    capi.fvgb_poisson_rhs(dm.handle, 1, dm.to_device(src, torch.float64), b)
    torch.cuda.synchronize()
    assert rel(dm.to_host(y), poisson.apply(g, bcs[1], u, coef=coef, weights=w)) < TOL64
    assert rel(dm.to_host(b), poisson.rhs(g, bcs[1], src, coef=coef, weights=w)) < TOL64
    dm.free()


def test_streamer_step_750k_fp64(dev, w750):
    capi, device = dev
    mesh, g = w750
    case = StreamerCase()
    p = oracle_params(case)
    dm = device.DeviceMesh(mesh, [case.bc_ne(), case.bc_phi()], prec="fp64")
    dt = case.dt(1.0 / 50)
    sp = capi.streamer_params(mu=case.mu, A=case.A, B=case.B, De=case.De, dt=dt,
                              solve=bench_solve(capi, "fp64"))
    ne0, ni0 = case.initial(mesh)
    ne, ni = dm.to_device(ne0), dm.to_device(ni0)
    phi = torch.zeros(dm.n_cell, dtype=torch.float64, device="cuda")
    capi.fvgb_streamer_step(dm.handle, sp, ne, ni, phi, None, 3)
    torch.cuda.synchronize()
    ne_h, ni_h = dm.to_host(ne), dm.to_host(ni)
    E = dm.empty(3, dm.n_cell)
    info = capi.fvgb_streamer_step(dm.handle, sp, ne, ni, phi, E, 1)[0]
    torch.cuda.synchronize()
    phi_h = dm.to_host(phi)
    assert info["rel_res"] <= 1e-8
    f = streamer.poisson_source(ne_h, ni_h)
    assert poisson.relative_residual(g, streamer.bc_phi(p), f, phi_h) <= 1.01e-8
    one, oni, _, oE, _ = streamer.step(g, p, ne_h, ni_h, dt, phi=phi_h)
    got_ne, got_ni = dm.to_host(ne), dm.to_host(ni)
    assert rel(got_ne, one) < TOL64
    assert rel(got_ni, oni) < TOL64
    assert rel(dm.to_host(E).T, oE) < TOL64
    # the increments themselves (n^{k+1} - n^k loses the digits the state shares)
    assert rel(got_ne - ne_h, one - ne_h) < 1e-9
    assert rel(got_ni - ni_h, oni - ni_h) < 1e-9
    dm.free()


def test_streamer_step_6m_mixed_sampled(dev):
    capi, device = dev
    mesh = streamer_mesh(100, 301)
    case = StreamerCase()
    p = oracle_params(case)
    dm = device.DeviceMesh(mesh, [case.bc_ne(), case.bc_phi()], prec="mixed")
    capi.fvgb_autotune(dm.handle)
    dt = case.dt(1.0 / 100)
    sp = capi.streamer_params(mu=case.mu, A=case.A, B=case.B, De=case.De, dt=dt,
                              solve=bench_solve(capi, "mixed"))
    ne0, ni0 = case.initial(mesh)
    ne, ni = dm.to_device(ne0), dm.to_device(ni0)
    phi = torch.zeros(dm.n_cell, dtype=torch.float64, device="cuda")
    capi.fvgb_streamer_step(dm.handle, sp, ne, ni, phi, None, 2)
    torch.cuda.synchronize()
    ne_h = dm.to_host(ne).astype(np.float64)
    ni_h = dm.to_host(ni).astype(np.float64)
    E = dm.empty(3, dm.n_cell)
    info = capi.fvgb_streamer_step(dm.handle, sp, ne, ni, phi, E, 1)[0]
    torch.cuda.synchronize()
    phi_h = dm.to_host(phi)
    got_ne, got_ni, got_E = dm.to_host(ne), dm.to_host(ni), dm.to_host(E).T
    dm.free()
    assert info["rel_res"] <= 1e-8
    g = geometry_of(mesh)
    f = streamer.poisson_source(ne_h, ni_h)
    assert poisson.relative_residual(g, streamer.bc_phi(p), f, phi_h) <= 1.01e-8
    del g
    rng = np.random.default_rng(6000)
    # half uniform, half from the seed's neighbourhood (where n_e and E vary most)
    near = np.flatnonzero(np.linalg.norm(mesh.vertex_mean() - np.array(case.centre), axis=1) < 0.05)
    sample = np.unique(np.concatenate([rng.choice(mesh.n_cell, 128, replace=False),
                                       rng.choice(near, 128, replace=False)]))
    sub, ids, pos = patch(mesh, sample)
    gs = geometry_of(sub)
    sne, sni, _, sE, _ = streamer.step(gs, p, ne_h[ids], ni_h[ids], dt, phi=phi_h[ids])
    assert rel(got_ne[sample], sne[pos]) < TOL32
    assert rel(got_ni[sample], sni[pos]) < TOL32
    assert rel(got_E[sample], sE[pos]) < TOL32


def test_muscl_residual_6m_fp32_sampled(dev):
    """MUSCL residual at 6M cells in FP32 (autotuned shapes), 256 sampled cells against the
    oracle on the patches they depend on (two node-neighbour rings: the limited gradients
    of the face neighbours), within 1e-5."""
    capi, device = dev
    mesh = streamer_mesh(100, 301)
    case = StreamerCase()
    dm = device.DeviceMesh(mesh, [case.bc_ne(), case.bc_phi()], prec="fp32")
    capi.fvgb_autotune(dm.handle)
    rng = np.random.default_rng(6001)
    cen = mesh.vertex_mean()
    u = np.sin(cen @ np.array([5.1, 3.3, 4.9])) + 0.2 * rng.normal(size=mesh.n_cell) + 2.0
    vel = rng.normal(size=(mesh.n_cell, 3))
    src = rng.normal(size=mesh.n_cell)
    res = dm.empty(dm.n_cell)
    capi.fvgb_fv_residual(dm.handle, capi.tcoef(vel=dm.to_device(vel.T), diff=0.1,
                                                src=dm.to_device(src), bcset=0, recon=1),
                          dm.to_device(u), res)
    torch.cuda.synchronize()
    got = dm.to_host(res)
    dm.free()
    sample = np.unique(rng.choice(mesh.n_cell, 256, replace=False))
    sub, ids, pos = patch(mesh, sample, rings=2)
    gs = geometry_of(sub)
    want = fv.residual(gs, case.bc_ne(), u[ids], vel[ids], 0.1, src=src[ids], recon=1)
    assert rel(got[sample], want[pos]) < TOL32


def test_ensemble_64_meshes_sampled(dev):
    """The 64-mesh ensemble (about 15.4M cells) as the benchmark runs it: mixed precision,
    autotuned launch shapes, graph mode, extrapolated start. After three steps, on the
    smallest, a middle and the largest mesh: the oracle's residual of that part's potential
    (whole part) <= 1e-8, and n_e, n_i, E on sampled cells from the oracle on patches
    within 1e-5. Every part's own relative residual <= 1e-8."""
    capi, device = dev
    from synth.workloads import ensemble_cases
    cases = ensemble_cases(64, seed=5000)
    meshes = [streamer_mesh(k, seed) for k, seed, _ in cases]
    dm = device.DeviceMesh(meshes, [[c.bc_ne(), c.bc_phi()] for _, _, c in cases], prec="mixed",
                           ensemble=True)
    capi.fvgb_autotune(dm.handle)
    c0 = cases[0][2]
    dt = min(c.dt(1.0 / k) for k, _, c in cases)
    sp = capi.streamer_params(mu=c0.mu, A=c0.A, B=c0.B, De=c0.De, dt=dt, extrapolate=True,
                              solve=bench_solve(capi, "mixed"))
    ne0 = np.concatenate([c.initial(m)[0] for m, (_, _, c) in zip(meshes, cases)])
    ne, ni = dm.to_device(ne0), dm.to_device(ne0)
    phi = torch.zeros(dm.n_cell, dtype=torch.float64, device="cuda")
    capi.fvgb_streamer_reset(dm.handle)
    capi.fvgb_set_graph_mode(dm.handle, True)
    capi.fvgb_streamer_step(dm.handle, sp, ne, ni, phi, None, 2)
    torch.cuda.synchronize()
    ne_h = dm.to_host(ne).astype(np.float64)
    ni_h = dm.to_host(ni).astype(np.float64)
    E = dm.empty(3, dm.n_cell)
    info = capi.fvgb_streamer_step(dm.handle, sp, ne, ni, phi, E, 1)[0]
    torch.cuda.synchronize()
    rel_parts, _, _ = capi.fvgb_solve_parts(dm.handle, dm.n_part)
    phi_h, got_ne, got_ni, got_E = dm.to_host(phi), dm.to_host(ne), dm.to_host(ni), dm.to_host(E).T
    dm.free()
    assert info["rel_res"] <= 1e-8 and np.max(rel_parts) <= 1e-8
    begin = np.concatenate([[0], np.cumsum([m.n_cell for m in meshes])])
    sizes = np.array([m.n_cell for m in meshes])
    order = np.argsort(sizes)
    rng = np.random.default_rng(5064)
    for p in (order[0], order[len(order) // 2], order[-1]):
        m, case = meshes[p], cases[p][2]
        sl = slice(begin[p], begin[p + 1])
        prm = oracle_params(case)
        g = geometry_of(m)
        f = streamer.poisson_source(ne_h[sl], ni_h[sl])
        assert poisson.relative_residual(g, streamer.bc_phi(prm), f, phi_h[sl]) <= 1.01e-8
        del g
        sample = np.unique(rng.choice(m.n_cell, 96, replace=False))
        sub, ids, pos = patch(m, sample)
        gs = geometry_of(sub)
        sne, sni, _, sE, _ = streamer.step(gs, prm, ne_h[sl][ids], ni_h[sl][ids], dt, phi=phi_h[sl][ids])
        assert rel(got_ne[sl][sample], sne[pos]) < TOL32
        assert rel(got_ni[sl][sample], sni[pos]) < TOL32
        assert rel(got_E[sl][sample], sE[pos]) < TOL32
