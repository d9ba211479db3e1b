"""Ensembles: several independent meshes packed into one index space and advanced by the
same launches (the batched workload). Each part must give what the part gives alone:
transport bitwise (same per-element arithmetic and order), Poisson solves to the
oracle's direct solution of that part (each part to its own tolerance)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from synth.meshgen import jittered_cube, gaussian  # noqa: E402
from synth.workloads import StreamerCase  # noqa: E402
from oracle import poisson, streamer  # noqa: E402
from tests.conftest import geometry_of  # noqa: E402


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_00925_gb300 import build
    build.build()
    from paper_2203_00925_gb300 import capi, device
    return capi, device


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _ensemble(n=3):
    ks = [4, 6, 5, 7][:n]
    meshes = [jittered_cube(k, seed=5000 + i) for i, k in enumerate(ks)]
    Vs = [15000.0, 25000.0, 19000.0, 21000.0][:n]
    cases = [StreamerCase(V=V, centre=(0.4 + 0.1 * i, 0.5, 0.85), sigma=0.12, peak=1e13) for i, V in enumerate(Vs)]
    return meshes, cases


def test_ensemble_layout_and_transport_bitwise(dev):
    capi, device = dev
    meshes, cases = _ensemble()
    bcs = [[c.bc_ne(), c.bc_phi()] for c in cases]
    ens = device.DeviceMesh(meshes, bcs, ensemble=True)
    assert ens.n_part == 3
    assert list(np.diff(ens.part_begin)) == [m.n_cell for m in meshes]
    rng = np.random.default_rng(1)
    fields = [2.0 + rng.random(m.n_cell) for m in meshes]
    vels = [rng.normal(size=(3, m.n_cell)) for m in meshes]
    u = ens.to_device(np.concatenate(fields))
    vel = ens.to_device(np.concatenate(vels, axis=1))
    tc = capi.tcoef(vel=vel, diff=0.05, bcset=0)
    capi.fvgb_fv_step(ens.handle, tc, u, 1e-4, 3)
    grad_e = ens.empty(3, ens.n_cell)
    capi.fvgb_gradient(ens.handle, 1, u, grad_e)
    torch.cuda.synchronize()
    got = ens.to_host(u)
    got_g = ens.to_host(grad_e)
    off = 0
    for m, bc, f, v in zip(meshes, bcs, fields, vels):
        one = device.DeviceMesh(m, bc)
        u1 = one.to_device(f)
        v1 = one.to_device(v)
        capi.fvgb_fv_step(one.handle, capi.tcoef(vel=v1, diff=0.05, bcset=0), u1, 1e-4, 3)
        g1 = one.empty(3, one.n_cell)
        capi.fvgb_gradient(one.handle, 1, u1, g1)
        torch.cuda.synchronize()
        assert np.array_equal(got[off:off + m.n_cell], one.to_host(u1))
        assert np.array_equal(got_g[:, off:off + m.n_cell], one.to_host(g1))
        off += m.n_cell
        one.free()
    ens.free()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("inner", [0, 2])
def test_ensemble_poisson_parts_converge_independently(dev, prec, inner):
    """Per-part stopping with the CG inner solve (inner = 0) and with multigrid V-cycles
    (inner = 2; the hierarchy never mixes parts)."""
    capi, device = dev
    meshes, cases = _ensemble()
    bcs = [[c.bc_ne(), c.bc_phi()] for c in cases]
    ens = device.DeviceMesh(meshes, bcs, ensemble=True, prec=prec)
    geos = [geometry_of(m) for m in meshes]
    fs = [-1e3 * (i + 1) * gaussian(g.cen, (0.5, 0.5, 0.5), 0.2) for i, g in enumerate(geos)]
    fd = ens.to_device(np.concatenate(fs), torch.float64)
    phi = torch.zeros(ens.n_cell, dtype=torch.float64, device="cuda")
    opts = capi.solve_opts(rtol=1e-9, prec=capi.FVGB_FP64 if prec == "fp64" else capi.FVGB_FP32,
                           inner=inner)
    st, info = capi.fvgb_poisson_solve(ens.handle, 1, fd, phi, opts)
    relres, outer, its = capi.fvgb_solve_parts(ens.handle, 3)
    assert np.all(relres <= 1e-9) and np.all(outer >= 1)
    got = ens.to_host(phi)
    off = 0
    for g, c, f in zip(geos, cases, fs):
        x = got[off:off + g.n_cell]
        assert poisson.relative_residual(g, c.bc_phi(), f, x) <= 1.01e-9
        assert rel(x, poisson.solve(g, c.bc_phi(), f)) < 1e-7
        off += g.n_cell
    # a second solve from the solution: no outer step needed for any part
    st, info = capi.fvgb_poisson_solve(ens.handle, 1, fd, phi, opts)
    relres, outer, its = capi.fvgb_solve_parts(ens.handle, 3)
    assert np.all(outer == 0)
    ens.free()


def test_ensemble_streamer_matches_oracle_per_part(dev):
    capi, device = dev
    meshes, cases = _ensemble()
    bcs = [[c.bc_ne(), c.bc_phi()] for c in cases]
    ens = device.DeviceMesh(meshes, bcs, ensemble=True)
    geos = [geometry_of(m) for m in meshes]
    dt = 2e-9
    ne0 = [gaussian(g.cen, c.centre, c.sigma, c.peak, c.background) for g, c in zip(geos, cases)]
    ni0 = [n * (1.0 + 0.03 * np.sin(6 * g.cen[:, 1])) for n, g in zip(ne0, geos)]
    ne = ens.to_device(np.concatenate(ne0))
    ni = ens.to_device(np.concatenate(ni0))
    phi = torch.zeros(ens.n_cell, dtype=torch.float64, device="cuda")
    c0 = cases[0]
    sp = capi.streamer_params(mu=c0.mu, A=c0.A, B=c0.B, De=c0.De, dt=dt, solve=capi.solve_opts(rtol=1e-10))
    capi.fvgb_streamer_step(ens.handle, sp, ne, ni, phi, None, 3)
    torch.cuda.synchronize()
    gne, gni, gphi = ens.to_host(ne), ens.to_host(ni), ens.to_host(phi)
    off = 0
    for g, c, a, b in zip(geos, cases, ne0, ni0):
        p = streamer.Params(V=c.V, mu=c.mu, A=c.A, B=c.B, De=c.De)
        for _ in range(3):
            a, b, ophi, _, _ = streamer.step(g, p, a, b, dt)
        sl = slice(off, off + g.n_cell)
        assert rel(gphi[sl], ophi) < 1e-7
        assert rel(gne[sl], a) < 1e-7
        assert rel(gni[sl], b) < 1e-7
        off += g.n_cell
    ens.free()
