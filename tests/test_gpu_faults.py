"""Failure detection without a GPU fault: the bounded grid barrier of the persistent CG
kernel made to run out by the test hook (one block never arrives, the wait limit cut to a
few milliseconds), reported as FVGB_ETIMEOUT by the host-driven solve and by a graph-mode
streamer step; and the latched status word of the transport kernels, set by a NaN placed
in the input on the host and reported by fvgb_sync and by the next Poisson solve. After
each, the mesh keeps working."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from synth.meshgen import jittered_cube  # noqa: E402
from synth.workloads import StreamerCase  # noqa: E402
from oracle import poisson  # noqa: E402
from tests.conftest import geometry_of  # noqa: E402

PHI3 = {1: ("neumann", 0.0), 2: ("neumann", 0.0), 3: ("neumann", 0.0), 4: ("neumann", 0.0),
        5: ("dirichlet", 0.0), 6: ("dirichlet", 100.0)}
NEU3 = {t: ("neumann", 0.0) for t in range(1, 7)}


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_00925_gb300 import build
    build.build()
    from paper_2203_00925_gb300 import capi, device
    return capi, device


def _status(capi, fn, *args, **kw):
    try:
        fn(*args, **kw)
    except capi.FvgbError as e:
        return e.status
    return capi.FVGB_OK


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_barrier_timeout_host_loop_and_graph(dev, prec):
    capi, device = dev
    m = jittered_cube(8, seed=11)
    g = geometry_of(m)
    dm = device.DeviceMesh(m, [NEU3, PHI3], prec=prec)
    inner_prec = capi.FVGB_FP64 if prec == "fp64" else capi.FVGB_FP32
    opts = capi.solve_opts(rtol=1e-8, prec=inner_prec)
    f = dm.to_device(np.sin(3 * g.cen[:, 0]) * 1e3, torch.float64)
    phi = torch.zeros(dm.n_cell, dtype=torch.float64, device="cuda")
    # host-driven solve: the waits of the first barrier run out after 5 ms
    capi.fvgb_test_barrier(dm.handle, 1, 5.0)
    assert _status(capi, capi.fvgb_poisson_solve, dm.handle, 1, f, phi, opts) == capi.FVGB_ETIMEOUT
    assert "timed out" in capi.lib.fvgb_last_error().decode()
    # graph mode: the device-side loop ends with the timeout status
    case = StreamerCase(V=100.0, peak=1e12, background=1e9, sigma=0.2)
    ne0, _ = case.initial(m)
    ne, ni = dm.to_device(ne0), dm.to_device(ne0 * 1.01)
    sp = capi.streamer_params(mu=case.mu, A=case.A, B=case.B, De=case.De, dt=1e-12, solve=opts)
    capi.fvgb_set_graph_mode(dm.handle, True)
    phi.zero_()
    assert _status(capi, capi.fvgb_streamer_step, dm.handle, sp, ne, ni, phi, None, 2) == capi.FVGB_ETIMEOUT
    capi.fvgb_set_graph_mode(dm.handle, False)
    # the graph's transport ran on the unconverged potential: clear whatever it latched
    assert _status(capi, capi.fvgb_sync, dm.handle) in (capi.FVGB_OK, capi.FVGB_ENONFINITE)
    # hook off: the same solve converges and matches the direct solution
    capi.fvgb_test_barrier(dm.handle, -1, 0.0)
    phi.zero_()
    _, info = capi.fvgb_poisson_solve(dm.handle, 1, f, phi, opts)
    assert info.rel_res <= 1e-8
    want = poisson.solve(g, PHI3, dm.to_host(f))
    got = dm.to_host(phi)
    assert np.linalg.norm(got - want) <= 1e-6 * np.linalg.norm(want)
    with pytest.raises(capi.FvgbError):
        capi.fvgb_test_barrier(dm.handle, 10 ** 6, 1.0)
    dm.free()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_nonfinite_transport_is_latched(dev, prec):
    capi, device = dev
    m = jittered_cube(6, seed=12)
    g = geometry_of(m)
    dm = device.DeviceMesh(m, [NEU3, PHI3], prec=prec)
    u0 = 1.0 + 0.1 * np.cos(4 * g.cen[:, 1])
    tc = capi.tcoef(vel_const=(0.2, 0.1, -0.3), diff=0.05, bcset=0)
    # a clean step leaves the status clear
    u = dm.to_device(u0)
    capi.fvgb_fv_step(dm.handle, tc, u, 1e-4, 2)
    capi.fvgb_sync(dm.handle)
    # NaN placed on the host: the step runs, fvgb_sync reports it once
    bad = u0.copy()
    bad[17] = np.nan
    u = dm.to_device(bad)
    capi.fvgb_fv_step(dm.handle, tc, u, 1e-4, 1)
    assert _status(capi, capi.fvgb_sync, dm.handle) == capi.FVGB_ENONFINITE
    capi.fvgb_sync(dm.handle)
    # a residual with NaN, then a Poisson solve with a clean right-hand side: the solve
    # reports the latched status, and the next one runs normally
    res = dm.empty(dm.n_cell)
    capi.fvgb_fv_residual(dm.handle, tc, u, res)
    f = dm.to_device(np.ones(g.n_cell), torch.float64)
    phi = torch.zeros(dm.n_cell, dtype=torch.float64, device="cuda")
    opts = capi.solve_opts(rtol=1e-8)
    assert _status(capi, capi.fvgb_poisson_solve, dm.handle, 1, f, phi, opts) == capi.FVGB_ENONFINITE
    _, info = capi.fvgb_poisson_solve(dm.handle, 1, f, phi, opts)
    assert info.rel_res <= 1e-8
    capi.fvgb_sync(dm.handle)
    dm.free()
