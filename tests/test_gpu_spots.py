"""GPU plasma spots of the branching streamer (Section 4, "Streamer Branching") against the
FP64 oracle: streamer steps whose windows cut the spots' switch-on intervals, one call or
two (the start time carried by the caller), host-driven and graph-captured (bitwise
equal), and the exact total that a spot deposits."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from synth.meshgen import jittered_cube, gaussian  # noqa: E402
from oracle import streamer, fv  # noqa: E402
from tests.conftest import geometry_of  # noqa: E402

TOL32 = 1e-5


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_00925_gb300 import build
    build.build()
    from paper_2203_00925_gb300 import capi, device
    return capi, device


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


DT = 2e-9
SPOTS = [dict(centre=(0.55, 0.5, 0.75), amplitude=4e21, sigma=0.12, t_on=2.5e-9, duration=3.2e-9),
         dict(centre=(0.45, 0.52, 0.7), amplitude=2e21, sigma=0.15, t_on=5e-9, duration=1e-9)]


def _case(k=6):
    m = jittered_cube(k, seed=201)
    g = geometry_of(m)
    p = streamer.Params(sigma=0.12, peak=1e13, background=1e9, V=12500.0)
    ne = gaussian(g.cen, p.centre, p.sigma, p.peak, p.background)
    ni = ne * (1.0 + 0.05 * np.sin(7 * g.cen[:, 0]))
    return m, g, p, ne, ni


def _oracle_run(g, p, ne, ni, nsteps):
    spots = [streamer.Spot(**s) for s in SPOTS]
    t = 0.0
    for _ in range(nsteps):
        ne, ni, phi, E, S = streamer.step(g, p, ne, ni, DT, spots=spots, t=t)
        t += DT
    return ne, ni, phi


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_streamer_steps_with_spots(dev, prec):
    capi, device = dev
    m, g, p, ne, ni = _case()
    nsteps = 5                       # windows [2.5, 5.7] and [5, 6] ns against steps of 2 ns
    one, oni, ophi = _oracle_run(g, p, ne, ni, nsteps)
    # the spots matter: the run without them differs by far more than the tolerance
    bne, bni, _ = ne.copy(), ni.copy(), None
    for _ in range(nsteps):
        bne, bni, _, _, _ = streamer.step(g, p, bne, bni, DT)
    assert rel(bni, oni) > 1e-3
    dm = device.DeviceMesh(m, [streamer.bc_ne(), streamer.bc_phi(p)], prec=prec)
    solve = capi.solve_opts(rtol=1e-10, prec=capi.FVGB_FP64 if prec == "fp64" else capi.FVGB_FP32)
    spots = [capi.spot(**s) for s in SPOTS]
    tol = 1e-7 if prec == "fp64" else TOL32
    # one call of five steps
    ned, nid = dm.to_device(ne), dm.to_device(ni)
    phid = torch.zeros(dm.n_cell, dtype=torch.float64, device="cuda")
    sp = capi.streamer_params(mu=p.mu, A=p.A, B=p.B, De=p.De, dt=DT, solve=solve, spots=spots)
    infos = capi.fvgb_streamer_step(dm.handle, sp, ned, nid, phid, None, nsteps)
    torch.cuda.synchronize()
    assert all(i["rel_res"] <= 1e-10 for i in infos)
    assert rel(dm.to_host(ned), one) < tol
    assert rel(dm.to_host(nid), oni) < tol
    assert rel(dm.to_host(phid), ophi) < 1e-7
    # two calls (2 + 3 steps), the second starting at the time the first reached
    ne2, ni2 = dm.to_device(ne), dm.to_device(ni)
    phi2 = torch.zeros(dm.n_cell, dtype=torch.float64, device="cuda")
    capi.fvgb_streamer_step(dm.handle, sp, ne2, ni2, phi2, None, 2)
    t0 = 0.0
    for _ in range(2):
        t0 += DT
    sp2 = capi.streamer_params(mu=p.mu, A=p.A, B=p.B, De=p.De, dt=DT, solve=solve, spots=spots, t0=t0)
    capi.fvgb_streamer_step(dm.handle, sp2, ne2, ni2, phi2, None, nsteps - 2)
    torch.cuda.synchronize()
    assert torch.equal(ne2, ned) and torch.equal(ni2, nid)
    dm.free()


def test_graph_steps_with_spots_match_host_steps(dev):
    capi, device = dev
    m, g, p, ne, ni = _case()
    dm = device.DeviceMesh(m, [streamer.bc_ne(), streamer.bc_phi(p)], prec="mixed")
    solve = capi.solve_opts(rtol=1e-10, prec=capi.FVGB_FP32)
    sp = capi.streamer_params(mu=p.mu, A=p.A, B=p.B, De=p.De, dt=DT, solve=solve,
                              spots=[capi.spot(**s) for s in SPOTS])
    out = []
    for graph in (False, True):
        ned, nid = dm.to_device(ne), dm.to_device(ni)
        phid = torch.zeros(dm.n_cell, dtype=torch.float64, device="cuda")
        capi.fvgb_set_graph_mode(dm.handle, graph)
        capi.fvgb_streamer_step(dm.handle, sp, ned, nid, phid, None, 5)
        torch.cuda.synchronize()
        out.append((ned.clone(), nid.clone(), phid.clone()))
    capi.fvgb_set_graph_mode(dm.handle, False)
    for a, b in zip(*out):
        assert torch.equal(a, b)
    dm.free()


def test_spot_total_deposit(dev):
    """Without ionisation the ions grow only by the spots: by sum_k S_k duration_k
    sum_i mu_i g_k(x_i) once both windows are past (FP64, to round-off)."""
    capi, device = dev
    m, g, p, ne, ni = _case()
    p.A = 0.0
    dm = device.DeviceMesh(m, [streamer.bc_ne(), streamer.bc_phi(p)], prec="fp64")
    ned, nid = dm.to_device(ne), dm.to_device(ni)
    phid = torch.zeros(dm.n_cell, dtype=torch.float64, device="cuda")
    sp = capi.streamer_params(mu=p.mu, A=0.0, B=p.B, De=p.De, dt=DT, solve=capi.solve_opts(rtol=1e-10),
                              spots=[capi.spot(**s) for s in SPOTS])
    q0 = capi.fvgb_integral(dm.handle, nid)
    capi.fvgb_streamer_step(dm.handle, sp, ned, nid, phid, None, 4)
    q1 = capi.fvgb_integral(dm.handle, nid)
    want = sum(s["amplitude"] * s["duration"] *
               fv.mass(g, np.exp(-((g.cen - np.array(s["centre"])) ** 2).sum(1) / s["sigma"] ** 2))
               for s in SPOTS)
    assert abs((q1 - q0) - want) <= 1e-11 * want
    dm.free()
