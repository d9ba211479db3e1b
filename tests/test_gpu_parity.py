"""GPU parity: every C-ABI operator against the FP64 CPU oracle on the same seeded
meshes and inputs. Tolerances (relative L2): 1e-12 on FP64 meshes, 1e-5 on FP32 meshes;
iterative solves are judged by the oracle-evaluated FP64 residual and by the distance
to the oracle's direct solution (1e-6)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from synth.meshgen import jittered_cube, jittered_square, gaussian  # noqa: E402
from oracle import fv, ls, poisson, streamer  # noqa: E402
from tests.conftest import geometry_of  # noqa: E402

TOL64, TOL32 = 1e-12, 1e-5


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_00925_gb300 import build
    build.build()
    from paper_2203_00925_gb300 import capi, device
    return capi, device


WALLS2 = {t: ("wall", 0.0) for t in range(1, 5)}
MIXED3 = {1: ("wall", 0.0), 2: ("neumann", 0.0), 3: ("neumann", 0.0), 4: ("wall", 0.0),
          5: ("dirichlet", 0.25), 6: ("dirichlet", 1.5)}
PHI3 = {1: ("neumann", 0.0), 2: ("neumann", 0.0), 3: ("neumann", 0.0), 4: ("neumann", 0.0),
        5: ("dirichlet", 0.0), 6: ("dirichlet", 100.0)}


def meshes():
    return {
        "square50": (jittered_square(50, 101, 102), [WALLS2, {1: ("dirichlet", 1.0), 2: ("dirichlet", -1.0), 3: ("neumann", 0.0), 4: ("wall", 0.0)}]),
        "cube7": (jittered_cube(7, seed=301), [MIXED3, PHI3]),   # 2058 cells: ragged last tile
    }


def smooth_field(cen, seed):
    rng = np.random.default_rng(seed)
    k = rng.uniform(1, 3, size=cen.shape[1])
    return np.sin(cen @ k) + 0.3 * rng.normal(size=cen.shape[0])


@pytest.mark.parametrize("name", ["square50", "cube7"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_gradient_and_vertex_values(dev, name, prec):
    capi, device = dev
    m, bcs = meshes()[name]
    g = geometry_of(m)
    dm = device.DeviceMesh(m, bcs, prec=prec)
    tol = TOL64 if prec == "fp64" else TOL32
    u = smooth_field(g.cen, 5)
    ud = dm.to_device(u)
    for k, bc in enumerate(bcs):
        gd = dm.empty(m.dim, dm.n_cell)
        capi.fvgb_gradient(dm.handle, k, ud, gd)
        uvd = dm.empty(dm.n_vert)
        capi.fvgb_vertex_values(dm.handle, k, ud, uvd)
        torch.cuda.synchronize()
        want = ls.ls_gradient(g, bc, u)
        assert rel(dm.to_host(gd).T, want) < tol
        assert rel(dm.vert_to_host(uvd), ls.vertex_values(g, bc, u)) < tol
    # linear fields: exact gradient on every cell (FP64). Wall and Neumann faces add no
    # least-squares point, so any linear field is exact with them; a Dirichlet set is exact
    # for the linear field that takes its boundary values (here: linear in z between the
    # plates z = 0 and z = 1, whose points only slide tangentially)
    if prec == "fp64":
        b = np.arange(1, m.dim + 1) * 0.7
        gd = dm.empty(m.dim, dm.n_cell)
        if name == "square50":
            capi.fvgb_gradient(dm.handle, 0, dm.to_device(0.5 + g.cen @ b), gd)
            torch.cuda.synchronize()
            assert np.abs(dm.to_host(gd).T - b).max() < 1e-11
        else:
            capi.fvgb_gradient(dm.handle, 1, dm.to_device(100.0 * g.cen[:, 2]), gd)
            torch.cuda.synchronize()
            assert np.abs(dm.to_host(gd).T - [0.0, 0.0, 100.0]).max() < 1e-10
            dn = device.DeviceMesh(m, [{t: ("neumann", 0.0) for t in range(1, 7)}], prec="fp64")
            gn = dn.empty(m.dim, dn.n_cell)
            capi.fvgb_gradient(dn.handle, 0, dn.to_device(0.5 + g.cen @ b), gn)
            torch.cuda.synchronize()
            assert np.abs(dn.to_host(gn).T - b).max() < 1e-11
            dn.free()
    dm.free()


@pytest.mark.parametrize("name", ["square50", "cube7"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_gradient_vertex_factorised(dev, name, prec):
    """The multiplicity-weighted (vertex-factorised) gradient against the oracle's plain
    sum over cell pairs weighted by their shared vertices, with both boundary sets."""
    capi, device = dev
    m, bcs = meshes()[name]
    g = geometry_of(m)
    dm = device.DeviceMesh(m, bcs, prec=prec)
    tol = TOL64 if prec == "fp64" else TOL32
    u = smooth_field(g.cen, 9)
    ud = dm.to_device(u)
    for k, bc in enumerate(bcs):
        gd = dm.empty(m.dim, dm.n_cell)
        capi.fvgb_gradient_vertex(dm.handle, k, ud, gd)
        torch.cuda.synchronize()
        assert rel(dm.to_host(gd).T, ls.ls_gradient_vertex(g, bc, u)) < tol
    dm.free()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_residual_all_boundary_kinds(dev, prec):
    capi, device = dev
    m, bcs = meshes()["cube7"]
    g = geometry_of(m)
    dm = device.DeviceMesh(m, bcs, prec=prec)
    rng = np.random.default_rng(3)
    u = smooth_field(g.cen, 7) + 2.0
    vel = rng.normal(size=(g.n_cell, 3))
    src = rng.normal(size=g.n_cell)
    want = fv.residual(g, bcs[0], u, vel, 0.1, src=src)
    ud, veld, srcd = dm.to_device(u), dm.to_device(vel.T), dm.to_device(src)
    res = dm.empty(dm.n_cell)
    capi.fvgb_fv_residual(dm.handle, capi.tcoef(vel=veld, diff=0.1, src=srcd, bcset=0), ud, res)
    torch.cuda.synchronize()
    assert rel(dm.to_host(res), want) < (TOL64 if prec == "fp64" else TOL32)
    # constant velocity, no source
    want = fv.residual(g, bcs[0], u, np.array([0.3, -0.4, 0.9]), 0.05)
    capi.fvgb_fv_residual(dm.handle, capi.tcoef(vel_const=(0.3, -0.4, 0.9), diff=0.05, bcset=0), ud, res)
    torch.cuda.synchronize()
    assert rel(dm.to_host(res), want) < (TOL64 if prec == "fp64" else TOL32)
    dm.free()


def _config1():
    m = jittered_square(50, 101, 102)
    g = geometry_of(m)
    u0 = gaussian(g.cen, (0.3, 0.3), 0.05)
    vel = np.array([1.0, 0.5])
    dt = fv.cfl_dt(g, WALLS2, vel, 0.01, 0.4)
    return m, g, u0, vel, dt


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_config1_200_euler_steps(dev, prec):
    """2D advection-diffusion, 5,000 cells, 200 explicit Euler steps at CFL 0.4:
    parity with the oracle and mass conserved to round-off."""
    capi, device = dev
    m, g, u0, vel, dt = _config1()
    coef = fv.diamond_coefficients(g)
    w = ls.vertex_weights(g)
    u = u0.copy()
    for _ in range(200):
        u = fv.rk_step(g, WALLS2, u, vel, 0.01, dt, coef=coef, weights=w)
    dm = device.DeviceMesh(m, [WALLS2], prec=prec)
    ud = dm.to_device(u0)
    capi.fvgb_fv_step(dm.handle, capi.tcoef(vel_const=vel, diff=0.01, bcset=0), ud, dt, 200)
    torch.cuda.synchronize()
    got = dm.to_host(ud)
    assert rel(got, u) < (TOL64 if prec == "fp64" else TOL32)
    m0 = fv.mass(g, u0)
    if prec == "fp64":
        assert abs(fv.mass(g, got) - m0) <= 1e-13 * abs(m0)
    else:
        assert abs(fv.mass(g, got) - m0) <= 1e-5 * abs(m0)
    # the device-side FP64 integral agrees with the oracle's and shows conservation too
    gm = capi.fvgb_integral(dm.handle, ud)
    assert gm == pytest.approx(fv.mass(g, got), rel=1e-13 if prec == "fp64" else 1e-7)
    assert abs(gm - m0) <= (1e-13 if prec == "fp64" else 1e-5) * abs(m0)
    dm.free()


def test_rk3_stages(dev):
    capi, device = dev
    m, g, u0, vel, dt = _config1()
    u = u0.copy()
    for _ in range(20):
        u = fv.rk_step(g, WALLS2, u, vel, 0.01, dt, alphas=(0.5, 0.5, 1.0))
    dm = device.DeviceMesh(m, [WALLS2])
    ud = dm.to_device(u0)
    capi.fvgb_fv_step(dm.handle, capi.tcoef(vel_const=vel, diff=0.01), ud, dt, 20, stage_alpha=[0.5, 0.5, 1.0])
    torch.cuda.synchronize()
    assert rel(dm.to_host(ud), u) < TOL64
    dm.free()


def test_poisson_operator_and_rhs(dev):
    capi, device = dev
    m, bcs = meshes()["cube7"]
    g = geometry_of(m)
    dm = device.DeviceMesh(m, bcs)
    x = smooth_field(g.cen, 11)
    f = smooth_field(g.cen, 12)
    xd, fd = dm.to_device(x, torch.float64), dm.to_device(f, torch.float64)
    y = dm.empty(dm.n_cell, dtype=torch.float64)
    b = dm.empty(dm.n_cell, dtype=torch.float64)
    capi.fvgb_poisson_apply(dm.handle, 1, xd, y)
    capi.fvgb_poisson_rhs(dm.handle, 1, fd, b)
    torch.cuda.synchronize()
    assert rel(dm.to_host(y), poisson.apply(g, PHI3, x)) < TOL64
    assert rel(dm.to_host(b), poisson.rhs(g, PHI3, f)) < TOL64
    dm.free()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_poisson_solve(dev, prec):
    capi, device = dev
    m, bcs = meshes()["cube7"]
    g = geometry_of(m)
    dm = device.DeviceMesh(m, bcs, prec="fp64" if prec == "fp64" else "mixed")
    f = -1e3 * gaussian(g.cen, (0.5, 0.5, 0.6), 0.2)
    want = poisson.solve(g, PHI3, f)
    fd = dm.to_device(f, torch.float64)
    phi = torch.zeros(dm.n_cell, dtype=torch.float64, device="cuda")
    opts = capi.solve_opts(rtol=1e-8, inner_rtol=0.1,
                           prec=capi.FVGB_FP64 if prec == "fp64" else capi.FVGB_FP32)
    st, info = capi.fvgb_poisson_solve(dm.handle, 1, fd, phi, opts)
    torch.cuda.synchronize()
    got = dm.to_host(phi)
    assert info.rel_res <= 1e-8
    assert poisson.relative_residual(g, PHI3, f, got) <= 1.01e-8
    assert rel(got, want) < 1e-6
    assert info.outer_its >= 1 and info.inner_its_total > 0
    # warm start from the solution: converged at once
    st, info2 = capi.fvgb_poisson_solve(dm.handle, 1, fd, phi, opts)
    assert info2.outer_its == 0
    # deterministic: a second cold solve gives identical bits
    phi2 = torch.zeros_like(phi)
    capi.fvgb_poisson_solve(dm.handle, 1, fd, phi2, opts)
    phi3 = torch.zeros_like(phi)
    capi.fvgb_poisson_solve(dm.handle, 1, fd, phi3, opts)
    assert torch.equal(phi2, phi3)
    dm.free()


def test_poisson_annex_on_gpu(dev):
    """Annex problem: P = 10 at x = 0, 0 at x = 1, Neumann elsewhere; exact 10 (1 - x)."""
    capi, device = dev
    m = jittered_cube(8, seed=17)
    g = geometry_of(m)
    annex = {1: ("dirichlet", 10.0), 2: ("dirichlet", 0.0), 3: ("neumann", 0.0),
             4: ("neumann", 0.0), 5: ("neumann", 0.0), 6: ("neumann", 0.0)}
    dm = device.DeviceMesh(m, [annex])
    phi = torch.zeros(dm.n_cell, dtype=torch.float64, device="cuda")
    capi.fvgb_poisson_solve(dm.handle, 0, None, phi, capi.solve_opts(rtol=1e-12))
    got = dm.to_host(phi)
    assert np.abs(got - 10.0 * (1.0 - g.cen[:, 0])).max() < 1e-8
    dm.free()


def test_annex_golden_fixture_on_gpu(dev):
    """The stored Annex example (tests/golden/annex_laplace.txt): the GPU solve gives the
    closed-form cell values."""
    capi, device = dev
    from tests.conftest import ANNEX_BC, load_annex
    m, expected = load_annex()
    for prec in ("fp64", "mixed"):
        dm = device.DeviceMesh(m, [ANNEX_BC], prec=prec)
        phi = torch.zeros(dm.n_cell, dtype=torch.float64, device="cuda")
        capi.fvgb_poisson_solve(dm.handle, 0, None, phi, capi.solve_opts(
            rtol=1e-12, prec=capi.FVGB_FP64 if prec == "fp64" else capi.FVGB_FP32))
        assert np.abs(dm.to_host(phi) - expected).max() < 1e-9
        dm.free()


def test_solver_error_paths(dev):
    capi, device = dev
    m, bcs = meshes()["cube7"]
    dm = device.DeviceMesh(m, bcs)
    f = torch.ones(dm.n_cell, dtype=torch.float64, device="cuda")
    phi = torch.zeros_like(f)
    st, info = capi.fvgb_poisson_solve(dm.handle, 1, f, phi, capi.solve_opts(maxit_outer=1), check=False)
    assert st == capi.FVGB_ENOCONV and info.outer_its == 1 and info.rel_res > 1e-8
    f[17] = float("nan")
    phi.zero_()
    st, info = capi.fvgb_poisson_solve(dm.handle, 1, f, phi, capi.solve_opts(), check=False)
    assert st == capi.FVGB_ENONFINITE
    dm.free()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_streamer_steps(dev, prec):
    capi, device = dev
    m = jittered_cube(6, seed=201)
    g = geometry_of(m)
    p = streamer.Params(sigma=0.12, peak=1e13, background=1e9, V=12500.0)
    ne = gaussian(g.cen, p.centre, p.sigma, p.peak, p.background)
    ni = ne * (1.0 + 0.05 * np.sin(7 * g.cen[:, 0]))
    dt = 2e-9
    nsteps = 4
    one, oni = ne.copy(), ni.copy()
    for _ in range(nsteps):
        one, oni, ophi, oE, _ = streamer.step(g, p, one, oni, dt)
    dm = device.DeviceMesh(m, [streamer.bc_ne(), streamer.bc_phi(p)],
                           prec="fp64" if prec == "fp64" else "mixed")
    ned, nid = dm.to_device(ne), dm.to_device(ni)
    phid = torch.zeros(dm.n_cell, dtype=torch.float64, device="cuda")
    Ed = dm.empty(3, dm.n_cell)
    sp = capi.streamer_params(mu=p.mu, A=p.A, B=p.B, De=p.De, dt=dt,
                              solve=capi.solve_opts(rtol=1e-10, prec=capi.FVGB_FP64 if prec == "fp64" else capi.FVGB_FP32))
    infos = capi.fvgb_streamer_step(dm.handle, sp, ned, nid, phid, Ed, nsteps)
    torch.cuda.synchronize()
    tol = 1e-7 if prec == "fp64" else TOL32
    assert rel(dm.to_host(phid), ophi) < 1e-7
    assert rel(dm.to_host(ned), one) < tol
    assert rel(dm.to_host(nid), oni) < tol
    assert rel(dm.to_host(Ed).T, oE) < 1e-6
    assert all(i["rel_res"] <= 1e-10 for i in infos)
    dm.free()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_muscl_residual_and_steps(dev, prec):
    """MUSCL + Barth-Jespersen (eq. 15): residual on a 3D mesh with every boundary kind,
    then 200 Euler steps and 20 RK3 steps of the 2D Gaussian (walls) against the oracle,
    mass conserved."""
    capi, device = dev
    tol = TOL64 if prec == "fp64" else TOL32
    m, bcs = meshes()["cube7"]
    g = geometry_of(m)
    dm = device.DeviceMesh(m, bcs, prec=prec)
    rng = np.random.default_rng(13)
    u = smooth_field(g.cen, 7) + 2.0
    vel = rng.normal(size=(g.n_cell, 3))
    src = rng.normal(size=g.n_cell)
    want = fv.residual(g, bcs[0], u, vel, 0.1, src=src, recon=1)
    assert rel(want, fv.residual(g, bcs[0], u, vel, 0.1, src=src)) > 1e-3
    res = dm.empty(dm.n_cell)
    capi.fvgb_fv_residual(dm.handle, capi.tcoef(vel=dm.to_device(vel.T), diff=0.1,
                                                src=dm.to_device(src), bcset=0, recon=1),
                          dm.to_device(u), res)
    torch.cuda.synchronize()
    assert rel(dm.to_host(res), want) < tol
    dm.free()
    m, g, u0, vel, dt = _config1()
    coef = fv.diamond_coefficients(g)
    w = ls.vertex_weights(g)
    dm = device.DeviceMesh(m, [WALLS2], prec=prec)
    for alphas, n in (((1.0,), 200), ((0.5, 0.5, 1.0), 20)):
        u = u0.copy()
        for _ in range(n):
            u = fv.rk_step(g, WALLS2, u, vel, 0.01, dt, alphas=alphas, coef=coef, weights=w, recon=1)
        ud = dm.to_device(u0)
        capi.fvgb_fv_step(dm.handle, capi.tcoef(vel_const=vel, diff=0.01, bcset=0, recon=1), ud, dt,
                          n, stage_alpha=list(alphas))
        torch.cuda.synchronize()
        got = dm.to_host(ud)
        assert rel(got, u) < tol
        m0 = fv.mass(g, u0)
        assert abs(capi.fvgb_integral(dm.handle, ud) - m0) <= (1e-13 if prec == "fp64" else 1e-5) * abs(m0)
    dm.free()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_streamer_steps_muscl(dev, prec):
    capi, device = dev
    m = jittered_cube(6, seed=201)
    g = geometry_of(m)
    p = streamer.Params(sigma=0.12, peak=1e13, background=1e9, V=12500.0)
    ne = gaussian(g.cen, p.centre, p.sigma, p.peak, p.background)
    ni = ne * (1.0 + 0.05 * np.sin(7 * g.cen[:, 0]))
    dt = 2e-9
    one, oni = ne.copy(), ni.copy()
    for _ in range(4):
        one, oni, ophi, oE, _ = streamer.step(g, p, one, oni, dt, recon=1)
    dm = device.DeviceMesh(m, [streamer.bc_ne(), streamer.bc_phi(p)],
                           prec="fp64" if prec == "fp64" else "mixed")
    ned, nid = dm.to_device(ne), dm.to_device(ni)
    phid = torch.zeros(dm.n_cell, dtype=torch.float64, device="cuda")
    sp = capi.streamer_params(mu=p.mu, A=p.A, B=p.B, De=p.De, dt=dt, recon=1,
                              solve=capi.solve_opts(rtol=1e-10, prec=capi.FVGB_FP64 if prec == "fp64" else capi.FVGB_FP32))
    infos = capi.fvgb_streamer_step(dm.handle, sp, ned, nid, phid, None, 4)
    torch.cuda.synchronize()
    tol = 1e-7 if prec == "fp64" else TOL32
    assert rel(dm.to_host(phid), ophi) < 1e-7
    assert rel(dm.to_host(ned), one) < tol
    assert rel(dm.to_host(nid), oni) < tol
    assert all(i["rel_res"] <= 1e-10 for i in infos)
    dm.free()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_poisson_solve_multigrid_inner(dev, prec):
    """Multigrid V-cycles as the inner solve: the same convergence guarantees (oracle
    residual, distance to the direct solution), far fewer outer steps than the CG needs
    inner iterations, a hierarchy that coarsens, bitwise reproducible."""
    capi, device = dev
    m, bcs = meshes()["cube7"]
    g = geometry_of(m)
    dm = device.DeviceMesh(m, bcs, prec="fp64" if prec == "fp64" else "mixed")
    f = -1e3 * gaussian(g.cen, (0.5, 0.5, 0.6), 0.2)
    want = poisson.solve(g, PHI3, f)
    fd = dm.to_device(f, torch.float64)
    opts = capi.solve_opts(rtol=1e-8, inner=2, prec=capi.FVGB_FP64 if prec == "fp64" else capi.FVGB_FP32)
    phi = torch.zeros(dm.n_cell, dtype=torch.float64, device="cuda")
    st, info = capi.fvgb_poisson_solve(dm.handle, 1, fd, phi, opts)
    torch.cuda.synchronize()
    got = dm.to_host(phi)
    assert info.rel_res <= 1e-8
    assert poisson.relative_residual(g, PHI3, f, got) <= 1.01e-8
    assert rel(got, want) < 1e-6
    assert 1 <= info.outer_its <= 40 and info.inner_its_total == 2 * info.outer_its
    sizes = capi.fvgb_amg_levels(dm.handle, 1, capi.FVGB_FP64 if prec == "fp64" else capi.FVGB_FP32)
    assert sizes[0] == dm.n_cell and sizes == sorted(sizes, reverse=True) and sizes[-1] <= 640
    phi2 = torch.zeros_like(phi)
    capi.fvgb_poisson_solve(dm.handle, 1, fd, phi2, opts)
    assert torch.equal(phi, phi2)
    dm.free()
    # a mesh larger than the coarsest size: several levels
    m2 = jittered_cube(12, seed=5)
    g2 = geometry_of(m2)
    dm2 = device.DeviceMesh(m2, [PHI3])
    f2 = -1e3 * gaussian(g2.cen, (0.4, 0.5, 0.7), 0.15)
    phi = torch.zeros(dm2.n_cell, dtype=torch.float64, device="cuda")
    st, info = capi.fvgb_poisson_solve(dm2.handle, 0, dm2.to_device(f2, torch.float64), phi,
                                       capi.solve_opts(rtol=1e-8, inner=2))
    torch.cuda.synchronize()
    assert poisson.relative_residual(g2, PHI3, f2, dm2.to_host(phi)) <= 1.01e-8
    assert len(capi.fvgb_amg_levels(dm2.handle, 0, capi.FVGB_FP64)) >= 3
    dm2.free()


@pytest.mark.parametrize("prec,recon", [("fp64", 0), ("mixed", 0), ("fp64", 1)])
def test_streamer_three_stage_steps(dev, prec, recon):
    """The eq. 6 three-stage streamer step (a Poisson solve per stage) against the oracle's,
    and graph mode (which runs such steps host-driven) gives the same bits."""
    capi, device = dev
    m = jittered_cube(6, seed=201)
    g = geometry_of(m)
    p = streamer.Params(sigma=0.12, peak=1e13, background=1e9, V=12500.0)
    ne = gaussian(g.cen, p.centre, p.sigma, p.peak, p.background)
    ni = ne * (1.0 + 0.05 * np.sin(7 * g.cen[:, 0]))
    dt, nsteps = 2e-9, 3
    one, oni = ne.copy(), ni.copy()
    for _ in range(nsteps):
        one, oni, ophi, oE, _ = streamer.step(g, p, one, oni, dt, recon=recon, alphas=(0.5, 0.5, 1.0))
    dm = device.DeviceMesh(m, [streamer.bc_ne(), streamer.bc_phi(p)],
                           prec="fp64" if prec == "fp64" else "mixed")
    outs = []
    for graph in (False, True):
        ned, nid = dm.to_device(ne), dm.to_device(ni)
        phid = torch.zeros(dm.n_cell, dtype=torch.float64, device="cuda")
        Ed = dm.empty(3, dm.n_cell)
        sp = capi.streamer_params(mu=p.mu, A=p.A, B=p.B, De=p.De, dt=dt, recon=recon, stages=3,
                                  solve=capi.solve_opts(rtol=1e-10, prec=capi.FVGB_FP64 if prec == "fp64" else capi.FVGB_FP32))
        capi.fvgb_set_graph_mode(dm.handle, graph)
        infos = capi.fvgb_streamer_step(dm.handle, sp, ned, nid, phid, Ed, nsteps)
        torch.cuda.synchronize()
        outs.append((ned, nid, phid, Ed))
        assert all(i["rel_res"] <= 1e-10 and i["outer_its"] >= 3 for i in infos[1:])
    capi.fvgb_set_graph_mode(dm.handle, False)
    ned, nid, phid, Ed = outs[0]
    tol = 1e-7 if prec == "fp64" else TOL32
    assert rel(dm.to_host(phid), ophi) < 1e-7
    assert rel(dm.to_host(ned), one) < tol
    assert rel(dm.to_host(nid), oni) < tol
    assert rel(dm.to_host(Ed).T, oE) < 1e-6
    for x, y in zip(outs[0], outs[1]):
        assert torch.equal(x, y)
    dm.free()
