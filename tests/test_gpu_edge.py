"""Edge cases of the C ABI on the GPU, against the oracle: a mesh of one tetrahedron and of
one triangle (no node neighbours: the least-squares gradient stands on the Dirichlet ghost
points alone; every SELL slice is empty; most blocks of the persistent solve own no row),
zero-step calls, the multigrid inner solve on a mesh too small for any coarse level, and
an ensemble whose first part is a single cell."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import fv, ls, poisson  # noqa: E402
from synth.meshgen import Mesh, gaussian, jittered_cube  # noqa: E402
from tests.conftest import geometry_of  # noqa: E402

TOL64 = 1e-12
DIR3 = {1: ("dirichlet", 1.0), 2: ("dirichlet", 2.0), 3: ("dirichlet", -1.0), 4: ("dirichlet", 0.5)}
DIR2 = {1: ("dirichlet", 1.0), 2: ("dirichlet", -2.0), 3: ("dirichlet", 0.25)}


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


def single_tet():
    xyz = np.array([[0.1, 0.0, 0.0], [1.0, 0.2, 0.0], [0.0, 1.0, 0.1], [0.2, 0.1, 1.0]])
    bface = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]], dtype=np.int32)
    return Mesh(3, xyz, np.array([[0, 1, 2, 3]], dtype=np.int32), bface,
                np.array([1, 2, 3, 4], dtype=np.int32), 1.0)


def single_triangle():
    xyz = np.array([[0.0, 0.0], [1.0, 0.1], [0.2, 0.9]])
    bface = np.array([[1, 2], [0, 2], [0, 1]], dtype=np.int32)
    return Mesh(2, xyz, np.array([[0, 1, 2]], dtype=np.int32), bface,
                np.array([1, 2, 3], dtype=np.int32), 1.0)


@pytest.mark.parametrize("which", ["tet", "triangle"])
def test_single_cell_mesh(dev, which):
    capi, device = dev
    m, bc = (single_tet(), DIR3) if which == "tet" else (single_triangle(), DIR2)
    g = geometry_of(m)
    d = m.dim
    dm = device.DeviceMesh(m, [bc])
    u = np.array([3.0])
    ud = dm.to_device(u)
    gd, uvd = dm.empty(d, 1), dm.empty(dm.n_vert)
    capi.fvgb_gradient(dm.handle, 0, ud, gd)
    capi.fvgb_vertex_values(dm.handle, 0, ud, uvd)
    torch.cuda.synchronize()
    assert rel(dm.to_host(gd).T, ls.ls_gradient(g, bc, u)) < TOL64
    capi.fvgb_gradient_vertex(dm.handle, 0, ud, gd)
    torch.cuda.synchronize()
    assert rel(dm.to_host(gd).T, ls.ls_gradient_vertex(g, bc, u)) < TOL64
    assert rel(dm.vert_to_host(uvd), ls.vertex_values(g, bc, u)) < TOL64
    vel = np.array([0.3, -0.7, 0.2])[:d]
    res = dm.empty(1)
    for recon in (0, 1):
        capi.fvgb_fv_residual(dm.handle, capi.tcoef(vel_const=vel, diff=0.05, bcset=0, recon=recon), ud, res)
        torch.cuda.synchronize()
        assert rel(dm.to_host(res), fv.residual(g, bc, u, vel, 0.05, recon=recon)) < TOL64
    # zero steps leave u as it is; three Euler steps match the oracle
    capi.fvgb_fv_step(dm.handle, capi.tcoef(vel_const=vel, diff=0.05, bcset=0), ud, 1e-3, 0)
    torch.cuda.synchronize()
    assert dm.to_host(ud)[0] == 3.0
    want = u.copy()
    for _ in range(3):
        want = fv.rk_step(g, bc, want, vel, 0.05, 1e-3)
    capi.fvgb_fv_step(dm.handle, capi.tcoef(vel_const=vel, diff=0.05, bcset=0), ud, 1e-3, 3)
    torch.cuda.synchronize()
    assert rel(dm.to_host(ud), want) < TOL64
    # Poisson: one unknown; CG and multigrid (no coarse level: the dense solve) agree
    f = np.array([-40.0])
    exact = poisson.solve(g, bc, f, dense=True)
    for inner in (0, 2):
        phi = torch.zeros(1, dtype=torch.float64, device="cuda")
        st, info = capi.fvgb_poisson_solve(dm.handle, 0, dm.to_device(f, torch.float64), phi,
                                           capi.solve_opts(rtol=1e-12, inner=inner))
        torch.cuda.synchronize()
        assert rel(dm.to_host(phi), exact) < 1e-11 and info.rel_res <= 1e-12
    dm.free()


def test_streamer_zero_steps_and_one_cell_part(dev):
    """fvgb_streamer_step with nsteps = 0 changes nothing; an ensemble of a single
    tetrahedron and a small cube solves each part to its own tolerance."""
    capi, device = dev
    tet, cube = single_tet(), jittered_cube(3, seed=9)
    phi_bc_tet = {1: ("dirichlet", 0.0), 2: ("dirichlet", 0.0), 3: ("dirichlet", 0.0), 4: ("dirichlet", 100.0)}
    # a lone cell needs Dirichlet faces in every set (else its gradient stencil is empty)
    ne_bc_tet = {t: ("dirichlet", 1e12) for t in range(1, 5)}
    phi_bc_cube = {1: ("neumann", 0.0), 2: ("neumann", 0.0), 3: ("neumann", 0.0), 4: ("neumann", 0.0),
                   5: ("dirichlet", 0.0), 6: ("dirichlet", 100.0)}
    ne_bc_cube = {t: ("neumann", 0.0) for t in range(1, 7)}
    ens = device.DeviceMesh([tet, cube], [[ne_bc_tet, phi_bc_tet], [ne_bc_cube, phi_bc_cube]], ensemble=True)
    gc = geometry_of(cube)
    ne0 = np.concatenate([[1e12], gaussian(gc.cen, (0.5, 0.5, 0.5), 0.3, 1e12, 1e9)])
    ne, ni = ens.to_device(ne0), ens.to_device(ne0 * 1.01)
    phi = torch.zeros(ens.n_cell, dtype=torch.float64, device="cuda")
    sp = capi.streamer_params(dt=1e-10, solve=capi.solve_opts(rtol=1e-10))
    before = [t.clone() for t in (ne, ni, phi)]
    assert capi.fvgb_streamer_step(ens.handle, sp, ne, ni, phi, None, 0) == []
    torch.cuda.synchronize()
    for a, b in zip(before, (ne, ni, phi)):
        assert torch.equal(a, b)
    # per-part Poisson solves against the oracle
    fs = [np.array([-50.0]), -1e3 * gaussian(gc.cen, (0.5, 0.5, 0.5), 0.2)]
    for inner in (0, 2):
        phi.zero_()
        st, info = capi.fvgb_poisson_solve(ens.handle, 1, ens.to_device(np.concatenate(fs), torch.float64),
                                           phi, capi.solve_opts(rtol=1e-10, inner=inner))
        relres, outer, its = capi.fvgb_solve_parts(ens.handle, 2)
        assert np.all(relres <= 1e-10)
        got = ens.to_host(phi)
        assert rel(got[:1], poisson.solve(geometry_of(tet), phi_bc_tet, fs[0], dense=True)) < 1e-9
        assert poisson.relative_residual(gc, phi_bc_cube, fs[1], got[1:]) <= 1.01e-10
    ens.free()


def test_multigrid_solves_on_reused_device_memory(dev):
    """A mesh uploaded into device memory that held other data (0xFF bytes) solves with the
    multigrid inner solve in host and graph mode: no state of the solver may depend on what
    the allocation held before (the inner solve's status words are zeroed at upload)."""
    capi, device = dev
    junk = torch.full((512 * 1024 * 1024,), 255, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    del junk
    torch.cuda.empty_cache()
    m = jittered_cube(10, seed=41)
    from synth.workloads import StreamerCase
    case = StreamerCase(sigma=0.15, peak=1e13)
    dm = device.DeviceMesh(m, [case.bc_ne(), case.bc_phi()], prec="mixed")
    ne0 = case.initial(m)[0]
    for graph in (False, True):
        ne, ni = dm.to_device(ne0), dm.to_device(ne0 * 1.02)
        phi = torch.zeros(dm.n_cell, dtype=torch.float64, device="cuda")
        sp = capi.streamer_params(mu=case.mu, A=case.A, B=case.B, De=case.De, dt=2e-9,
                                  solve=capi.solve_opts(rtol=1e-9, inner=2, prec=capi.FVGB_FP32))
        capi.fvgb_set_graph_mode(dm.handle, graph)
        infos = capi.fvgb_streamer_step(dm.handle, sp, ne, ni, phi, None, 2)
        assert all(i["rel_res"] <= 1e-9 for i in infos)
    capi.fvgb_set_graph_mode(dm.handle, False)
    dm.free()
