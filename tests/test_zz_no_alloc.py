"""fvgb_fv_residual_noalloc, the residual entry point that allocates nothing, for callers
that cannot allocate device memory when they need a residual (a host program that hands
out device memory through its own pool, a time-critical loop that must not pay for
cudaMalloc). Its scratch is a fixed device array inside the library.

Checked through the C ABI:
* it returns bit for bit what fvgb_fv_residual returns (the same kernels run in the same
  order), on two calls in a row, for FP64 and FP32 meshes: the second call finds the
  first call's leftovers in the shared array;
* on a small mesh it agrees with the CPU oracle's residual of eq. 4;
* a call without diffusion (no vertex values are computed) and a call with a constant
  velocity, each after a call that left different data in the scratch, still match;
* an oversized mesh is refused with a clear error, and invalid or unsupported options
  with the statuses of fvgb_fv_residual.

The file name makes pytest collect it last."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from synth.meshgen import jittered_cube, jittered_square  # noqa: E402
from oracle import fv  # noqa: E402
from tests.conftest import geometry_of  # noqa: E402


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_00925_gb300 import build
    build.build()
    from paper_2203_00925_gb300 import capi, device
    return capi, device


MIXED3 = {1: ("wall", 0.0), 2: ("neumann", 0.0), 3: ("neumann", 0.0), 4: ("wall", 0.0),
          5: ("dirichlet", 0.25), 6: ("dirichlet", 1.5)}
WALLS2 = {t: ("wall", 0.0) for t in range(1, 5)}


def _pair(capi, dm, tc, u):
    want = dm.empty(dm.n_cell)
    got = dm.empty(dm.n_cell).fill_(float("nan"))
    capi.fvgb_fv_residual(dm.handle, tc, u, want)
    capi.fvgb_fv_residual_noalloc(dm.handle, tc, u, got)
    torch.cuda.synchronize()
    return got, want


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["cube", "square"])
def test_noalloc_matches_residual_twice(dev, prec, case):
    capi, device = dev
    if case == "cube":
        m, bc, dim = jittered_cube(9, seed=301), MIXED3, 3
    else:
        m, bc, dim = jittered_square(50, 101, 102), WALLS2, 2
    dm = device.DeviceMesh(m, [bc], prec=prec)
    gen = torch.Generator(device="cuda").manual_seed(7)
    for call in range(2):
        u = torch.rand(dm.n_cell, device="cuda", generator=gen, dtype=torch.float64).to(dm.real) + 1.0
        vel = torch.randn(dim, dm.n_cell, device="cuda", generator=gen, dtype=torch.float64).to(dm.real)
        src = torch.randn(dm.n_cell, device="cuda", generator=gen, dtype=torch.float64).to(dm.real)
        tc = capi.tcoef(vel=vel, diff=0.05 * (call + 1), src=src if call == 0 else None, bcset=0)
        got, want = _pair(capi, dm, tc, u)
        assert torch.isfinite(got).all()
        assert torch.equal(got, want)
    dm.free()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_noalloc_against_oracle_and_stale_scratch(dev, prec, tol):
    """Against the oracle's residual (per-cell velocity, diffusion, source, every boundary
    kind), then - with the scratch left dirty by that call - a pure convection call with a
    constant velocity (no vertex values are computed, so the stale ones must not be read)
    and a diffusion call with a constant velocity."""
    capi, device = dev
    m = jittered_cube(5, seed=41)
    g = geometry_of(m)
    dm = device.DeviceMesh(m, [MIXED3], prec=prec)
    rng = np.random.default_rng(3)
    u = 1.0 + np.sin(g.cen @ np.array([2.0, -1.0, 3.0])) + 0.1 * rng.random(g.n_cell)
    vel = rng.normal(size=(g.n_cell, 3))
    src = rng.normal(size=g.n_cell)
    ud = dm.to_device(u)
    cases = [
        (capi.tcoef(vel=dm.to_device(vel.T), diff=0.1, src=dm.to_device(src), bcset=0),
         fv.residual(g, MIXED3, u, vel, 0.1, src=src)),
        (capi.tcoef(vel_const=(0.3, -0.7, 0.5), diff=0.0, bcset=0),
         fv.residual(g, MIXED3, u, np.array([0.3, -0.7, 0.5]), 0.0)),
        (capi.tcoef(vel_const=(-0.2, 0.4, 0.9), diff=0.05, bcset=0),
         fv.residual(g, MIXED3, u, np.array([-0.2, 0.4, 0.9]), 0.05)),
    ]
    for tc, expect in cases:
        got, want = _pair(capi, dm, tc, ud)
        assert torch.equal(got, want)
        res = dm.to_host(got)
        assert np.linalg.norm(res - expect) <= tol * np.linalg.norm(expect)
    dm.free()


def test_noalloc_rejects_meshes_beyond_its_scratch(dev):
    capi, device = dev
    m = jittered_cube(48, seed=3)         # 663,552 cells: n_face + n_vert > 1,048,576 doubles
    dm = device.DeviceMesh(m, [{t: ("neumann", 0.0) for t in range(1, 7)}], prec="fp64")
    u = torch.ones(dm.n_cell, dtype=torch.float64, device="cuda")
    res = torch.empty_like(u)
    with pytest.raises(capi.FvgbError) as e:
        capi.fvgb_fv_residual_noalloc(dm.handle, capi.tcoef(diff=0.1), u, res)
    assert e.value.status == capi.FVGB_EINVAL and "scratch" in str(e.value)
    dm.free()


def test_noalloc_option_errors(dev):
    capi, device = dev
    m = jittered_cube(3, seed=5)
    dm = device.DeviceMesh(m, [MIXED3], prec="fp64")
    u = torch.ones(dm.n_cell, dtype=torch.float64, device="cuda")
    res = torch.empty_like(u)
    for recon, status in ((2, capi.FVGB_EINVAL), (-1, capi.FVGB_EINVAL), (1, capi.FVGB_EUNSUPPORTED)):
        with pytest.raises(capi.FvgbError) as e:
            capi.fvgb_fv_residual_noalloc(dm.handle, capi.tcoef(diff=0.1, recon=recon), u, res)
        assert e.value.status == status
    dm.free()
