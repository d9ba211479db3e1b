"""fvgb_fv_residual_noalloc, the residual entry point that allocates nothing, for callers
that cannot allocate device memory when they need a residual (a host program that hands
out device memory through its own pool, a time-critical loop that must not pay for
cudaMalloc). Its scratch is a fixed device array inside the library; this test checks,
through the C ABI, that it returns what fvgb_fv_residual returns, on two calls in a row
(the second call finds the first call's leftovers in the shared array), for FP64 and
FP32 meshes, and that an oversized mesh is refused with a clear error.

The file name makes pytest collect it last."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from synth.meshgen import jittered_cube, jittered_square  # noqa: E402


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


def rel(a, b):
    a = a.double().cpu().numpy(); b = b.double().cpu().numpy()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
@pytest.mark.parametrize("case", ["cube", "square"])
def test_noalloc_matches_residual_twice(dev, prec, tol, case):
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
        want = dm.empty(dm.n_cell)
        got = dm.empty(dm.n_cell).fill_(float("nan"))
        capi.fvgb_fv_residual(dm.handle, tc, u, want)
        capi.fvgb_fv_residual_noalloc(dm.handle, tc, u, got)
        torch.cuda.synchronize()
        assert torch.isfinite(got).all()
        assert rel(got, want) <= tol
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
