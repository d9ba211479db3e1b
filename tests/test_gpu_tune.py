"""Autotuned launch shapes change timing only: every shape gives the same bits."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from synth.meshgen import jittered_cube  # noqa: E402
from synth.workloads import StreamerCase  # noqa: E402


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_00925_gb300 import build
    build.build()
    from paper_2203_00925_gb300 import capi, device
    return capi, device


def _work(capi, dm, u0, vel0):
    u = u0.clone()
    capi.fvgb_fv_step(dm.handle, capi.tcoef(vel=vel0, diff=0.05, bcset=0), u, 1e-4, 3)
    g = dm.empty(3, dm.n_cell)
    capi.fvgb_gradient(dm.handle, 1, u, g)
    uv = dm.empty(dm.n_vert)
    capi.fvgb_vertex_values(dm.handle, 1, u, uv)
    torch.cuda.synchronize()
    return u, g, uv


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_shapes_do_not_change_results(dev, prec):
    capi, device = dev
    m = jittered_cube(9, seed=301)
    case = StreamerCase()
    dm = device.DeviceMesh(m, [case.bc_ne(), case.bc_phi()], prec=prec)
    rng = np.random.default_rng(0)
    u0 = dm.to_device(1.0 + rng.random(dm.n_cell))
    vel0 = dm.to_device(rng.normal(size=(3, dm.n_cell)))
    ref = _work(capi, dm, u0, vel0)
    shapes = capi.fvgb_autotune(dm.handle, force=True)
    assert shapes.shape == (4, 2)
    assert all(t in (128, 256, 512, 1024) and e in (1, 2, 4) for t, e in shapes)
    got = _work(capi, dm, u0, vel0)
    for a, b in zip(ref, got):
        assert torch.equal(a, b)
    for k in range(4):
        capi.fvgb_set_launch_shape(dm.handle, k, 32, 7)
    got = _work(capi, dm, u0, vel0)
    for a, b in zip(ref, got):
        assert torch.equal(a, b)
    # a second mesh of the same class takes the cached shapes
    dm2 = device.DeviceMesh(jittered_cube(9, seed=7), [case.bc_ne(), case.bc_phi()], prec=prec)
    assert np.array_equal(capi.fvgb_autotune(dm2.handle), shapes)
    with pytest.raises(capi.FvgbError):
        capi.fvgb_set_launch_shape(dm.handle, 2, 100, 1)
    dm.free()
    dm2.free()
