"""GPU message-passing warm start against the FP64 oracle: forward, loss and gradient of
the multilevel network (BF16 tensor-core products, so a BF16 tolerance) on a mesh with
three aggregate levels and on an ensemble of parts, training, and the gain of the learned
warm start over the previous potential on held-out streamer runs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from synth.meshgen import jittered_cube  # noqa: E402
from synth.workloads import StreamerCase, streamer_mesh  # noqa: E402
from oracle import mpnn as om  # noqa: E402
from tests.conftest import geometry_of  # noqa: E402


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_00925_gb300 import build
    build.build()
    from paper_2203_00925_gb300 import capi, device, learned
    return capi, device, learned


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _bf16_layers(theta):
    t = np.asarray(theta, dtype=np.float32).astype(np.float64)
    p = om.unpack(t)
    for l in range(om.LAYERS):
        p[f"W{l}"] = om.round_bf16(p[f"W{l}"])
    return om.pack(p)


@pytest.mark.parametrize("multilevel", [True, False])
def test_forward_loss_gradient_parity(dev, multilevel):
    capi, device, _ = dev
    m = jittered_cube(6, seed=21)
    g = geometry_of(m)
    case = StreamerCase()
    dm = device.DeviceMesh(m, [case.bc_ne(), case.bc_phi()])
    rng = np.random.default_rng(5)
    theta = (om.init_params(2) + 0.02 * rng.normal(size=om.n_params())).astype(np.float32)
    V, s0, s1, s2 = 1.0e4, 3.0e-6, 0.5, 1.0e-6
    dq = 1e9 * rng.normal(size=g.n_cell) * np.exp(-20 * ((g.cen - 0.5) ** 2).sum(1))
    phi = V * g.cen[:, 2] + 50.0 * rng.normal(size=g.n_cell)
    target = V * s2 * rng.normal(size=g.n_cell)
    net = capi.fvgb_mpnn_create(dm.handle, 1, multilevel=multilevel)
    capi.fvgb_mpnn_set_params(net, theta)
    capi.fvgb_mpnn_set_scales(net, V, s0, s1, s2)
    assert np.array_equal(capi.fvgb_mpnn_get_params(net), theta)
    dqd, phid, td = (dm.to_device(x, torch.float64) for x in (dq, phi, target))
    pred = torch.empty_like(dqd)
    capi.fvgb_mpnn_predict(net, dqd, phid, pred)
    loss, grad = capi.fvgb_mpnn_loss_grad(net, dqd, phid, td)
    torch.cuda.synchronize()
    graph = om.network_graph(g, multilevel=multilevel)
    assert not multilevel or len(graph[1]) == 3
    f = om.features(g, dq, phi, V, s0, s1)
    th = _bf16_layers(theta)
    want = V * s2 * om.predict(graph, th, f)
    assert rel(dm.to_host(pred), want) < 3e-2
    ol, og = om.backward(graph, th, f, target / (V * s2))
    assert loss == pytest.approx(ol, rel=3e-2)
    assert rel(grad, og) < 5e-2
    cos = float(np.dot(grad, og) / (np.linalg.norm(grad) * np.linalg.norm(og)))
    assert cos > 0.998
    # no charge change predicts no increment, exactly
    capi.fvgb_mpnn_predict(net, torch.zeros_like(dqd), phid, pred)
    torch.cuda.synchronize()
    assert torch.count_nonzero(pred).item() == 0
    capi.fvgb_mpnn_free(net)
    dm.free()


def test_ensemble_parity(dev):
    """Two meshes as one ensemble: the hierarchy is built per part (no aggregate and no
    message crosses between the meshes); message weights are normalised by the largest
    c1 of the whole ensemble."""
    from oracle import fv
    capi, device, _ = dev
    meshes = [jittered_cube(5, seed=31), jittered_cube(6, seed=32)]
    geos = [geometry_of(m) for m in meshes]
    case = StreamerCase()
    dm = device.DeviceMesh(meshes, [[case.bc_ne(), case.bc_phi()]] * 2, ensemble=True)
    nb = np.cumsum([0] + [g.n_cell for g in geos])
    assert list(dm.part_begin) == list(nb)
    L, R, c1 = [], [], []
    for g, o in zip(geos, nb):
        inr = g.face_R >= 0
        L.append(g.face_L[inr] + o)
        R.append(g.face_R[inr] + o)
        c1.append(fv.diamond_coefficients(g)[inr, 0])
    c1 = np.concatenate(c1)
    cen = np.concatenate([g.cen for g in geos])
    graph = ((np.concatenate(L), np.concatenate(R), c1 / c1.max()), om.hierarchy(cen, nb))
    rng = np.random.default_rng(8)
    theta = (om.init_params(4) + 0.02 * rng.normal(size=om.n_params())).astype(np.float32)
    V, s0, s1, s2 = 1.0e4, 3.0e-6, 0.5, 1.0e-6
    dq = 1e9 * rng.normal(size=nb[-1]) * np.exp(-20 * ((cen - 0.5) ** 2).sum(1))
    phi = V * cen[:, 2] + 50.0 * rng.normal(size=nb[-1])
    target = V * s2 * rng.normal(size=nb[-1])
    net = capi.fvgb_mpnn_create(dm.handle, 1)
    capi.fvgb_mpnn_set_params(net, theta)
    capi.fvgb_mpnn_set_scales(net, V, s0, s1, s2)
    dqd, phid, td = (dm.to_device(x, torch.float64) for x in (dq, phi, target))
    pred = torch.empty_like(dqd)
    capi.fvgb_mpnn_predict(net, dqd, phid, pred)
    loss, grad = capi.fvgb_mpnn_loss_grad(net, dqd, phid, td)
    torch.cuda.synchronize()
    f = np.concatenate([om.features(g, dq[a:b], phi[a:b], V, s0, s1) for g, a, b in zip(geos, nb[:-1], nb[1:])])
    th = _bf16_layers(theta)
    want = V * s2 * om.predict(graph, th, f)
    assert rel(dm.to_host(pred), want) < 3e-2
    ol, og = om.backward(graph, th, f, target / (V * s2))
    assert loss == pytest.approx(ol, rel=3e-2)
    cos = float(np.dot(grad, og) / (np.linalg.norm(grad) * np.linalg.norm(og)))
    assert rel(grad, og) < 5e-2 and cos > 0.998
    capi.fvgb_mpnn_free(net)
    dm.free()


def test_training_reduces_loss(dev):
    capi, device, _ = dev
    m = jittered_cube(6, seed=22)
    g = geometry_of(m)
    case = StreamerCase()
    dm = device.DeviceMesh(m, [case.bc_ne(), case.bc_phi()])
    rng = np.random.default_rng(1)
    dq = dm.to_device(1e9 * rng.normal(size=g.n_cell), torch.float64)
    phi = dm.to_device(1e4 * g.cen[:, 2], torch.float64)
    # a smooth target the network can fit
    tgt = dm.to_device(1e-2 * np.sin(3 * g.cen[:, 0]), torch.float64)
    net = capi.fvgb_mpnn_create(dm.handle, 1)
    capi.fvgb_mpnn_set_params(net, om.init_params(0).astype(np.float32))
    capi.fvgb_mpnn_set_scales(net, 1e4, 3e-6, 0.5, 1e-6)
    l0, _ = capi.fvgb_mpnn_loss_grad(net, dq, phi, tgt, want_grad=False)
    for _ in range(300):
        capi.fvgb_mpnn_train_step(net, dq, phi, tgt, 1e-3)
    l1, _ = capi.fvgb_mpnn_loss_grad(net, dq, phi, tgt, want_grad=False)
    assert l1 < 0.2 * l0
    capi.fvgb_mpnn_free(net)
    dm.free()


def test_learned_warm_start_beats_previous_potential(dev):
    """Train on streamer runs of the plain solver (18 seeds), evaluate on 2 held-out seed
    positions: the solves started from the learned guess take fewer CG iterations in total,
    every step still converged to 1e-8. The same on top of the start from the linear
    extrapolation in time, which alone saves most of the iterations. The first network is
    multilevel, the correction of the extrapolation local (the trainer's choice)."""
    capi, device, learned = dev
    k = 16
    mesh = streamer_mesh(k, 301)
    rng = np.random.default_rng(4000)
    cases = [StreamerCase(centre=(rng.uniform(0.3, 0.7), rng.uniform(0.3, 0.7), rng.uniform(0.8, 0.95)))
             for _ in range(20)]
    c0 = cases[0]
    dm = device.DeviceMesh(mesh, [c0.bc_ne(), c0.bc_phi()])
    dt = c0.dt(1.0 / k)
    solve = capi.solve_opts(rtol=1e-8)
    pairs_p, pairs_x = [], []
    for c in cases[:-2]:
        _, pp, px = learned.streamer_run(dm, c, mesh, dt, 100, solve, record=True)
        pairs_p += pp
        pairs_x += px
    nets = []
    for pairs, extrap in ((pairs_p, False), (pairs_x, True)):
        net = capi.fvgb_mpnn_create(dm.handle, 1, multilevel=learned.MULTILEVEL[extrap])
        capi.fvgb_mpnn_set_params(net, learned.init_params(0, learned.MULTILEVEL[extrap]))
        capi.fvgb_mpnn_set_scales(net, c0.V, *learned.scales_for(pairs, c0.V, dm.n_cell))
        for ep in range(4):
            learned.train(net, pairs, epochs=1, lr=1e-3 if ep < 3 else 3e-4, seed=ep)
        nets.append(net)
    variants = {"plain": dict(), "learned": dict(warm=nets[0]), "extrap": dict(extrapolate=True),
                "learned_extrap": dict(warm=nets[1], extrapolate=True)}
    inner = dict.fromkeys(variants, 0)
    outer = dict.fromkeys(variants, 0)
    for c in cases[-2:]:
        for name, kw in variants.items():
            a, _ = learned.streamer_run(dm, c, mesh, dt, 40, solve, **kw)
            assert all(i["rel_res"] <= 1e-8 for i in a), name
            inner[name] += sum(i["inner_its_total"] for i in a[2:])
            outer[name] += sum(i["outer_its"] for i in a[2:])
    print("held-out CG iterations (inner / outer):",
          {n: (inner[n], outer[n]) for n in variants})
    # the learned correction (in full where it lowers the residual, else residual-minimising
    # scaled) saves CG iterations both from the previous potential and on top of the
    # extrapolation; measured 17 % and 11 % on this mesh (Jacobi-scaled inner CG)
    assert inner["learned"] < 0.95 * inner["plain"], inner
    assert outer["learned"] <= outer["plain"], outer
    assert inner["extrap"] < 0.6 * inner["plain"], inner
    assert inner["learned_extrap"] < 0.95 * inner["extrap"], inner
    assert outer["learned_extrap"] <= outer["extrap"], outer
    for net in nets:
        capi.fvgb_mpnn_free(net)
    dm.free()


@pytest.mark.parametrize("multilevel,extrapolate", [(True, False), (False, True)])
def test_learned_start_graph_matches_host(dev, multilevel, extrapolate):
    """Streamer steps with the learned start: captured as graphs (the network's kernels
    inside the captured step) they give bitwise the results of host-driven steps."""
    capi, device, learned = dev
    m = jittered_cube(8, seed=41)
    case = StreamerCase()
    dm = device.DeviceMesh(m, [case.bc_ne(), case.bc_phi()], prec="mixed")
    net = capi.fvgb_mpnn_create(dm.handle, 1, multilevel=multilevel)
    capi.fvgb_mpnn_set_params(net, learned.init_params(3, multilevel))
    capi.fvgb_mpnn_set_scales(net, case.V, 1e-6, 0.6, 1e-5)
    sp = capi.streamer_params(mu=case.mu, A=case.A, B=case.B, De=case.De, dt=case.dt(1.0 / 8),
                              solve=capi.solve_opts(rtol=1e-8, prec=capi.FVGB_FP32), warm=net,
                              extrapolate=extrapolate)
    ne0, ni0 = case.initial(m)
    out = []
    for graph in (False, True):
        ne, ni = dm.to_device(ne0), dm.to_device(ni0)
        phi = torch.zeros(dm.n_cell, dtype=torch.float64, device="cuda")
        capi.fvgb_streamer_reset(dm.handle)
        capi.fvgb_set_graph_mode(dm.handle, graph)
        infos = capi.fvgb_streamer_step(dm.handle, sp, ne, ni, phi, None, 6)
        torch.cuda.synchronize()
        out.append((ne.clone(), ni.clone(), phi.clone(), [i["inner_its_total"] for i in infos]))
    capi.fvgb_set_graph_mode(dm.handle, False)
    assert out[0][3] == out[1][3]
    for a, b in zip(out[0][:3], out[1][:3]):
        assert torch.equal(a, b)
    capi.fvgb_mpnn_free(net)
    dm.free()


def test_learned_start_gain_750k(dev):
    """The configuration's recipe on the 750,000-cell mesh (50^3 x 6): both networks trained
    by the library while the solver generates their pairs (18 seed positions x 100 steps),
    then 2 held-out positions x 40 steps in mixed precision, every solve to 1e-8. The
    multilevel start from the previous potential takes at least 5 % fewer CG iterations
    than the previous potential (measured 45 % and 23 % in two builds whose FP32 transport
    summed in different orders, so that the training trajectories and the networks differ,
    and 11 % once the inner CG ran on the Jacobi-scaled operator, which alone took 17 % of
    the previous potential's iterations); the residual check keeps it on most steps. The local correction of the extrapolation
    is safeguarded: it may gain little (measured 6 % in both), but it costs no more than
    5 % of the extrapolation's iterations."""
    capi, device, learned = dev
    k = 50
    mesh = streamer_mesh(k, 301)
    rng = np.random.default_rng(4000)
    cases = [StreamerCase(centre=(rng.uniform(0.3, 0.7), rng.uniform(0.3, 0.7), rng.uniform(0.8, 0.95)))
             for _ in range(20)]
    c0 = cases[0]
    dm = device.DeviceMesh(mesh, [c0.bc_ne(), c0.bc_phi()], prec="mixed")
    assert dm.n_cell == 750_000
    dt = c0.dt(1.0 / k)
    gen = capi.solve_opts(rtol=1e-8, inner_rtol=0.2, prec=capi.FVGB_FP32, inner=2)
    nets, info = learned.train_streaming(dm, mesh, cases[:18], dt, 100, gen, c0.V)
    assert info["pairs_trained"]["previous_phi"] == 18 * 99
    solve = capi.solve_opts(rtol=1e-8, inner_rtol=0.2, prec=capi.FVGB_FP32)
    res = {}
    for name, kw in (("previous_phi", {}), ("learned", {"net": nets[False]}),
                     ("extrapolated", {"extrapolate": True}),
                     ("learned_extrapolated", {"net": nets[True], "extrapolate": True})):
        tot = {"inner": 0, "outer": 0, "kept": 0, "steps": 0}
        for c in cases[18:]:
            r = learned.held_out_run(dm, mesh, c, dt, 40, solve, V=c0.V, **kw)
            assert r["max_rel_res"] <= 1e-8, name
            tot["inner"] += r["inner"]
            tot["outer"] += r["outer"]
            tot["kept"] += r["accepted_steps"]
            tot["steps"] += r["steps"]
        res[name] = tot
    print("held-out, 750k cells:", res)
    assert res["learned"]["inner"] < 0.95 * res["previous_phi"]["inner"], res
    assert res["learned"]["kept"] >= 0.8 * res["learned"]["steps"], res
    assert res["learned_extrapolated"]["inner"] <= 1.05 * res["extrapolated"]["inner"], res
    dm.free()
