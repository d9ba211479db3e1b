"""Learned warm start for the Poisson solve of the streamer step: data generation with
the plain solver, training with the library's own forward/backward/Adam kernels, and
evaluation against the plain warm start (the previous potential).

The network, its gradients and the optimiser run in libfvgb (fvgb_mpnn_*); this module
only orders the calls and keeps the training pairs on the device.
"""
from __future__ import annotations

import numpy as np
import torch

from . import capi

E_OVER_EPS0 = 1.602176634e-19 / 8.8541878128e-12


def init_params(seed, multilevel=True):
    """Seeded initial parameters (FP32), layout of fvgb_mpnn_set_params: weight matrices and
    the decoder vector uniform in +-b, biases zero; b = 1 / sqrt(fan_in) for the multilevel
    architecture (its middle layer is applied twice on every aggregate level and the levels'
    outputs are summed, so larger initial weights compound into outputs far above the
    targets), b = sqrt(6 / fan_in) for the local one (measured the better start for each)."""
    rng = np.random.default_rng(seed)
    blocks = [("W", 64, 2), ("b", 64, 0)]
    for _ in range(3):
        blocks += [("W", 64, 128), ("b", 64, 0)]
    blocks += [("W", 1, 64), ("b", 1, 0)]
    out = []
    for kind, n, fan in blocks:
        if kind == "W":
            bound = 1.0 / np.sqrt(fan) if multilevel else np.sqrt(6.0 / fan)
            out.append(rng.uniform(-bound, bound, size=(n, fan)).ravel())
        else:
            out.append(np.zeros(n))
    theta = np.concatenate(out).astype(np.float32)
    assert theta.size == capi.fvgb_mpnn_param_count()
    return theta


def streamer_run(dm, case, mesh, dt, steps, solve, warm=None, extrapolate=False, record=False,
                 graph=False, on_pair=None):
    """Run ``steps`` streamer steps of one case from its initial state (phi from 0).

    Returns per-step solve infos and, when ``record``, two lists of training pairs as FP64
    device tensors, built by the library from its warm-start history
    (fvgb_streamer_pair): (dq, phi_prev, dphi) for a start from the previous potential
    (steps 1..) and (d2q, phi_prev, dphi - dphi_prev) for a start from the linear
    extrapolation in time (steps 2..). With ``on_pair`` each pair is handed to
    on_pair(which, dq, phi_prev, dphi) instead, in buffers reused for the next pair.
    Recording keeps a warm-start history, so a recording run starts its solves from the
    extrapolation (the pairs are those of the converged trajectory either way)."""
    ne0, ni0 = case.initial(mesh)
    ne, ni = dm.to_device(ne0), dm.to_device(ni0)
    phi = torch.zeros(dm.n_cell, dtype=torch.float64, device=dm.device)
    keep = record or on_pair is not None
    sp = capi.streamer_params(mu=case.mu, A=case.A, B=case.B, De=case.De, dt=dt, solve=solve,
                              warm=warm, extrapolate=extrapolate or (keep and warm is None))
    capi.fvgb_streamer_reset(dm.handle)
    capi.fvgb_set_graph_mode(dm.handle, graph)
    infos, pairs = [], ([], [])
    bufs = [tuple(torch.empty_like(phi) for _ in range(3)) for _ in range(2)]
    for s in range(steps):
        infos += capi.fvgb_streamer_step(dm.handle, sp, ne, ni, phi, None, 1)
        if not keep:
            continue
        for which in (0, 1):
            if s < 1 + which:
                continue
            out = bufs[which] if on_pair is not None else tuple(torch.empty_like(phi) for _ in range(3))
            capi.fvgb_streamer_pair(dm.handle, which, phi, *out)
            if on_pair is not None:
                on_pair(which, *out)
            else:
                pairs[which].append(out)
    capi.fvgb_set_graph_mode(dm.handle, False)
    if record:
        return infos, pairs[0], pairs[1]
    return infos, []


def scales_for(pairs, V, n_cell):
    """Normalisation of inputs and target from the training pairs: RMS of the charge
    feature (with mu^(2/3) taken as the mean cell size squared), of phi / V, of dphi / V."""
    h2 = (1.0 / n_cell) ** (2.0 / 3.0)
    rq = float(torch.sqrt(torch.mean(torch.stack([torch.mean(p[0] ** 2) for p in pairs]))))
    rp = float(torch.sqrt(torch.mean(torch.stack([torch.mean(p[1] ** 2) for p in pairs]))))
    rd = float(torch.sqrt(torch.mean(torch.stack([torch.mean(p[2] ** 2) for p in pairs]))))
    s0 = max(E_OVER_EPS0 * rq * h2 / V, 1e-30)
    return s0, max(rp / V, 1e-30), max(rd / V, 1e-30)


def train(net, pairs, epochs=2, lr=1e-3, seed=0, log_every=0):
    """Adam over the pairs in a seeded random order; returns the loss history."""
    rng = np.random.default_rng(seed)
    hist = []
    for ep in range(epochs):
        for k, i in enumerate(rng.permutation(len(pairs))):
            dq, phi_prev, dphi = pairs[i]
            want = log_every and (k % log_every == 0)
            l = capi.fvgb_mpnn_train_step(net, dq, phi_prev, dphi, lr, want_loss=bool(want))
            if want:
                hist.append((ep, k, l))
    return hist


def mean_loss(net, pairs):
    return float(np.mean([capi.fvgb_mpnn_loss_grad(net, *p, want_grad=False)[0] for p in pairs]))


def _rms_scales(sums, count, V, n_cell):
    """Scales of fvgb_mpnn_set_scales from mean squares of dq, phi_prev, dphi."""
    h2 = (1.0 / n_cell) ** (2.0 / 3.0)
    rq, rp, rd = (float(torch.sqrt(x / count)) for x in sums)
    return max(E_OVER_EPS0 * rq * h2 / V, 1e-30), max(rp / V, 1e-30), max(rd / V, 1e-30)


# architecture of each network: the start from the previous potential needs the reach of
# the aggregate hierarchy (the increment is the global response to the charge change); the
# correction of the extrapolation does better with the local network (measured)
MULTILEVEL = {False: True, True: False}


def train_streaming(dm, mesh, cases, dt, steps, solve, V, lr=1e-3, lr_final=3e-4, seed=0,
                    log_every=25, log=None, multilevel=None):
    """Train the two networks of the learned start (start from the previous potential, and
    correction of the extrapolation) while the solver generates their pairs: one Adam step
    per pair, as each streamer step of each case produces it, so that no pair is stored.
    The normalisation scales come from a first run of cases[0]. The cases run in a seeded
    random order; the last third of them with the smaller learning rate. multilevel: the
    architecture per network ({extrapolated: bool}, default MULTILEVEL).

    Returns ({False: (theta, scales, multilevel), True: (...)}, info)."""
    arch = dict(MULTILEVEL if multilevel is None else multilevel)
    nets = {}
    sums = {w: [torch.zeros((), dtype=torch.float64, device=dm.device) for _ in range(3)] for w in (0, 1)}
    count = {0: 0, 1: 0}

    def acc(which, dq, pp, dp):
        for k, x in enumerate((dq, pp, dp)):
            sums[which][k] += torch.mean(x * x)
        count[which] += 1

    streamer_run(dm, cases[0], mesh, dt, steps, solve, on_pair=acc)
    scales = {w: _rms_scales(sums[w], count[w], V, dm.n_cell) for w in (0, 1)}
    for w in (0, 1):
        nets[w] = capi.fvgb_mpnn_create(dm.handle, 1, multilevel=arch[bool(w)])
        capi.fvgb_mpnn_set_params(nets[w], init_params(w, arch[bool(w)]))
        capi.fvgb_mpnn_set_scales(nets[w], V, *scales[w])
    order = np.random.default_rng(seed).permutation(len(cases))
    hist = {0: [], 1: []}
    n_pairs = {0: 0, 1: 0}
    for rank, ci in enumerate(order):
        rate = lr if rank < (2 * len(cases)) // 3 else lr_final

        def step(which, dq, pp, dp):
            want = n_pairs[which] % log_every == 0
            loss = capi.fvgb_mpnn_train_step(nets[which], dq, pp, dp, rate, want_loss=want)
            if want:
                hist[which].append(loss)
            n_pairs[which] += 1

        streamer_run(dm, cases[ci], mesh, dt, steps, solve, on_pair=step)
        if log:
            log(f"trained on case {rank + 1}/{len(cases)}")
    out = {}
    for w in (0, 1):
        out[bool(w)] = (capi.fvgb_mpnn_get_params(nets[w]), scales[w], arch[bool(w)])
        capi.fvgb_mpnn_free(nets[w])
    info = {"pairs_trained": {"previous_phi": n_pairs[0], "extrapolated": n_pairs[1]},
            "loss_first_last": {"previous_phi": [hist[0][0], hist[0][-1]] if hist[0] else None,
                                "extrapolated": [hist[1][0], hist[1][-1]] if hist[1] else None},
            "loss_history_every": log_every,
            "scales": {"previous_phi": scales[0], "extrapolated": scales[1]},
            "learning_rates": [lr, lr_final],
            "architecture": {"previous_phi": "multilevel" if arch[False] else "local",
                             "extrapolated": "multilevel" if arch[True] else "local"}}
    return out, info


def held_out_run(dm, mesh, case, dt, steps, solve, V, net=None, extrapolate=False, skip=2):
    """Steps of a held-out case with the learned start ``net`` = (theta, scales, multilevel) or without
    it; returns inner / outer iterations and device time summed over steps skip.., the
    largest relative residual and how many learned starts passed the residual check."""
    handle = None
    if net is not None:
        handle = capi.fvgb_mpnn_create(dm.handle, 1, multilevel=net[2])
        capi.fvgb_mpnn_set_params(handle, net[0])
        capi.fvgb_mpnn_set_scales(handle, V, *net[1])
    ne0, ni0 = case.initial(mesh)
    ne, ni = dm.to_device(ne0), dm.to_device(ni0)
    phi = torch.zeros(dm.n_cell, dtype=torch.float64, device=dm.device)
    sp = capi.streamer_params(mu=case.mu, A=case.A, B=case.B, De=case.De, dt=dt, solve=solve,
                              warm=handle, extrapolate=extrapolate)
    capi.fvgb_streamer_reset(dm.handle)
    capi.fvgb_set_graph_mode(dm.handle, False)
    capi.fvgb_streamer_step(dm.handle, sp, ne, ni, phi, None, skip)
    capi.fvgb_stats_get(dm.handle, reset=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    infos = capi.fvgb_streamer_step(dm.handle, sp, ne, ni, phi, None, steps - skip)
    e1.record()
    torch.cuda.synchronize()
    st = capi.fvgb_stats_get(dm.handle, reset=True)
    if handle is not None:
        capi.fvgb_mpnn_free(handle)
    return {"inner": sum(i["inner_its_total"] for i in infos), "outer": sum(i["outer_its"] for i in infos),
            "ms": e0.elapsed_time(e1), "max_rel_res": max(i["rel_res"] for i in infos),
            "accepted_steps": st["learned_kept"], "steps": len(infos)}
