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


def init_params(seed):
    """Seeded initial parameters (FP32): weight matrices uniform in +-sqrt(6 / fan_in),
    the decoder vector in +-sqrt(3 / 64), biases zero; layout of fvgb_mpnn_set_params."""
    rng = np.random.default_rng(seed)
    blocks = [("W", 64, 2), ("b", 64, 0)]
    for _ in range(3):
        blocks += [("W", 64, 128), ("b", 64, 0)]
    blocks += [("d", 64, 0), ("b", 1, 0)]
    out = []
    for kind, n, fan in blocks:
        if kind == "W":
            bound = np.sqrt(6.0 / fan)
            out.append(rng.uniform(-bound, bound, size=(n, fan)).ravel())
        elif kind == "d":
            out.append(rng.uniform(-np.sqrt(3.0 / 64), np.sqrt(3.0 / 64), size=n))
        else:
            out.append(np.zeros(n))
    theta = np.concatenate(out).astype(np.float32)
    assert theta.size == capi.fvgb_mpnn_param_count()
    return theta


def streamer_run(dm, case, mesh, dt, steps, solve, warm=None, extrapolate=False, record=False,
                 graph=False):
    """Run ``steps`` streamer steps of one case from its initial state (phi from 0).

    Returns per-step solve infos and, when ``record``, two lists of training pairs as FP64
    device tensors: (dq, phi_prev, dphi) for a start from the previous potential (steps
    1..) and (d2q, phi_prev, dphi - dphi_prev) for a start from the linear extrapolation in
    time (steps 2..), where dq is the change of n_i - n_e between step starts and d2q the
    change of dq."""
    ne0, ni0 = case.initial(mesh)
    ne, ni = dm.to_device(ne0), dm.to_device(ni0)
    phi = torch.zeros(dm.n_cell, dtype=torch.float64, device=dm.device)
    sp = capi.streamer_params(mu=case.mu, A=case.A, B=case.B, De=case.De, dt=dt, solve=solve,
                              warm=warm, extrapolate=extrapolate)
    capi.fvgb_streamer_reset(dm.handle)
    capi.fvgb_set_graph_mode(dm.handle, graph)
    infos, plain_pairs, extrap_pairs = [], [], []
    qh, ph = [], []          # charges at the last step starts, potentials of the last steps
    for s in range(steps):
        if record:
            qh = (qh + [ni.double() - ne.double()])[-3:]
        infos += capi.fvgb_streamer_step(dm.handle, sp, ne, ni, phi, None, 1)
        if record:
            ph = (ph + [phi.clone()])[-3:]
            if len(qh) >= 2:
                plain_pairs.append((qh[-1] - qh[-2], ph[-2], ph[-1] - ph[-2]))
            if len(qh) >= 3:
                extrap_pairs.append(((qh[-1] - qh[-2]) - (qh[-2] - qh[-3]), ph[-2],
                                     ph[-1] - 2.0 * ph[-2] + ph[-3]))
    capi.fvgb_set_graph_mode(dm.handle, False)
    if record:
        return infos, plain_pairs, extrap_pairs
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
