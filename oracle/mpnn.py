"""Message-passing warm start for the Poisson solve (oracle, FP64; test infrastructure).

Not in the paper: the learned warm start of the synthetic workloads (3 layers, hidden
64) predicts the potential increment of a step from the change of the space charge and
the previous potential; the Poisson solve then starts from phi_prev + prediction.

Architecture (per cell i; messages over interior faces, weight w_ij = c1_f / max c1):
    f_i   = [ (e/eps0) dq_i mu_i^(2/3) / (V s0),  phi_prev_i / (V s1) ]
    h0    = relu(W_enc f + b_enc)                                 (64)
    for l = 0, 1, 2:
        m_i   = sum_j w_ij (h_j - h_i)
        z     = W_l [h ; m] + b_l                                 (64 x 128)
        h     = h + relu(z)
    out_i = w_dec . h + b_dec = N(f)_i
    prediction delta phi_i = V s2 (N(f) - N(f with f0 = 0))_i  (the response to the charge
    change; the part the network would give for an unchanged charge is removed),
    loss = mean_i (pred_i - t_i)^2,  pred = N(f) - N(f0 = 0),  t_i = delta phi_i / (V s2).

Parameters are one flat vector (see ``layout``). ``forward`` keeps the activations,
``backward`` is the hand-derived gradient (message passing is symmetric, so its adjoint
is the same operator). Pinned by central finite differences.
"""
from __future__ import annotations

import numpy as np

from . import fv

HIDDEN = 64
LAYERS = 3
E_OVER_EPS0 = 1.602176634e-19 / 8.8541878128e-12


def layout():
    """(name, shape) of every parameter block in the flat vector, in order."""
    out = [("W_enc", (HIDDEN, 2)), ("b_enc", (HIDDEN,))]
    for l in range(LAYERS):
        out += [(f"W{l}", (HIDDEN, 2 * HIDDEN)), (f"b{l}", (HIDDEN,))]
    out += [("w_dec", (HIDDEN,)), ("b_dec", (1,))]
    return out


def n_params():
    return sum(int(np.prod(s)) for _, s in layout())


def unpack(theta):
    p, o = {}, 0
    for name, shape in layout():
        n = int(np.prod(shape))
        p[name] = np.asarray(theta[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return p


def pack(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in layout()])


def message_graph(geo):
    """Interior faces as (L, R, w) with w = c1 / max c1 (c1 = |S|^2 / (e1 . S))."""
    c = fv.diamond_coefficients(geo)
    inr = geo.face_R >= 0
    c1 = c[inr, 0]
    return geo.face_L[inr], geo.face_R[inr], c1 / c1.max()


def messages(graph, h):
    """m_i = sum_j w_ij (h_j - h_i) over the face neighbours j of i."""
    L, R, w = graph
    d = (h[R] - h[L]) * w[:, None]
    m = np.zeros_like(h)
    np.add.at(m, L, d)
    np.add.at(m, R, -d)
    return m


def features(geo, dq, phi_prev, V, s0, s1):
    f0 = E_OVER_EPS0 * np.asarray(dq) * geo.vol ** (2.0 / 3.0) / (V * s0)
    f1 = np.asarray(phi_prev) / (V * s1)
    return np.stack([f0, f1], axis=1)


def forward(graph, theta, f):
    p = unpack(theta)
    z0 = f @ p["W_enc"].T + p["b_enc"]
    h = np.maximum(z0, 0.0)
    cache = {"f": f, "z0": z0, "h": [h], "m": [], "z": []}
    for l in range(LAYERS):
        m = messages(graph, h)
        z = np.concatenate([h, m], axis=1) @ p[f"W{l}"].T + p[f"b{l}"]
        h = h + np.maximum(z, 0.0)
        cache["m"].append(m)
        cache["z"].append(z)
        cache["h"].append(h)
    out = h @ p["w_dec"] + p["b_dec"][0]
    return out, cache


def predict(graph, theta, f):
    """N(f) - N(f with the charge feature zeroed)."""
    f_zero = f.copy()
    f_zero[:, 0] = 0.0
    return forward(graph, theta, f)[0] - forward(graph, theta, f_zero)[0]


def loss(graph, theta, f, t):
    return float(np.mean((predict(graph, theta, f) - t) ** 2))


def _backward_one(graph, p, c, dout):
    """Gradient of sum_i dout_i N(f)_i for one forward cache."""
    g = {}
    g["w_dec"] = c["h"][-1].T @ dout
    g["b_dec"] = np.array([dout.sum()])
    dh = np.outer(dout, p["w_dec"])
    for l in reversed(range(LAYERS)):
        dz = dh * (c["z"][l] > 0.0)
        hm = np.concatenate([c["h"][l], c["m"][l]], axis=1)
        g[f"W{l}"] = dz.T @ hm
        g[f"b{l}"] = dz.sum(axis=0)
        G = dz @ p[f"W{l}"]                    # N x 128: [d/dh ; d/dm]
        dh = dh + G[:, :HIDDEN] + messages(graph, G[:, HIDDEN:])
    dz0 = dh * (c["z0"] > 0.0)
    g["W_enc"] = dz0.T @ c["f"]
    g["b_enc"] = dz0.sum(axis=0)
    return pack(g)


def backward(graph, theta, f, t):
    """(loss, gradient of the loss with respect to the flat parameter vector)."""
    p = unpack(theta)
    f_zero = f.copy()
    f_zero[:, 0] = 0.0
    out_a, ca = forward(graph, theta, f)
    out_b, cb = forward(graph, theta, f_zero)
    pred = out_a - out_b
    dout = 2.0 * (pred - t) / pred.shape[0]
    grad = _backward_one(graph, p, ca, dout) - _backward_one(graph, p, cb, dout)
    return float(np.mean((pred - t) ** 2)), grad


def init_params(seed):
    """Kaiming-uniform-like initialisation from numpy's PCG64 stream."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shape in layout():
        if name.startswith("W"):
            bound = np.sqrt(6.0 / shape[1])
            p[name] = rng.uniform(-bound, bound, size=shape)
        elif name == "w_dec":
            p[name] = rng.uniform(-np.sqrt(3.0 / HIDDEN), np.sqrt(3.0 / HIDDEN), size=shape)
        else:
            p[name] = np.zeros(shape)
    return pack(p)


def round_bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as FP64."""
    a = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((a + 0x7FFF + ((a >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)
