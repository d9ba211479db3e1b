"""Message-passing warm start for the Poisson solve (oracle, FP64; test infrastructure).

Not in the paper: the learned warm start of the synthetic workloads (3 layers, hidden
64) predicts the potential increment of a step from the change of the space charge and
the previous potential; the Poisson solve then starts from phi_prev + prediction.

Architecture (per cell i; fine messages over interior faces, weight w_ij = c1_f / max c1):
    f_i   = [ (e/eps0) dq_i mu_i^(2/3) / (V s0),  phi_prev_i / (V s1) ]
    h     = relu(W_enc f + b_enc)                                 (64)
    layer(l, h; graph): m_i = sum_j w_ij (h_j - h_i); z = W_l [h ; m] + b_l; h + relu(z)
    h     = layer(0, h; faces)
    middle layer, one of two architectures:
    local: h = layer(1, h; faces) (reach: three face hops in all);
    multilevel: the middle layer runs on a hierarchy of cubic aggregates (``hierarchy``),
    which gives the network the reach of the whole domain (the potential's increment is
    the global response to a local charge change):
        c_1 = mean over each level-1 aggregate of h;  c_k = mean over the level-k aggregate
        of c_{k-1};  at every level, before moving down, HOPS times c_k = layer(1, c_k;
        aggregate graph k), whose weights are 1/6 between face-adjacent aggregates
        (shared weights W_1, b_1 at every level and hop);
        then back up: c_{k-1} += c_k of its aggregate, down to h += c_1 of the cell's;
    h     = layer(2, h; faces)
    out_i = w_dec . h + b_dec = N(f)_i
    prediction delta phi_i = V s2 (N(f) - N(f with f0 = 0))_i  (the response to the charge
    change; the part the network would give for an unchanged charge is removed),
    loss = mean_i (pred_i - t_i)^2,  pred = N(f) - N(f0 = 0),  t_i = delta phi_i / (V s2).

Parameters are one flat vector (see ``layout``). ``forward`` keeps the activations,
``backward`` is the hand-derived gradient (message passing is symmetric, so its adjoint
is the same operator; the mean over an aggregate and the copy back are each other's
adjoints up to the aggregate's size). Pinned by central finite differences.

Aggregate hierarchy (per part, from the cell centres): with the part's bounding box
[lo, hi] of the centres and r_1 = max(1, round((n / 6)^(1/3))) boxes per axis, a cell's
level-1 box index per axis is min(r_1 - 1, floor((x - lo) / (hi - lo) * r_1)) (0 when
hi = lo); level k + 1 halves the box indices (r_{k+1} = ceil(r_k / 2)); aggregates are the
non-empty boxes, levels continue while r_k > 2 (the last level has r = 2 or less, or 1
box). Neighbours at a level: the non-empty boxes that share a face.
"""
from __future__ import annotations

import numpy as np

from . import fv

HIDDEN = 64
LAYERS = 3
HOPS = 2          # applications of the middle layer per aggregate level
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


class Level:
    """One aggregate level: parent[i] = aggregate of node i of the level below (cells for
    level 1), count[a] = nodes in aggregate a, and the face-adjacent pairs (a, b)."""

    def __init__(self, parent, n, pairs):
        self.parent = parent
        self.n = n
        self.count = np.bincount(parent, minlength=n).astype(np.float64)
        self.pairs = pairs


def hierarchy(cen, part_begin=None):
    """The aggregate levels of the cells with centres cen (one part per range of
    part_begin; the whole set by default), numbered part by part, boxes in increasing
    (x, y, z) index order within a part."""
    cen = np.asarray(cen, dtype=np.float64)
    n_all = cen.shape[0]
    part_begin = [0, n_all] if part_begin is None else list(part_begin)
    levels = []
    # level 1 box coordinates of every cell, per part
    coords, radii = [], []
    for p in range(len(part_begin) - 1):
        c = cen[part_begin[p]:part_begin[p + 1]]
        n = c.shape[0]
        r = max(1, int(np.round((n / 6.0) ** (1.0 / 3.0))))
        lo, hi = c.min(axis=0), c.max(axis=0)
        k = np.zeros((n, 3), dtype=np.int64)
        for a in range(3):
            if hi[a] > lo[a]:
                k[:, a] = np.minimum(r - 1, np.floor((c[:, a] - lo[a]) / (hi[a] - lo[a]) * r).astype(np.int64))
        coords.append(k)
        radii.append(r)
    first = True
    while True:
        if not first:
            if all(r <= 2 for r in radii):
                break
            coords = [k >> 1 for k in coords]
            radii = [(r + 1) // 2 for r in radii]
        first = False
        parent_parts, pairs, offset = [], [], 0
        new_coords = []
        for p, (k, r) in enumerate(zip(coords, radii)):
            key = (k[:, 0] * r + k[:, 1]) * r + k[:, 2]
            boxes, inv = np.unique(key, return_inverse=True)
            parent_parts.append(offset + inv.ravel())
            bx = np.stack([boxes // (r * r), (boxes // r) % r, boxes % r], axis=1)
            pos = {int(b): i for i, b in enumerate(boxes)}
            for i, (x, y, z) in enumerate(bx):
                for d in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
                    nx, ny, nz = x + d[0], y + d[1], z + d[2]
                    if nx < r and ny < r and nz < r:
                        j = pos.get(int((nx * r + ny) * r + nz))
                        if j is not None:
                            pairs.append((offset + i, offset + j))
            new_coords.append(bx)
            offset += boxes.size
        # parent of every node of the level below (cells for level 1, else the previous
        # level's aggregates, whose box coordinates were halved above)
        parent = np.concatenate(parent_parts)
        levels.append(Level(parent, offset, np.array(pairs, dtype=np.int64).reshape(-1, 2)))
        coords = new_coords
        if offset <= len(radii):
            break
    return levels


def level_messages(level, h):
    """m_a = (1/6) sum over the face-adjacent aggregates b of (h_b - h_a)."""
    m = np.zeros_like(h)
    if level.pairs.size:
        a, b = level.pairs[:, 0], level.pairs[:, 1]
        d = (h[b] - h[a]) / 6.0
        np.add.at(m, a, d)
        np.add.at(m, b, -d)
    return m


def restrict(level, h):
    """Mean over every aggregate of its nodes."""
    out = np.zeros((level.n, h.shape[1]))
    np.add.at(out, level.parent, h)
    return out / level.count[:, None]


def features(geo, dq, phi_prev, V, s0, s1):
    f0 = E_OVER_EPS0 * np.asarray(dq) * geo.vol ** (2.0 / 3.0) / (V * s0)
    f1 = np.asarray(phi_prev) / (V * s1)
    return np.stack([f0, f1], axis=1)


def network_graph(geo, part_begin=None, multilevel=True):
    """(fine face graph, aggregate levels or None for the local architecture)."""
    return message_graph(geo), hierarchy(geo.cen, part_begin) if multilevel else None


def sum_children(level, d):
    """Sum over every aggregate of its nodes' rows (adjoint of copying the aggregate's row
    back to its nodes)."""
    out = np.zeros((level.n, d.shape[1]))
    np.add.at(out, level.parent, d)
    return out


def _layer(p, l, h, msg):
    m = msg(h)
    z = np.concatenate([h, m], axis=1) @ p[f"W{l}"].T + p[f"b{l}"]
    return h + np.maximum(z, 0.0), (h, m, z)


def _layer_back(p, l, g, cache, d, msg):
    """Gradient through h_out = h + relu(W_l [h ; m(h)] + b_l); accumulates into g."""
    h, m, z = cache
    dz = d * (z > 0.0)
    g[f"W{l}"] = g.get(f"W{l}", 0.0) + dz.T @ np.concatenate([h, m], axis=1)
    g[f"b{l}"] = g.get(f"b{l}", 0.0) + dz.sum(axis=0)
    G = dz @ p[f"W{l}"]                        # [d/dh ; d/dm]
    return d + G[:, :HIDDEN] + msg(G[:, HIDDEN:])


def forward(net, theta, f):
    fine, levels = net
    p = unpack(theta)
    z0 = f @ p["W_enc"].T + p["b_enc"]
    h = np.maximum(z0, 0.0)
    cache = {"f": f, "z0": z0}
    h1, cache["l0"] = _layer(p, 0, h, lambda v: messages(fine, v))
    if levels is None:
        h2, cache["l1"] = _layer(p, 1, h1, lambda v: messages(fine, v))
        h3, cache["l2"] = _layer(p, 2, h2, lambda v: messages(fine, v))
        cache["h3"] = h3
        return h3 @ p["w_dec"] + p["b_dec"][0], cache
    # down the aggregate levels: mean, then HOPS middle layers per level
    x, down = h1, []
    for lev in levels:
        c = restrict(lev, x)
        hops = []
        for _ in range(HOPS):
            c, hc = _layer(p, 1, c, lambda v, lev=lev: level_messages(lev, v))
            hops.append(hc)
        down.append((c, hops))
        x = c
    # back up: every level adds its aggregate's value, down to the cells
    h2 = h1
    if levels:
        u = down[-1][0]
        for k in range(len(levels) - 1, 0, -1):
            u = down[k - 1][0] + u[levels[k].parent]
        h2 = h1 + u[levels[0].parent]
    cache["down"] = down
    h3, cache["l2"] = _layer(p, 2, h2, lambda v: messages(fine, v))
    cache["h3"] = h3
    out = h3 @ p["w_dec"] + p["b_dec"][0]
    return out, cache


def predict(net, theta, f):
    """N(f) - N(f with the charge feature zeroed)."""
    f_zero = f.copy()
    f_zero[:, 0] = 0.0
    return forward(net, theta, f)[0] - forward(net, theta, f_zero)[0]


def loss(net, theta, f, t):
    return float(np.mean((predict(net, theta, f) - t) ** 2))


def _backward_one(net, p, c, dout):
    """Gradient of sum_i dout_i N(f)_i for one forward cache."""
    fine, levels = net
    fmsg = lambda v: messages(fine, v)
    g = {}
    g["w_dec"] = c["h3"].T @ dout
    g["b_dec"] = np.array([dout.sum()])
    d = np.outer(dout, p["w_dec"])
    d = _layer_back(p, 2, g, c["l2"], d, fmsg)                  # d h2
    dh1 = d.copy()
    if levels is None:
        dh1 = _layer_back(p, 1, g, c["l1"], d, fmsg)
    elif levels:
        L = len(levels)
        dC = [None] * L
        du = sum_children(levels[0], d)
        for k in range(L):                                       # adjoint of the way up
            dC[k] = du
            if k + 1 < L:
                du = sum_children(levels[k + 1], du)
        for k in range(L - 1, -1, -1):                           # adjoint of the way down
            lev = levels[k]
            dk = dC[k]
            for hc in reversed(c["down"][k][1]):
                dk = _layer_back(p, 1, g, hc, dk, lambda v, lev=lev: level_messages(lev, v))
            back = dk[lev.parent] / lev.count[lev.parent][:, None]   # adjoint of the mean
            if k > 0:
                dC[k - 1] = dC[k - 1] + back
            else:
                dh1 = dh1 + back
    else:
        g["W1"] = np.zeros((HIDDEN, 2 * HIDDEN))
        g["b1"] = np.zeros(HIDDEN)
    d0 = _layer_back(p, 0, g, c["l0"], dh1, fmsg)
    dz0 = d0 * (c["z0"] > 0.0)
    g["W_enc"] = dz0.T @ c["f"]
    g["b_enc"] = dz0.sum(axis=0)
    return pack(g)


def backward(net, theta, f, t):
    """(loss, gradient of the loss with respect to the flat parameter vector)."""
    p = unpack(theta)
    f_zero = f.copy()
    f_zero[:, 0] = 0.0
    out_a, ca = forward(net, theta, f)
    out_b, cb = forward(net, theta, f_zero)
    pred = out_a - out_b
    dout = 2.0 * (pred - t) / pred.shape[0]
    grad = _backward_one(net, p, ca, dout) - _backward_one(net, p, cb, dout)
    return float(np.mean((pred - t) ** 2)), grad


def init_params(seed):
    """Uniform weights in +-1 / sqrt(fan_in) (the decoder vector too), zero biases, from
    numpy's PCG64 stream."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shape in layout():
        if name.startswith("W"):
            bound = 1.0 / np.sqrt(shape[1])
            p[name] = rng.uniform(-bound, bound, size=shape)
        elif name == "w_dec":
            p[name] = rng.uniform(-1.0 / np.sqrt(HIDDEN), 1.0 / np.sqrt(HIDDEN), size=shape)
        else:
            p[name] = np.zeros(shape)
    return pack(p)


def round_bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as FP64."""
    a = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((a + 0x7FFF + ((a >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)
