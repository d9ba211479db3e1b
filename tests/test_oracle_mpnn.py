"""Pins for the message-passing warm start oracle (CPU): the hand-derived gradient
against central finite differences, and the message operator against its definition
on a hand-checkable case."""
import numpy as np

from synth.meshgen import jittered_cube
from oracle import mpnn
from tests.conftest import geometry_of


def test_messages_of_constant_and_linear_fields():
    g = geometry_of(jittered_cube(3, seed=4))
    graph = mpnn.message_graph(g)
    h = np.ones((g.n_cell, 5))
    assert np.abs(mpnn.messages(graph, h)).max() == 0.0        # constants carry no message
    # the message operator is minus a weighted graph Laplacian: symmetric, rows sum to 0
    N = g.n_cell
    M = np.stack([mpnn.messages(graph, np.eye(N)[:, [k]])[:, 0] for k in range(N)], axis=1)
    assert np.allclose(M, M.T) and np.abs(M.sum(axis=1)).max() < 1e-12
    L, R, w = graph
    assert w.max() == 1.0 and np.all(w > 0)
    i, j = L[0], R[0]
    e = np.zeros((N, 1)); e[j] = 1.0
    assert mpnn.messages(graph, e)[i, 0] == w[0]


def test_gradient_matches_finite_differences():
    g = geometry_of(jittered_cube(3, seed=9))
    graph = mpnn.message_graph(g)
    rng = np.random.default_rng(0)
    f = rng.normal(size=(g.n_cell, 2))
    t = rng.normal(size=g.n_cell)
    theta = mpnn.init_params(3) + 0.05 * rng.normal(size=mpnn.n_params())
    L0, grad = mpnn.backward(graph, theta, f, t)
    assert L0 == mpnn.loss(graph, theta, f, t)
    idx = rng.choice(mpnn.n_params(), size=60, replace=False)
    # include every block's first entry
    offs, o = [], 0
    for _, s in mpnn.layout():
        offs.append(o); o += int(np.prod(s))
    idx = np.unique(np.concatenate([idx, offs]))
    eps = 1e-6
    for k in idx:
        tp = theta.copy(); tp[k] += eps
        tm = theta.copy(); tm[k] -= eps
        fd = (mpnn.loss(graph, tp, f, t) - mpnn.loss(graph, tm, f, t)) / (2 * eps)
        assert abs(fd - grad[k]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (k, fd, grad[k])


def test_layout_and_bf16_rounding():
    assert mpnn.n_params() == 2 * 64 + 64 + 3 * (64 * 128 + 64) + 64 + 1
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -3.14159, 1e-3])
    r = mpnn.round_bf16(x)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2 ** -7   # a tie goes to even; above it rounds up
    assert np.all(np.abs(r - x) <= 2 ** -8 * np.abs(x))
