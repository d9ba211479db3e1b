"""Pins for the message-passing warm start oracle (CPU): the hand-derived gradient of the
multilevel network against central finite differences, the message operators against
their definitions on hand-checkable cases, and the aggregate hierarchy against the
lattice it must reproduce on an unjittered Kuhn mesh."""
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


def _fd_check(net, n_cell, seed):
    rng = np.random.default_rng(seed)
    f = rng.normal(size=(n_cell, 2))
    t = rng.normal(size=n_cell)
    theta = mpnn.init_params(3) + 0.05 * rng.normal(size=mpnn.n_params())
    L0, grad = mpnn.backward(net, theta, f, t)
    assert L0 == mpnn.loss(net, theta, f, t)
    idx = rng.choice(mpnn.n_params(), size=60, replace=False)
    # every block's first entry, and entries of the middle layer's message columns
    offs, o = [], 0
    for name, s in mpnn.layout():
        offs.append(o)
        if name == "W1":
            offs += [o + 64 + 5, o + 128 * 7 + 100]
        o += int(np.prod(s))
    idx = np.unique(np.concatenate([idx, offs]))
    eps = 1e-6
    for k in idx:
        tp = theta.copy(); tp[k] += eps
        tm = theta.copy(); tm[k] -= eps
        fd = (mpnn.loss(net, tp, f, t) - mpnn.loss(net, tm, f, t)) / (2 * eps)
        assert abs(fd - grad[k]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (k, fd, grad[k])


def test_gradient_matches_finite_differences():
    g = geometry_of(jittered_cube(4, seed=9))
    net = mpnn.network_graph(g)
    assert [l.n for l in net[1]] == [64, 8]             # two levels, HOPS layers on each
    _fd_check(net, g.n_cell, 0)


def test_gradient_matches_finite_differences_local():
    g = geometry_of(jittered_cube(3, seed=9))
    _fd_check(mpnn.network_graph(g, multilevel=False), g.n_cell, 4)


def test_gradient_matches_finite_differences_two_parts():
    """Two parts (the halves of the cell list): levels per part, three levels deep."""
    g = geometry_of(jittered_cube(6, seed=5))
    half = g.n_cell // 2
    net = mpnn.network_graph(g, [0, half, g.n_cell])
    assert len(net[1]) >= 2
    _fd_check(net, g.n_cell, 1)


def test_hierarchy_reproduces_the_lattice():
    """Unjittered Kuhn cube of k^3 cubes: the 6 tetrahedra of a cube form one level-1
    aggregate (r_1 = k); level k + 1 is the 2x2x2 blocks of level k; neighbours are the
    face-adjacent boxes, 3 r^2 (r - 1) pairs."""
    k = 8
    g = geometry_of(jittered_cube(k, seed=1, jitter=0.0))
    levels = mpnn.hierarchy(g.cen)
    assert [l.n for l in levels] == [512, 64, 8]
    assert np.all(levels[0].count == 6) and np.all(levels[1].count == 8) and np.all(levels[2].count == 8)
    for lev, r in zip(levels, (8, 4, 2)):
        assert lev.pairs.shape[0] == 3 * r * r * (r - 1)
    # a level-1 aggregate is one cube: its cells' centres lie in one cell of the lattice
    cube = np.floor(g.cen * k + 1e-9).astype(int)
    key = (cube[:, 0] * k + cube[:, 1]) * k + cube[:, 2]
    for a in range(levels[0].n):
        assert np.unique(key[levels[0].parent == a]).size == 1
    # neighbours at level 1 are the cubes one lattice step apart
    cub = np.zeros((512, 3), dtype=int)
    cub[levels[0].parent] = cube
    step = np.abs(cub[levels[0].pairs[:, 0]] - cub[levels[0].pairs[:, 1]]).sum(axis=1)
    assert np.all(step == 1)


def test_hierarchy_of_parts_keeps_parts_apart():
    g = geometry_of(jittered_cube(6, seed=5))
    nb = [0, 500, g.n_cell]
    levels = mpnn.hierarchy(g.cen, nb)
    lev1 = levels[0]
    part_of_cell = np.repeat([0, 1], np.diff(nb))
    part_of_agg = np.zeros(lev1.n, dtype=int)
    part_of_agg[lev1.parent] = part_of_cell
    # every aggregate is in one part, aggregates are numbered part by part
    for a in range(lev1.n):
        assert np.unique(part_of_cell[lev1.parent == a]).size == 1
    assert np.all(np.diff(part_of_agg) >= 0)
    assert np.all(part_of_agg[lev1.pairs[:, 0]] == part_of_agg[lev1.pairs[:, 1]])
    # the same hierarchy as each part on its own, offset
    alone = mpnn.hierarchy(g.cen[500:])
    assert np.array_equal(lev1.parent[500:] - lev1.parent[500], alone[0].parent)


def test_level_operators():
    """Mean over aggregates of a constant is the constant; messages of a constant are 0;
    the copy back and the child sum are adjoint; the level message operator is minus
    (1/6) the graph Laplacian of the aggregates."""
    g = geometry_of(jittered_cube(4, seed=2))
    lev = mpnn.hierarchy(g.cen)[0]
    rng = np.random.default_rng(3)
    c = np.full((g.n_cell, 3), 2.5)
    assert np.allclose(mpnn.restrict(lev, c), 2.5)
    assert np.abs(mpnn.level_messages(lev, np.ones((lev.n, 2)))).max() == 0.0
    u = rng.normal(size=(lev.n, 4))
    d = rng.normal(size=(g.n_cell, 4))
    assert np.isclose((u[lev.parent] * d).sum(), (u * mpnn.sum_children(lev, d)).sum())
    Adj = np.zeros((lev.n, lev.n))
    Adj[lev.pairs[:, 0], lev.pairs[:, 1]] = 1.0
    Adj[lev.pairs[:, 1], lev.pairs[:, 0]] = 1.0
    Lap = np.diag(Adj.sum(1)) - Adj
    assert np.allclose(mpnn.level_messages(lev, u), -(Lap @ u) / 6.0)


def test_network_reaches_the_whole_domain():
    """A charge change in one cell changes the prediction in every cell (the coarse
    levels carry it), while the local network reaches only the cells within three face
    hops."""
    g = geometry_of(jittered_cube(4, seed=9))
    net = mpnn.network_graph(g)
    theta = mpnn.init_params(7)
    rng = np.random.default_rng(2)
    f = rng.normal(size=(g.n_cell, 2))
    base = mpnn.forward(net, theta, f)[0]
    f2 = f.copy()
    f2[0, 0] += 1.0
    delta = np.abs(mpnn.forward(net, theta, f2)[0] - base)
    assert np.all(delta > 0.0)
    local = mpnn.network_graph(g, multilevel=False)
    delta_local = np.abs(mpnn.forward(local, theta, f2)[0] - mpnn.forward(local, theta, f)[0])
    # cells within three face hops of cell 0
    L, R, _ = local[0]
    near = {0}
    for _ in range(3):
        near |= {int(b) for a, b in zip(L, R) if a in near} | {int(a) for a, b in zip(L, R) if b in near}
    far = np.setdiff1d(np.arange(g.n_cell), sorted(near))
    assert far.size > 0 and np.all(delta_local[far] == 0.0) and np.any(delta_local > 0.0)


def test_layout_and_bf16_rounding():
    assert mpnn.n_params() == 2 * 64 + 64 + 3 * (64 * 128 + 64) + 64 + 1
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -3.14159, 1e-3])
    r = mpnn.round_bf16(x)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2 ** -7   # a tie goes to even; above it rounds up
    assert np.all(np.abs(r - x) <= 2 ** -8 * np.abs(x))
