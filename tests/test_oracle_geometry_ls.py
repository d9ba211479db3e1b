"""Pins for the oracle's geometry and least-squares operators (CPU only).

Each check compares the oracle with something other than itself: closed forms,
invariants of the unit square/cube, or a library least-squares routine applied to
the stencil written out by hand.
"""
import numpy as np
import pytest

from synth.meshgen import jittered_cube, jittered_square
from oracle.geometry import Geometry, MeshError
from oracle import ls
from tests.conftest import geometry_of

ALL_NEUMANN_3D = {t: ("neumann", 0.0) for t in range(1, 7)}
ALL_NEUMANN_2D = {t: ("neumann", 0.0) for t in range(1, 5)}


def test_single_tet_closed_form():
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    cells = np.array([[0, 1, 2, 3]])
    bf = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]])
    g = Geometry(3, xyz, cells, bf, np.array([1, 2, 3, 4]))
    assert g.vol[0] == pytest.approx(1.0 / 6.0, abs=1e-16)
    assert np.allclose(g.cen[0], [0.25, 0.25, 0.25])
    # outward area vectors: the three axis faces have area 1/2, the slanted one sqrt(3)/2
    S = {tuple(fv): s for fv, s in zip(g.face_vert.tolist(), g.S)}
    assert np.allclose(S[(0, 1, 2)], [0, 0, -0.5])
    assert np.allclose(S[(0, 1, 3)], [0, -0.5, 0])
    assert np.allclose(S[(0, 2, 3)], [-0.5, 0, 0])
    assert np.allclose(S[(1, 2, 3)], [0.5, 0.5, 0.5])


@pytest.mark.parametrize("maker", [lambda: jittered_cube(5, seed=3), lambda: jittered_square(9, 4, 5)])
def test_volume_closure_orientation(maker):
    m = maker()
    g = geometry_of(m)
    assert abs(g.vol.sum() - 1.0) < 1e-14
    # sum of outward area vectors of every closed cell vanishes
    clo = np.zeros((g.n_cell, g.dim))
    for a in range(g.dim):
        clo[:, a] += np.bincount(g.face_L, weights=g.S[:, a], minlength=g.n_cell)
        inr = g.face_R >= 0
        clo[:, a] -= np.bincount(g.face_R[inr], weights=g.S[inr, a], minlength=g.n_cell)
    assert np.abs(clo).max() < 1e-15
    inr = g.face_R >= 0
    assert np.all(np.einsum("fi,fi->f", g.S[inr], g.cen[g.face_R[inr]] - g.cen[g.face_L[inr]]) > 0)
    # face counts of the recipe
    if g.dim == 3:
        k = 5
        assert g.n_cell == 6 * k ** 3 and g.n_face == 12 * k ** 3 + 6 * k ** 2
        assert (~inr).sum() == 12 * k ** 2
    # total boundary area of the unit cube/square
    assert abs(np.linalg.norm(g.S[~inr], axis=1).sum() - 2 * g.dim) < 1e-13


def test_mesh_errors():
    m = jittered_cube(2, seed=1)
    bad = m.cells.copy()
    bad[0, [1, 2]] = bad[0, [2, 1]]
    with pytest.raises(MeshError):
        Geometry(3, m.xyz, bad, m.bface_vert, m.bface_tag)
    with pytest.raises(MeshError):
        Geometry(3, m.xyz, m.cells, m.bface_vert[1:], m.bface_tag[1:])
    bad = m.cells.copy(); bad[3, 0] = m.xyz.shape[0]
    with pytest.raises(MeshError):
        Geometry(3, m.xyz, bad, m.bface_vert, m.bface_tag)


@pytest.mark.parametrize("dim", [2, 3])
def test_ls_gradient_linear_exact(dim):
    m = jittered_cube(5, seed=9) if dim == 3 else jittered_square(10, 1, 2)
    g = geometry_of(m)
    rng = np.random.default_rng(0)
    b = rng.normal(size=dim)
    u = 0.7 + g.cen @ b
    bc = ALL_NEUMANN_3D if dim == 3 else ALL_NEUMANN_2D
    gr = ls.ls_gradient(g, bc, u)
    assert np.abs(gr - b).max() < 1e-12 * np.abs(b).max()
    # Dirichlet ghost points at x=0 and x=1 consistent with u = 0.7 + 2.5 x
    bcd = dict(bc); bcd[1] = ("dirichlet", 0.7); bcd[2] = ("dirichlet", 0.7 + 2.5)
    gr = ls.ls_gradient(g, bcd, 0.7 + 2.5 * g.cen[:, 0])
    want = np.zeros(dim); want[0] = 2.5
    assert np.abs(gr - want).max() < 1e-12


def test_ls_gradient_matches_lstsq_stencil():
    """Against numpy's least-squares solver on the stencil written out cell by cell."""
    m = jittered_cube(3, seed=5)
    g = geometry_of(m)
    bc = dict(ALL_NEUMANN_3D); bc[6] = ("dirichlet", 1.5)
    rng = np.random.default_rng(1)
    u = rng.normal(size=g.n_cell)
    gr = ls.ls_gradient(g, bc, u)
    cellsets = [set(c) for c in g.cells.tolist()]
    top = [f for f in range(g.n_face) if g.face_R[f] < 0 and g.face_tag[f] == 6]
    for i in range(g.n_cell):
        rows, rhs = [], []
        for j in range(g.n_cell):
            if j != i and cellsets[i] & cellsets[j]:
                rows.append(g.cen[j] - g.cen[i]); rhs.append(u[j] - u[i])
        for f in top:
            if cellsets[i] & set(g.face_vert[f].tolist()):
                rows.append(g.xf[f] - g.cen[i]); rhs.append(1.5 - u[i])
        sol = np.linalg.lstsq(np.array(rows), np.array(rhs), rcond=None)[0]
        assert np.allclose(gr[i], sol, rtol=1e-10, atol=1e-10)


def test_vertex_interpolation_pins():
    m = jittered_cube(4, seed=2)
    g = geometry_of(m)
    A, c, alpha = ls.vertex_weights(g)
    # weights sum to one at every vertex (constants are reproduced)
    assert np.abs(np.bincount(A, weights=alpha) - 1.0).max() < 1e-12
    # library least squares (fit of a + b.(x - x_A)) on every vertex star
    rng = np.random.default_rng(3)
    u = rng.normal(size=g.n_cell)
    uv = ls.vertex_values(g, ALL_NEUMANN_3D, u)
    n = np.bincount(A, minlength=g.n_vert)
    nondeg = 0
    for v in range(g.n_vert):
        cs = c[A == v]
        X = np.concatenate([np.ones((cs.size, 1)), g.cen[cs] - g.xyz[v]], axis=1)
        if cs.size < 4 or np.linalg.matrix_rank(X) < 4:
            assert uv[v] == pytest.approx(u[cs].mean(), rel=1e-12, abs=1e-12)
            continue
        nondeg += 1
        sol = np.linalg.lstsq(X, u[cs], rcond=None)[0]
        assert uv[v] == pytest.approx(sol[0], rel=1e-9, abs=1e-10)
    assert nondeg > 0.9 * g.n_vert
    # linear fields are reproduced at non-degenerate vertices; Dirichlet vertices take g
    b = np.array([1.0, -2.0, 0.5])
    uv = ls.vertex_values(g, ALL_NEUMANN_3D, 0.3 + g.cen @ b)
    ok = n >= 4
    assert np.abs(uv[ok] - (0.3 + g.xyz[ok] @ b)).max() < 1e-12
    bcd = dict(ALL_NEUMANN_3D); bcd[5] = ("dirichlet", -4.0); bcd[1] = ("dirichlet", 9.0)
    mask, val = ls.dirichlet_vertices(g, bcd)
    assert np.all(mask == ((np.abs(g.xyz[:, 2]) < 1e-15) | (np.abs(g.xyz[:, 0]) < 1e-15)))
    # smallest tag wins on the shared edge x = 0, z = 0
    edge = (np.abs(g.xyz[:, 2]) < 1e-15) & (np.abs(g.xyz[:, 0]) < 1e-15)
    assert np.all(val[edge] == 9.0)
