"""Pins of the oracle's multiplicity-weighted (vertex-factorised) least-squares gradient:
linear exactness with and without Dirichlet ghost points, a brute-force sum over the
vertices of each cell and the cells and Dirichlet faces around them, weighted least
squares through numpy's lstsq, and that the weighting matters (it differs from the
set-union gradient of Algorithm "grad")."""
import numpy as np

from oracle import ls
from synth.meshgen import jittered_cube, jittered_square
from tests.conftest import geometry_of

NEU3 = {t: ("neumann", 0.0) for t in range(1, 7)}


def test_linear_fields_are_exact():
    g = geometry_of(jittered_cube(5, seed=31))
    b = np.array([0.7, -1.3, 2.1])
    u = 0.5 + g.cen @ b
    assert np.abs(ls.ls_gradient_vertex(g, NEU3, u) - b).max() < 1e-12
    # Dirichlet ghost points carrying the same linear field (constant on z = 0, z = 1)
    v = 0.5 + 3.0 * g.cen[:, 2]
    bc = dict(NEU3)
    bc[5], bc[6] = ("dirichlet", 0.5), ("dirichlet", 3.5)
    assert np.abs(ls.ls_gradient_vertex(g, bc, v) - [0.0, 0.0, 3.0]).max() < 1e-11
    g2 = geometry_of(jittered_square(9, 3, 4))
    u2 = -1.0 + g2.cen @ np.array([2.0, 0.4])
    assert np.abs(ls.ls_gradient_vertex(g2, {t: ("wall", 0.0) for t in range(1, 5)}, u2) - [2.0, 0.4]).max() < 1e-12


def test_brute_force_vertex_sums_and_weighted_lstsq():
    g = geometry_of(jittered_cube(3, seed=32))
    bc = {1: ("dirichlet", 1.0), 2: ("neumann", 0.0), 3: ("wall", 0.0), 4: ("neumann", 0.0),
          5: ("dirichlet", -0.5), 6: ("neumann", 0.0)}
    rng = np.random.default_rng(7)
    u = rng.normal(size=g.n_cell)
    star = [[] for _ in range(g.n_vert)]
    for c, cell in enumerate(g.cells):
        for a in cell:
            star[a].append(c)
    gval = {t: val for t, (k, val) in bc.items() if k == "dirichlet"}
    dfaces = [[] for _ in range(g.n_vert)]
    for f in range(g.n_face):
        if g.face_R[f] < 0 and g.face_tag[f] in gval:
            for a in g.face_vert[f]:
                dfaces[a].append(f)
    got = ls.ls_gradient_vertex(g, bc, u)
    for i in range(g.n_cell):
        M = np.zeros((3, 3)); J = np.zeros(3); rows = []; rhs = []
        for a in g.cells[i]:
            for c in star[a]:
                if c == i:
                    continue
                d = g.cen[c] - g.cen[i]
                M += np.outer(d, d); J += d * (u[c] - u[i]); rows.append(d); rhs.append(u[c] - u[i])
            for f in dfaces[a]:
                d = g.xf[f] - g.cen[i]
                du = gval[g.face_tag[f]] - u[i]
                M += np.outer(d, d); J += d * du; rows.append(d); rhs.append(du)
        want = np.linalg.solve(M, J)
        assert np.abs(got[i] - want).max() <= 1e-12 * max(1.0, np.abs(want).max())
        # the same as the least-squares fit over the repeated rows
        fit = np.linalg.lstsq(np.array(rows), np.array(rhs), rcond=None)[0]
        assert np.abs(fit - want).max() <= 1e-10 * max(1.0, np.abs(want).max())


def test_weighting_differs_from_the_set_gradient():
    g = geometry_of(jittered_cube(4, seed=33))
    u = np.random.default_rng(8).normal(size=g.n_cell)
    a = ls.ls_gradient_vertex(g, NEU3, u)
    b = ls.ls_gradient(g, NEU3, u)
    assert np.linalg.norm(a - b) > 1e-3 * np.linalg.norm(b)
