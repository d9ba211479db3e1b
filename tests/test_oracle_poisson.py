"""Pins for the oracle's Poisson operator and solve (CPU)."""
import numpy as np
import pytest

from synth.meshgen import jittered_cube, jittered_square
from oracle import poisson
from tests.conftest import geometry_of

ANNEX = {1: ("dirichlet", 10.0), 2: ("dirichlet", 0.0), 3: ("neumann", 0.0),
         4: ("neumann", 0.0), 5: ("neumann", 0.0), 6: ("neumann", 0.0)}


def test_annex_laplace_is_exact():
    """Annex: Lap P = 0, P = 10 on x = 0 ("in"), 0 on x = 1 ("out"), Neumann
    elsewhere; exact solution 10 (1 - x), reproduced by a linear-exact scheme."""
    g = geometry_of(jittered_cube(6, seed=17))
    P = poisson.solve(g, ANNEX, np.zeros(g.n_cell))
    assert np.abs(P - 10.0 * (1.0 - g.cen[:, 0])).max() < 1e-11
    # the annex's error norm (cell-volume weighted L2) is round-off
    err = np.sqrt(np.sum(g.vol * (P - 10.0 * (1.0 - g.cen[:, 0])) ** 2))
    assert err < 1e-11


def test_direct_solve_matches_dense_lu_and_matrix_free():
    g = geometry_of(jittered_cube(3, seed=5))
    bc = {t: ("dirichlet", float(t)) for t in range(1, 7)}
    rng = np.random.default_rng(0)
    f = rng.normal(size=g.n_cell)
    x1 = poisson.solve(g, bc, f)
    x2 = poisson.solve(g, bc, f, dense=True)
    assert np.abs(x1 - x2).max() < 1e-11 * np.abs(x2).max()
    A = poisson.assemble(g, bc)
    x = rng.normal(size=g.n_cell)
    assert np.abs(A @ x - poisson.apply(g, bc, x)).max() < 1e-12 * np.abs(A @ x).max()
    assert poisson.relative_residual(g, bc, f, x1) < 1e-12


def test_operator_signs():
    """With all-Neumann faces constants are in the kernel of A; with Dirichlet faces
    the total of A 1 is the boundary two-point sum sum_f c1_f > 0 (every boundary
    vertex is then Dirichlet, so only u_R - u_L = -1 survives on those faces), the
    diagonal is positive and the spectrum lies in the right half-plane."""
    g = geometry_of(jittered_cube(3, seed=6))
    neu = {t: ("neumann", 0.0) for t in range(1, 7)}
    one = np.ones(g.n_cell)
    assert np.abs(poisson.apply(g, neu, one)).max() < 1e-13
    dirb = {t: ("dirichlet", 0.0) for t in range(1, 7)}
    y = poisson.apply(g, dirb, one)
    from oracle import fv
    c = fv.diamond_coefficients(g)
    assert y.sum() == pytest.approx(c[g.face_R < 0, 0].sum(), rel=1e-12)
    A = poisson.assemble(g, dirb).toarray()
    assert np.all(np.diag(A) > 0)
    ev = np.linalg.eigvals(A)
    assert ev.real.min() > 0


@pytest.mark.slow
def test_manufactured_second_order():
    """phi = sin(pi x) sin(pi y) sin(pi z), f = -3 pi^2 phi, phi = 0 on the boundary:
    the L2 error at the centroids falls at observed order close to 2."""
    errs = []
    for k in (4, 8, 16):
        g = geometry_of(jittered_cube(k, seed=31))
        ex = np.prod(np.sin(np.pi * g.cen), axis=1)
        P = poisson.solve(g, {t: ("dirichlet", 0.0) for t in range(1, 7)}, -3 * np.pi ** 2 * ex)
        errs.append(np.sqrt(np.sum(g.vol * (P - ex) ** 2)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders[-1] > 1.6, (errs, orders)


def test_2d_manufactured():
    """sin(pi x) sin(pi y) with zero Dirichlet data: every boundary vertex is
    Dirichlet, so the 2D vertex stencils with too few triangles for a linear fit
    (edge vertices with 2 triangles, which fall back to the mean) do not enter."""
    errs = []
    for n in (8, 16, 32):
        g = geometry_of(jittered_square(n, 7, 8))
        ex = np.sin(np.pi * g.cen[:, 0]) * np.sin(np.pi * g.cen[:, 1])
        P = poisson.solve(g, {t: ("dirichlet", 0.0) for t in range(1, 5)}, -2 * np.pi ** 2 * ex)
        errs.append(np.sqrt(np.sum(g.vol * (P - ex) ** 2)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders.min() > 1.6, (errs, orders)
