"""Stored values of the paper's worked example (Annex, 3D Poisson: P = 10 on x = 0,
0 on x = 1, Neumann elsewhere, exact P = 10 (1 - x)) against the oracle's direct solve.
The fixture's values are the Annex's closed form at the cell centres
(tests/golden/make_annex.py)."""
import numpy as np

from oracle import poisson
from tests.conftest import ANNEX_BC, geometry_of, load_annex


def test_annex_fixture_oracle_solve():
    mesh, expected = load_annex()
    g = geometry_of(mesh)
    np.testing.assert_allclose(g.cen[:, 0], 1.0 - expected / 10.0, rtol=0, atol=1e-15)
    P = poisson.solve(g, ANNEX_BC, np.zeros(g.n_cell))
    np.testing.assert_allclose(P, expected, rtol=0, atol=1e-11)
    # a flipped boundary value is seen: the fixture is not symmetric in x
    swapped = dict(ANNEX_BC)
    swapped[1], swapped[2] = ANNEX_BC[2], ANNEX_BC[1]
    assert np.abs(poisson.solve(g, swapped, np.zeros(g.n_cell)) - expected).max() > 1.0
