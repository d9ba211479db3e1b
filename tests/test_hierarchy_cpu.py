"""The library's aggregate hierarchy of the learned warm start (fvgb_mpnn_hierarchy, host
code, no GPU) against the oracle's rule: identical levels, parents and neighbour sets
(integer work, compared exactly), for one part and for an ensemble of parts, and the
argument checks."""
import numpy as np
import pytest

from synth.meshgen import jittered_cube
from oracle import mpnn
from tests.conftest import geometry_of


@pytest.fixture(scope="module")
def capi():
    from paper_2203_00925_gb300 import build
    build.build()
    from paper_2203_00925_gb300 import capi as c
    return c


def _same(lib_levels, ora_levels):
    assert len(lib_levels) == len(ora_levels)
    for (n, parent, nbr), lev in zip(lib_levels, ora_levels):
        assert n == lev.n
        assert np.array_equal(parent, lev.parent)
        want = [set() for _ in range(n)]
        for a, b in lev.pairs:
            want[a].add(b)
            want[b].add(a)
        for a in range(n):
            got = [int(x) for x in nbr[a] if x != a]
            assert len(got) == len(set(got)) and set(got) == want[a], a
            assert np.all(nbr[a][len(got):] == a)          # padding with the aggregate itself


@pytest.mark.parametrize("k,seed", [(4, 3), (6, 5), (11, 7)])
def test_hierarchy_matches_oracle(capi, k, seed):
    g = geometry_of(jittered_cube(k, seed=seed))
    _same(capi.fvgb_mpnn_hierarchy(g.cen), mpnn.hierarchy(g.cen))


def test_hierarchy_of_parts_matches_oracle(capi):
    cen = np.concatenate([geometry_of(jittered_cube(k, seed=s)).cen for k, s in ((5, 1), (3, 2), (8, 3), (1, 4))])
    nb = np.cumsum([0, 6 * 125, 6 * 27, 6 * 512, 6])
    lib = capi.fvgb_mpnn_hierarchy(cen, nb)
    _same(lib, mpnn.hierarchy(cen, nb))
    assert lib[-1][0] >= 4                   # a part of 6 cells stays one aggregate


def test_hierarchy_rejects_bad_arguments(capi):
    cen = geometry_of(jittered_cube(3, seed=1)).cen
    for pb in ([0, 100], [0, 0, 162], [0, 90, 80, 162]):
        with pytest.raises(capi.FvgbError):
            capi.fvgb_mpnn_hierarchy(cen, pb)
    bad = cen.copy()
    bad[5, 1] = np.nan
    with pytest.raises(capi.FvgbError):
        capi.fvgb_mpnn_hierarchy(bad)
