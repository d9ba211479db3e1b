import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def cube6():
    from synth.meshgen import jittered_cube
    return jittered_cube(6, seed=7)


@pytest.fixture(scope="session")
def square12():
    from synth.meshgen import jittered_square
    return jittered_square(12, seed_jitter=11, seed_diag=12)


def geometry_of(m):
    from oracle.geometry import Geometry
    return Geometry(m.dim, m.xyz, m.cells, m.bface_vert, m.bface_tag)
