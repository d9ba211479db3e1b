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


ANNEX_BC = {1: ("dirichlet", 10.0), 2: ("dirichlet", 0.0), 3: ("neumann", 0.0),
            4: ("neumann", 0.0), 5: ("neumann", 0.0), 6: ("neumann", 0.0)}


def load_annex():
    """The Annex Poisson example fixture: (mesh, expected cell values P = 10 (1 - x))."""
    import numpy as np
    from synth.meshgen import Mesh
    path = os.path.join(ROOT, "tests", "golden", "annex_laplace.txt")
    lines = [ln for ln in open(path) if not ln.startswith("#")]
    pos = 0

    def block():
        nonlocal pos
        n = int(lines[pos].split()[1])
        rows = [ln.split() for ln in lines[pos + 1:pos + 1 + n]]
        pos += 1 + n
        return rows

    xyz = np.array(block(), dtype=np.float64)
    cells = np.array(block(), dtype=np.int32)
    bf = np.array(block(), dtype=np.int64)
    expected = np.array(block(), dtype=np.float64).ravel()
    mesh = Mesh(3, xyz, cells, bf[:, :3].astype(np.int32), bf[:, 3].astype(np.int32), 1.0 / 3)
    return mesh, expected
