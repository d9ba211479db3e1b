"""Writes annex_laplace.txt: the Poisson example of the paper's Annex on a small seeded
mesh, with the expected cell values from the Annex's closed-form solution.

Annex: P = 10 on the inlet x = 0, P = 0 on the outlet x = 1, homogeneous Neumann on the
four other sides of the unit cube; the exact solution is P(x, y, z) = 10 (1 - x). The
expected value of each cell is that formula at the cell's centre (the mean of its four
vertices); the scheme is exact for linear solutions, so the discrete solution equals it.
The mesh comes from the seeded generator (jittered 3 x 3 x 3 Kuhn cube, seed 17).

    python tests/golden/make_annex.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from synth.meshgen import jittered_cube  # noqa: E402


def main():
    m = jittered_cube(3, seed=17)
    cen = m.xyz[m.cells].mean(axis=1)
    P = 10.0 * (1.0 - cen[:, 0])
    with open(os.path.join(HERE, "annex_laplace.txt"), "w") as fh:
        fh.write("# Annex (3D Poisson example): P = 10 on x = 0 (tag 1), P = 0 on x = 1 (tag 2),\n")
        fh.write("# homogeneous Neumann on tags 3-6; exact solution P = 10 (1 - x).\n")
        fh.write("# mesh: jittered_cube(3, seed=17); expected: the closed form at each cell centre\n")
        fh.write(f"vertices {m.n_vert}\n")
        for p in m.xyz:
            fh.write(" ".join(repr(float(c)) for c in p) + "\n")
        fh.write(f"cells {m.n_cell}\n")
        for c in m.cells:
            fh.write(" ".join(str(int(v)) for v in c) + "\n")
        fh.write(f"bfaces {m.bface_vert.shape[0]}\n")
        for f, t in zip(m.bface_vert, m.bface_tag):
            fh.write(" ".join(str(int(v)) for v in f) + f" {int(t)}\n")
        fh.write(f"expected {m.n_cell}\n")
        for v in P:
            fh.write(repr(float(v)) + "\n")


if __name__ == "__main__":
    main()
