"""Synthetic workload recipes (inputs only, no method arithmetic).

The streamer workloads of the benchmark: a jittered Kuhn-tetrahedron unit cube, an
electron seed 1e16 exp(-r^2 / 0.01^2) + 1e9 at (0.5, 0.5, 0.9), n_i = n_e at t = 0,
potential 0 on z = 0 and V on z = 1 (homogeneous Neumann elsewhere), homogeneous
Neumann for n_e everywhere, mobility 0.0382, ionisation A exp(-B/|E|) with A = 4332,
B = 2e5, electron diffusivity 0.1 (SI units, lengths in metres).

The time step is an input: dt = 0.4 min(eps0 / (e mu n_max), h^2 / (6 D_e), h / (mu V))
from the recipe's parameters and the lattice spacing h, held fixed over a run.
"""
from __future__ import annotations

from dataclasses import dataclass

from .meshgen import TAG_X0, TAG_X1, TAG_Y0, TAG_Y1, TAG_Z0, TAG_Z1, gaussian, jittered_cube

E_CHARGE = 1.602176634e-19
EPS0 = 8.8541878128e-12


@dataclass
class StreamerCase:
    V: float = 12500.0
    mu: float = 0.0382
    A: float = 4332.0
    B: float = 2.0e5
    De: float = 0.1
    centre: tuple = (0.5, 0.5, 0.9)
    sigma: float = 0.01
    peak: float = 1e16
    background: float = 1e9

    def bc_ne(self):
        return {t: ("neumann", 0.0) for t in (TAG_X0, TAG_X1, TAG_Y0, TAG_Y1, TAG_Z0, TAG_Z1)}

    def bc_phi(self):
        bc = {t: ("neumann", 0.0) for t in (TAG_X0, TAG_X1, TAG_Y0, TAG_Y1)}
        bc[TAG_Z0] = ("dirichlet", 0.0)
        bc[TAG_Z1] = ("dirichlet", self.V)
        return bc

    def initial(self, mesh):
        ne = gaussian(mesh.vertex_mean(), self.centre, self.sigma, self.peak, self.background)
        return ne, ne.copy()

    def dt(self, h):
        n_max = self.peak + self.background
        return 0.4 * min(EPS0 / (E_CHARGE * self.mu * n_max), h * h / (6.0 * self.De),
                         h / (self.mu * self.V))


def streamer_mesh(k, seed=201):
    """Unit cube, k^3 jittered hexes x 6 Kuhn tetrahedra (6 k^3 cells)."""
    return jittered_cube(k, seed=seed)


def ensemble_cases(n_mesh=64, seed=5000, lo=20_000, hi=1_000_000):
    """The batched workload: n_mesh jittered Kuhn cubes with cell-count targets
    log-uniform in [lo, hi] (k_i = round((n_i / 6)^(1/3))), mesh seeds seed + i, and per
    case a seed position uniform in [0.3, 0.7]^2 x [0.8, 0.95] and a voltage uniform in
    [15, 25] kV drawn from the stream seeded by ``seed``."""
    import numpy as np
    from .meshgen import ensemble_sizes
    _, ks = ensemble_sizes(n_mesh, lo, hi, seed)
    rng = np.random.default_rng(seed + 1)
    cases = []
    for i, k in enumerate(ks):
        centre = (rng.uniform(0.3, 0.7), rng.uniform(0.3, 0.7), rng.uniform(0.8, 0.95))
        V = rng.uniform(15e3, 25e3)
        cases.append((int(k), seed + i, StreamerCase(V=V, centre=centre)))
    return cases
