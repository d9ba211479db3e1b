"""Electron drift-diffusion coupled to Poisson (eq. 10) - oracle, test infrastructure.

System (eq. 10): dn_e/dt + div(n_e v_e) - div(D_e grad n_e) = S_e, dn_p/dt = S_e,
Lap V = -(e / eps)(n_p - n_e), E = -grad V, S_e = alpha |v_e| n_e.

The paper's electron velocity (eq. "velo") needs constants C1, C2 it does not give,
and its alpha/N (eq. "alphaN") carries a garbled constant; the synthetic workloads
replace them with (SI units, lengths in metres):

* v = -mu E with mu = 0.0382, alpha = A exp(-B / |E|), A = 4332, B = 2e5, alpha = 0
  where |E| = 0;
* D_e = 0.1 constant (the paper's eq. "diff" depends on the missing v_e law);
* homogeneous Neumann for n_e on every side (ghost = interior, no diffusive flux),
  Dirichlet V = 0 on z = 0 and V = V_applied on z = 1, homogeneous Neumann for V on
  the other sides;
* one explicit Euler step: solve Poisson with n^k, E = -grad V (least-squares cell
  gradient with the Dirichlet ghost points), fluxes and source with n_e^k, then
  n_e^{k+1} = n_e^k + dt R(n_e^k), n_p^{k+1} = n_p^k + dt S_e;
* the three-stage scheme of eq. 6 applies that update per stage, with the Poisson
  solve, the field and the source recomputed from the stage densities:
  n^(j) = n^k + alpha_j dt Res(n^(j-1)), alpha = (1/2, 1/2, 1), n^{k+1} = n^(3).

The ion density is written n_i here (the paper's n_p).

Plasma spots (Section 4, "Streamer Branching"): Gaussian sources of electron-ion pairs,
S_k(x) = S_0 exp(-|x - c_k|^2 / sigma^2), switched on at t_on for a given duration. The
paper prints the exponent without its minus sign; the reading is the decaying Gaussian
(the printed form grows without bound away from the spot). A spot adds to S_e, so it
enters both the n_e and the n_i equations of eq. 10 (the spot is quasi-neutral and the
charge balance is unchanged). Within a time step [t, t + dt] the spot contributes its
average over the step, S_k(x) |[t, t + dt] n [t_on, t_on + duration]| / dt, so that steps
of any length deposit the spot's exact total S_k(x) * duration; the three stages of eq. 6
all use that step average.
"""
from __future__ import annotations

import numpy as np

from . import fv, ls, poisson

E_CHARGE = 1.602176634e-19      # C
EPS0 = 8.8541878128e-12         # F/m


class Params:
    def __init__(self, V=12500.0, mu=0.0382, A=4332.0, B=2.0e5, De=0.1,
                 centre=(0.5, 0.5, 0.9), sigma=0.01, peak=1e16, background=1e9):
        self.V, self.mu, self.A, self.B, self.De = V, mu, A, B, De
        self.centre, self.sigma, self.peak, self.background = centre, sigma, peak, background


class Spot:
    """One plasma spot: source S_0 exp(-|x - centre|^2 / sigma^2) for t in
    [t_on, t_on + duration). The defaults are the paper's values (amplitude 1e25, width
    0.005, on at 1.26e-8 s for 0.5e-9 s)."""

    def __init__(self, centre, amplitude=1e25, sigma=0.005, t_on=1.26e-8, duration=0.5e-9):
        self.centre = np.asarray(centre, dtype=np.float64)
        self.amplitude, self.sigma = float(amplitude), float(sigma)
        self.t_on, self.duration = float(t_on), float(duration)


def spot_source(geo, spots, t, dt):
    """Per-cell source of the plasma spots averaged over the step [t, t + dt]."""
    S = np.zeros(geo.n_cell)
    for sp in spots:
        lo = max(t, sp.t_on)
        hi = min(t + dt, sp.t_on + sp.duration)
        if hi <= lo:
            continue
        r2 = ((geo.cen - sp.centre) ** 2).sum(axis=1)
        S += sp.amplitude * np.exp(-r2 / sp.sigma ** 2) * ((hi - lo) / dt)
    return S


def bc_phi(p):
    return {1: ("neumann", 0.0), 2: ("neumann", 0.0), 3: ("neumann", 0.0),
            4: ("neumann", 0.0), 5: ("dirichlet", 0.0), 6: ("dirichlet", p.V)}


def bc_ne():
    return {t: ("neumann", 0.0) for t in range(1, 7)}


def poisson_source(ne, ni):
    """f of Lap V = f: -(e / eps0)(n_i - n_e)."""
    return -(E_CHARGE / EPS0) * (np.asarray(ni) - np.asarray(ne))


def cell_physics(p, E, ne):
    """v = -mu E, S = alpha(|E|) |v| n_e with alpha = A exp(-B/|E|)."""
    En = np.sqrt((E * E).sum(axis=1))
    v = -p.mu * E
    with np.errstate(divide="ignore"):
        alpha = np.where(En > 0.0, p.A * np.exp(-p.B / np.where(En > 0.0, En, 1.0)), 0.0)
    S = alpha * p.mu * En * ne
    return v, S


def step(geo, p, ne, ni, dt, phi=None, dense=False, recon=0, alphas=(1.0,), spots=(), t=0.0):
    """One step of eq. 10 from time t; returns (ne, ni, phi, E, S) of the last stage.
    alphas = (1,) is explicit Euler, (0.5, 0.5, 1) the three stages of eq. 6 (Poisson solved
    per stage). A given phi replaces the first stage's solve. recon = 1 takes the
    convective face values of n_e from the MUSCL reconstruction (eq. 15). spots: plasma
    spots added to the source S (see ``spot_source``)."""
    bphi = bc_phi(p)
    ne0, ni0 = np.asarray(ne, dtype=np.float64), np.asarray(ni, dtype=np.float64)
    ne_k, ni_k = ne0, ni0
    S_spot = spot_source(geo, spots, t, dt) if spots else None
    for j, a in enumerate(alphas):
        if j > 0 or phi is None:
            phi = poisson.solve(geo, bphi, poisson_source(ne_k, ni_k), dense=dense)
        E = -ls.ls_gradient(geo, bphi, phi)
        v, S = cell_physics(p, E, ne_k)
        if S_spot is not None:
            S = S + S_spot
        R = fv.residual(geo, bc_ne(), ne_k, v, p.De, src=S, recon=recon)
        ne_k, ni_k = ne0 + a * dt * R, ni0 + a * dt * S
    return ne_k, ni_k, phi, E, S


def time_step(p, h):
    """dt = 0.4 min(dielectric relaxation eps0/(e mu n_max), diffusion h^2/(6 D_e),
    drift h/(mu V)), from the inputs only (held fixed over the run)."""
    n_max = p.peak + p.background
    return 0.4 * min(EPS0 / (E_CHARGE * p.mu * n_max), h * h / (6.0 * p.De), h / (p.mu * p.V))


def boundary_outflow(geo, p, ne, v):
    """Net n_e flux leaving through the boundary (homogeneous Neumann ghost)."""
    b = geo.face_R < 0
    vn = np.einsum("fi,fi->f", v[geo.face_L[b]], geo.S[b])
    return float((vn * ne[geo.face_L[b]]).sum())
