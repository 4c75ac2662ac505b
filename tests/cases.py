"""Problem descriptions shared by the parity tests.

A ``Case`` is a plain description (lattice, extents, tau, faces, sponges,
noise, solids, initial state).  ``to_oracle`` configures the CPU oracle from
it and ``to_gpu`` configures liblbm through its C ABI, so that both sides
receive the same inputs without sharing any arithmetic.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

import oracle
from paper_1710_02065_gb300 import inputs

D2Q9, D3Q19, D3Q27 = 0, 1, 2
PERIODIC, VELOCITY, OUTFLOW, FREESLIP, PRESSURE = 0, 1, 2, 3, 4
CS = 1.0 / math.sqrt(3.0)


@dataclasses.dataclass
class Case:
    name: str
    lattice: int
    n: tuple
    tau: float
    faces: dict = dataclasses.field(default_factory=dict)       # face -> (kind, u, profile[, rho])
    sponges: dict = dataclasses.field(default_factory=dict)     # face -> (width, chi)
    rho_ref: float = 1.0
    u_ref: tuple = (0.0, 0.0, 0.0)
    noise: tuple = (0, 0.0)                                    # (seed, amplitude)
    solid: np.ndarray | None = None
    rho0: np.ndarray | None = None
    u0: np.ndarray | None = None
    f0: np.ndarray | None = None                               # explicit populations (q, ncell)
    radial: tuple | None = None                                # (center, r0, width, chi)

    @property
    def ncell(self):
        return int(np.prod(self.n))

    @property
    def q(self):
        return {D2Q9: 9, D3Q19: 19, D3Q27: 27}[self.lattice]


def to_oracle(c: Case):
    P = oracle.Problem(c.lattice, c.n, c.tau)
    for face, spec in c.faces.items():
        kind, u, prof = spec[:3]
        P.set_boundary(face, kind, u, prof, rho=spec[3] if len(spec) > 3 else 1.0)
    for face, (w, chi) in c.sponges.items():
        P.set_sponge(face, w, chi, c.rho_ref, c.u_ref)
    if c.radial is not None:
        P.set_radial_sponge(c.radial[0], c.radial[1], c.radial[2], c.radial[3], c.rho_ref, c.u_ref)
    P.rho_ref, P.u_ref = c.rho_ref, list(c.u_ref)
    P.noise_seed, P.noise_amp = c.noise
    if c.solid is not None:
        P.solid = c.solid
    if c.f0 is not None:
        f = np.array(c.f0, dtype=np.float64)
    else:
        f = P.equilibrium(c.rho0, c.u0)
    return P, f


def to_gpu(c: Case, precision, block=None):
    from paper_1710_02065_gb300 import lbm
    s = lbm.Solver(c.lattice, c.n, c.tau, precision)
    for face, spec in c.faces.items():
        kind, u, prof = spec[:3]
        if kind == PRESSURE:
            lbm.lbm_set_pressure(s.h, face, spec[3] if len(spec) > 3 else 1.0)
        else:
            lbm.lbm_set_boundary(s.h, face, kind, u, prof)
    for face, (w, chi) in c.sponges.items():
        lbm.lbm_set_sponge(s.h, face, w, chi, c.rho_ref, c.u_ref)
    if c.radial is not None:
        lbm.lbm_set_radial_sponge(s.h, c.radial[0], c.radial[1], c.radial[2], c.radial[3], c.rho_ref, c.u_ref)
    if c.noise[1] > 0:
        lbm.lbm_set_inlet_noise(s.h, c.noise[0], c.noise[1])
    if c.solid is not None:
        lbm.lbm_set_geometry(s.h, c.solid)
    if c.f0 is not None:
        s.set_populations(c.f0)
    else:
        s.set_state(c.rho0, c.u0)
    return s


# ---------------------------------------------------------------------------
# The workloads (sizes of the paper's benchmark adaptations, or scaled copies)
# ---------------------------------------------------------------------------
def acoustic_pulse(n=128, tau=0.6):
    """D2Q9 n^2 periodic Gaussian pulse (amplitude 1e-3, half-width 6) on u = (0.05, 0)."""
    rho, u = inputs.gaussian_pulse_2d(n, 1e-3, 6.0, (0.05, 0.0))
    return Case("acoustic_pulse", D2Q9, (n, n, 1), tau, rho0=rho, u0=u)


def taylor_green_3d(n=24, tau=0.7, u0=0.02, lattice=D3Q19):
    rho, u = inputs.taylor_green_3d(n, u0)
    return Case("tgv3d", lattice, (n, n, n), tau, rho0=rho, u0=u)


def cylinder(nx=1600, ny=800, diameter=40.0, xc=None, yc=None, Ma=0.2, Re=150.0, sponge=100,
             chi=0.5, seed=2):
    """D2Q9 cylinder: inflow on -x at U = Ma c_s, zero-gradient outflow behind
    a sponge on +x, y periodic, halfway bounce-back disc, +-1% seeded u_y."""
    U = Ma * CS
    nu = U * diameter / Re
    tau = 3 * nu + 0.5
    xc = nx / 4 if xc is None else xc
    yc = ny / 2 if yc is None else yc
    rho, u = inputs.uniform_flow_perturbed(nx, ny, U, seed)
    solid = inputs.cylinder_mask(nx, ny, xc, yc, diameter)
    u[solid == 1] = 0.0
    c = Case("cylinder", D2Q9, (nx, ny, 1), tau, rho0=rho, u0=u, solid=solid,
             rho_ref=1.0, u_ref=(U, 0.0, 0.0))
    c.faces = {0: (VELOCITY, (U, 0.0, 0.0), None), 1: (OUTFLOW, (0, 0, 0), None)}
    c.sponges = {1: (sponge, chi)}
    return c


def round_jet(nx=384, ny=256, nz=256, diameter=24.0, Ma=0.3, Re=1e4, sponge=32, chi=0.5, seed=3,
              noise=0.01):
    """D3Q19 round jet: top-hat inflow of the given diameter on -x at U = Ma c_s
    (tanh shear layer, momentum thickness D/40), ambient at rest, sponges and
    zero-gradient outflow on the five other faces."""
    U = Ma * CS
    nu = U * diameter / Re
    tau = 3 * nu + 0.5
    prof = inputs.top_hat_profile(ny, nz, ny / 2, nz / 2, diameter / 2, U, diameter / 40.0)
    n = nx * ny * nz
    c = Case("round_jet", D3Q19, (nx, ny, nz), tau, rho0=np.ones(n), u0=np.zeros((n, 3)),
             rho_ref=1.0, u_ref=(0.0, 0.0, 0.0), noise=(seed, noise))
    c.faces = {0: (VELOCITY, (0, 0, 0), prof)}
    for f in (1, 2, 3, 4, 5):
        c.faces[f] = (OUTFLOW, (0, 0, 0), None)
        c.sponges[f] = (sponge, chi)
    return c


def with_random_state(c: Case, seed=11, spread=0.05):
    """Replace the initial state by strongly off-equilibrium random populations."""
    _, _, _, w, _ = oracle.lattice(c.lattice)
    c.f0 = inputs.random_populations(w, c.ncell, seed, spread)
    return c


def cylinder_two_level(nxc=200, nyc=100, patch=(40, 30, 80, 40), diameter_c=10.0, xc=None, yc=None,
                       Ma=0.2, Re=150.0, sponge=25, chi=0.5, seed=2):
    """The cylinder workload on a 2:1 two-level grid: coarse box with inflow,
    sponge and outflow; a fine patch over coarse nodes X0..X0+Wc, Y0..Y0+Hc
    holding the cylinder (diameter 2 diameter_c fine cells).  tau from Re on
    the fine level (the cylinder's resolution), tau_c = (tau_f + 1/2) / 2.
    Returns (coarse Case, patch, fine rho, fine u, fine solid)."""
    X0, Y0, Wc, Hc = patch
    U = Ma * CS
    D_f = 2 * diameter_c
    tau_f = 3 * U * D_f / Re + 0.5
    tau_c = (tau_f + 0.5) / 2
    rho, u = inputs.uniform_flow_perturbed(nxc, nyc, U, seed)
    c = Case("cylinder2", D2Q9, (nxc, nyc, 1), tau_c, rho0=rho, u0=u, rho_ref=1.0, u_ref=(U, 0.0, 0.0))
    c.faces = {0: (VELOCITY, (U, 0.0, 0.0), None), 1: (OUTFLOW, (0, 0, 0), None)}
    c.sponges = {1: (sponge, chi)}
    nfx, nfy = 2 * Wc + 1, 2 * Hc + 1
    xc = (Wc // 2) if xc is None else xc
    yc = (Hc // 2) if yc is None else yc
    solid_f = inputs.cylinder_mask(nfx, nfy, 2 * xc, 2 * yc, D_f)
    rho_f, u_f = inputs.uniform_flow_perturbed(nfx, nfy, U, seed + 1)
    u_f[solid_f == 1] = 0.0
    return c, patch, rho_f, u_f, solid_f
