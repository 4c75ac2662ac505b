"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds only input generation (initial fields, masks, random
populations).  It contains none of the method's arithmetic: equilibria,
collisions and boundary rules live in the CUDA library and, separately, in
the oracle.  Every generator is deterministic in its seed.

Workload recipes (the paper's own benchmarks use these shapes, Sec. III-IV):
  * acoustic pulse (D2Q9, periodic): rho = 1 + A exp(-ln2 r^2 / h^2), uniform u
  * Taylor-Green vortex, 2D and 3D (periodic)
  * cylinder in a channel (D2Q9): solid disc mask, uniform inflow, seeded
    transverse perturbation at t = 0
  * round jet (D3Q19): top-hat inlet profile on the x = 0 face
"""
from __future__ import annotations

import math

import numpy as np

MASK64 = (1 << 64) - 1


def splitmix64_np(x: np.ndarray) -> np.ndarray:
    """splitmix64 output function (Steele, Lea and Flood 2014) on uint64 arrays."""
    z = (x.astype(np.uint64) + np.uint64(0x9E3779B97F4A7C15))
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def u01_np(counter: np.ndarray) -> np.ndarray:
    """Counter-based uniform numbers in [0, 1): (splitmix64(c) >> 11) * 2^-53."""
    with np.errstate(over="ignore"):
        return (splitmix64_np(counter) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def gaussian_pulse_2d(n: int = 128, amp: float = 1e-3, half_width: float = 6.0,
                      u0=(0.05, 0.0)):
    """Acoustic pulse: rho = 1 + amp exp(-ln2 r^2 / hw^2) centred at (n/2, n/2).

    Returns (rho[ncell], u[ncell, 3]) in x-fastest cell order.
    """
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    r2 = (x - n / 2) ** 2 + (y - n / 2) ** 2
    rho = 1.0 + amp * np.exp(-math.log(2.0) * r2 / half_width ** 2)
    u = np.zeros((n * n, 3))
    u[:, 0] = u0[0]
    u[:, 1] = u0[1]
    return rho.reshape(-1), u


def plane_pulse_2d(nx: int = 256, ny: int = 4, amp: float = 1e-3, half_width: float = 6.0,
                   u0: float = 0.0):
    """Planar density pulse along x (uniform in y): two plane acoustic waves."""
    x = np.arange(nx)
    prof = 1.0 + amp * np.exp(-math.log(2.0) * (x - nx / 2) ** 2 / half_width ** 2)
    rho = np.tile(prof, ny)
    u = np.zeros((nx * ny, 3))
    u[:, 0] = u0
    return rho, u


def taylor_green_2d(n: int, u0: float = 0.01):
    """u = U0 (sin kx cos ky, -cos kx sin ky), rho = 1 - rho-correction-free, k = 2 pi / n."""
    k = 2 * math.pi / n
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    u = np.zeros((n * n, 3))
    u[:, 0] = (u0 * np.sin(k * x) * np.cos(k * y)).reshape(-1)
    u[:, 1] = (-u0 * np.cos(k * x) * np.sin(k * y)).reshape(-1)
    rho = np.ones(n * n)
    return rho, u


def double_shear_layer(n: int, U: float = 0.1, kappa: float = 80.0, delta: float = 0.05):
    """Periodic double shear layer on an n x n box (the classic stability test
    of lattice Boltzmann collision models): u_x = U tanh(kappa (y/n - 1/4))
    for y <= n/2 and U tanh(kappa (3/4 - y/n)) above, u_y = delta U
    sin(2 pi (x/n + 1/4)), rho = 1."""
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    yy = y / n
    ux = np.where(yy <= 0.5, U * np.tanh(kappa * (yy - 0.25)), U * np.tanh(kappa * (0.75 - yy)))
    u = np.zeros((n * n, 3))
    u[:, 0] = ux.reshape(-1)
    u[:, 1] = (delta * U * np.sin(2 * math.pi * (x / n + 0.25))).reshape(-1)
    return np.ones(n * n), u


def taylor_green_3d(n: int, u0: float = 0.01):
    """u = U0 (sin kx cos ky cos kz, -cos kx sin ky cos kz, 0), k = 2 pi / n."""
    k = 2 * math.pi / n
    c = np.arange(n)
    s1, c1 = np.sin(k * c), np.cos(k * c)  # separable: same products, evaluated left to right
    u = np.zeros((n ** 3, 3))
    u[:, 0] = ((u0 * s1)[None, None, :] * c1[None, :, None] * c1[:, None, None]).reshape(-1)
    u[:, 1] = ((-u0 * c1)[None, None, :] * s1[None, :, None] * c1[:, None, None]).reshape(-1)
    rho = np.ones(n ** 3)
    return rho, u


def cylinder_mask(nx: int, ny: int, xc: float, yc: float, diameter: float) -> np.ndarray:
    """uint8 mask, 1 where (x - xc)^2 + (y - yc)^2 <= R^2 (cell centres at integers)."""
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    r2 = (x - xc) ** 2 + (y - yc) ** 2
    return (r2 <= (diameter / 2.0) ** 2).astype(np.uint8).reshape(-1)


def uniform_flow_perturbed(nx: int, ny: int, U: float, seed: int, rel: float = 0.01,
                           nz: int = 1):
    """Uniform flow u = (U, 0, 0) plus a transverse u_y = rel U (2 U01 - 1).

    U01 is counter-based: counter = seed * 2^32 + cell.
    """
    n = nx * ny * nz
    cnt = (np.uint64(seed) << np.uint64(32)) + np.arange(n, dtype=np.uint64)
    rho = np.ones(n)
    u = np.zeros((n, 3))
    u[:, 0] = U
    u[:, 1] = rel * U * (2.0 * u01_np(cnt) - 1.0)
    return rho, u


def top_hat_profile(ny: int, nz: int, yc: float, zc: float, radius: float, U: float,
                    theta: float = 0.0):
    """Per-face-cell inlet velocity (ny*nz, 3) for the x faces.

    theta = 0: sharp top hat, (U, 0, 0) where r < radius.  theta > 0: the
    usual smoothed top hat U/2 (1 - tanh((r - radius) / (2 theta))) with
    shear-layer momentum thickness theta (cells).
    """
    z, y = np.meshgrid(np.arange(nz), np.arange(ny), indexing="ij")
    r = np.sqrt((y - yc) ** 2 + (z - zc) ** 2).reshape(-1)
    prof = np.zeros((ny * nz, 3))
    if theta > 0:
        prof[:, 0] = 0.5 * U * (1.0 - np.tanh((r - radius) / (2.0 * theta)))
    else:
        prof[:, 0] = np.where(r < radius, U, 0.0)
    return prof


def random_populations(weights: np.ndarray, ncell: int, seed: int, spread: float = 0.05):
    """Positive random populations f_i = w_i (1 + spread (2 U - 1)) around rest.

    ``weights`` is the lattice weight vector supplied by the caller; the
    result has shape (q, ncell) and is strongly off equilibrium (random
    second and third moments), which exercises every term of a collision.
    """
    rng = np.random.default_rng(seed)
    r = rng.random((len(weights), ncell))
    return np.asarray(weights)[:, None] * (1.0 + spread * (2.0 * r - 1.0))


def serving_requests(n: int = 512, seed: int = 5, rate_per_s: float = 8.0, steps_scale: float = 1.0,
                     sizes_2d=(64, 128, 256, 512, 1024), sizes_3d=(32, 48, 64, 96, 128, 192)):
    """Seeded stream of independent solve requests.

    Arrivals are a Poisson process of the given rate; half of the requests are
    D2Q9 periodic acoustic pulses of N^2 cells, half D3Q19 Taylor-Green
    vortices of N^3 cells (N uniform over the given sets), tau ~ U[0.52, 0.9],
    steps ~ U{500..5000} (times steps_scale), storage FP32 or FP16 50/50.
    Returns a list of dicts sorted by arrival time.
    """
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))
    out = []
    for k in range(n):
        is2d = rng.random() < 0.5
        N = int(rng.choice(sizes_2d if is2d else sizes_3d))
        steps = int(rng.integers(500, 5001))
        out.append({
            "arrival": float(t[k]),
            "lattice": 0 if is2d else 1,
            "extents": (N, N, 1) if is2d else (N, N, N),
            "tau": float(rng.uniform(0.52, 0.9)),
            "steps": max(1, int(round(steps * steps_scale))),
            "precision": 1 if rng.random() < 0.5 else 2,
        })
    return out


def request_initial_state(req: dict):
    """(rho, u) of a request: a Gaussian pulse (amplitude 1e-3, half-width N/20)
    on a fluid at rest in 2D, a Taylor-Green vortex (U0 = 0.02) in 3D."""
    N = req["extents"][0]
    if req["lattice"] == 0:
        return gaussian_pulse_2d(N, 1e-3, max(2.0, N / 20.0), (0.0, 0.0))
    return taylor_green_3d(N, 0.02)
