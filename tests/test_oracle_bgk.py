"""Pins of the oracle's plain LBM-BGK collision (Eq. standardLB with the
quadratic equilibrium Eq. truncatedEq), the A/B counterpart of rrBGK.

  * the quadratic equilibrium carries rho, rho u and Pi = rho c_s^2 I + rho u u
    (tau = 1 returns it), and its third moment lacks the rho u u u term that
    rrBGK's equilibrium carries: the difference of the two at tau = 1 has
    exactly the moments rho u_a u_b u_c on the supported components
  * collision invariants: rho, rho u are conserved for any tau
  * relaxation: f* - f^eq = (1 - 1/tau)(f - f^eq) on every direction
  * a non-hydrodynamic (ghost) component of f survives BGK scaled by
    (1 - 1/tau) and is removed by the regularized collision
  * Taylor-Green decay at nu = c_s^2 (tau - 1/2)
"""
import math

import numpy as np
import pytest

import oracle
from oracle import BGK, D2Q9, D3Q19, RR
from paper_1710_02065_gb300 import inputs

CS2 = 1.0 / 3.0


def _one_cell(lattice, tau, model):
    """A single periodic cell: streaming is the identity, so one update is
    one collision."""
    P = oracle.Problem(lattice, (1, 1, 1) if lattice == D3Q19 else (1, 1), tau)
    P.collision = model
    return P


def _random_f(lattice, seed, spread=0.1):
    _, q, _, w, _ = oracle.lattice(lattice)
    rng = np.random.default_rng(seed)
    return w * (1.0 + spread * (2 * rng.random(q) - 1)) * 1.02


def _moments(lattice, f):
    _, q, xi, _, _ = oracle.lattice(lattice)
    rho = f.sum()
    j = (f[:, None] * xi).sum(0)
    Pi = np.einsum("i,ia,ib->ab", f, xi, xi)
    Q = np.einsum("i,ia,ib,ic->abc", f, xi, xi, xi)
    return rho, j, Pi, Q


@pytest.mark.parametrize("lattice", [D2Q9, D3Q19])
def test_quadratic_equilibrium_moments_and_missing_third_order(lattice):
    d = 2 if lattice == D2Q9 else 3
    for seed in range(4):
        f = _random_f(lattice, seed)
        feq_bgk = _one_cell(lattice, 1.0, BGK).update_cell(f, 0)
        feq_rr = _one_cell(lattice, 1.0, RR).update_cell(f, 0)
        rho, j, _, _ = _moments(lattice, f)
        u = j / rho
        r2, j2, Pi2, Q2 = _moments(lattice, feq_bgk)
        assert abs(r2 - rho) < 1e-15 and np.abs(j2 - j).max() < 1e-15
        Pi_expect = rho * CS2 * np.eye(3) + rho * np.outer(u, u)
        Pi_expect[d:, :] = 0
        Pi_expect[:, d:] = 0
        assert np.abs(Pi2 - Pi_expect).max() < 1e-15
        # the rrBGK equilibrium adds rho u_a u_b u_c on the third-order
        # components the lattice supports (a a b with a != b; D3Q19 keeps
        # them as the sums and differences of its three pairs)
        dQ = _moments(lattice, feq_rr)[3] - Q2
        uuu = rho * np.einsum("a,b,c->abc", u, u, u)
        if lattice == D2Q9:
            for a, b in ((0, 1), (1, 0)):
                assert abs(dQ[a, a, b] - uuu[a, a, b]) < 1e-15
        else:
            for (p, q) in (((0, 0, 1), (1, 2, 2)), ((0, 2, 2), (0, 1, 1)), ((1, 1, 2), (0, 0, 2))):
                assert abs((dQ[p] + dQ[q]) - (uuu[p] + uuu[q])) < 1e-15
                assert abs((dQ[p] - dQ[q]) - (uuu[p] - uuu[q])) < 1e-15


@pytest.mark.parametrize("lattice", [D2Q9, D3Q19])
@pytest.mark.parametrize("tau", [0.51, 0.8, 1.7])
def test_bgk_conserves_and_relaxes(lattice, tau):
    f = _random_f(lattice, 7)
    out = _one_cell(lattice, tau, BGK).update_cell(f, 0)
    feq = _one_cell(lattice, 1.0, BGK).update_cell(f, 0)
    r0, j0, _, _ = _moments(lattice, f)
    r1, j1, _, _ = _moments(lattice, out)
    assert abs(r1 - r0) < 1e-15 and np.abs(j1 - j0).max() < 1e-15
    assert np.abs((out - feq) - (1 - 1 / tau) * (f - feq)).max() < 1e-15


def test_ghost_mode_survives_bgk_and_not_the_regularized_collision():
    """D2Q9 ghost mode w_i (xi_x^2 - c_s^2)(xi_y^2 - c_s^2) (the fourth-order
    Hermite polynomial H_xxyy): orthogonal to every moment up to order three,
    so it leaves rho, u, Pi and the supported third moments untouched."""
    _, q, xi, w, _ = oracle.lattice(D2Q9)
    ghost = w * (xi[:, 0] ** 2 - CS2) * (xi[:, 1] ** 2 - CS2)
    base = _random_f(D2Q9, 3, spread=0.02)
    f = base + 0.01 * ghost
    tau = 0.6
    out_bgk = _one_cell(D2Q9, tau, BGK).update_cell(f, 0)
    ref_bgk = _one_cell(D2Q9, tau, BGK).update_cell(base, 0)
    out_rr = _one_cell(D2Q9, tau, RR).update_cell(f, 0)
    ref_rr = _one_cell(D2Q9, tau, RR).update_cell(base, 0)
    assert np.abs((out_bgk - ref_bgk) - (1 - 1 / tau) * 0.01 * ghost).max() < 1e-15
    assert np.abs(out_rr - ref_rr).max() < 1e-15


@pytest.mark.parametrize("tau", [0.6, 0.8])
def test_bgk_taylor_green_viscosity(tau):
    n = 64
    P = oracle.Problem(D2Q9, (n, n), tau)
    P.collision = BGK
    rho, u = inputs.taylor_green_2d(n, 0.01)
    f = P.equilibrium(rho, u)
    k = 2 * math.pi / n
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    basis = (np.sin(k * x) * np.cos(k * y)).reshape(-1)
    ts, amps = [], []
    for t in range(0, 401, 50):
        if t:
            f = P.run(f, 50, step0=t - 50)
        _, uu, _ = P.moments(f)
        ts.append(t)
        amps.append((uu[:, 0] * basis).sum() / (basis * basis).sum())
    ts, amps = np.array(ts[1:]), np.array(amps[1:])
    rate = -np.polyfit(ts, np.log(np.abs(amps)), 1)[0]
    nu_fit = rate / (2 * k * k)
    assert abs(nu_fit / (CS2 * (tau - 0.5)) - 1) < 0.01
