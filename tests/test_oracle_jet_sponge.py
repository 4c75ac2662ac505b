"""Pins of the round-jet similarity reference of the outflow sponge (Sec. IV
uses the jet similarity solution of Pope 2000 as the sponge's reference field
in the outflow region; reading R21).

  * on the axis the reference is the centreline velocity B D U_J / (x - x0),
    capped at U_J; at the half-width r = S (x - x0) it is half of that
  * self-similarity: the axial momentum flux of the reference through a
    cross-section, sum of u_x^2 over the plane, is the same at every x
  * outside the +x layer, or without a jet reference, the uniform u_ref
"""
import numpy as np

import oracle
from oracle import D3Q19, Problem


def _problem(n=(200, 96, 96), W=60):
    P = Problem(D3Q19, n, 0.6)
    P.set_sponge(1, W, 0.5, 1.0, (0.01, 0.0, 0.0))
    return P


def test_centreline_and_half_width():
    P = _problem()
    U, D, x0, B, S = 0.1, 6.0, -5.0, 5.8, 0.094
    for x in (150, 170, 199):
        xi = x - x0
        Uc = min(U, B * D * U / xi)
        # a reference centred so that the cell (x, 10, 40) is exactly at the half-width
        P.set_jet_reference(10.0 + S * xi, 40.0, U, D, x0, B, S)
        assert abs(P.sponge_reference(x, 10, 40)[0] - Uc / 2) < 1e-15
        P.set_jet_reference(10.0, 40.0, U, D, x0, B, S)
        u = P.sponge_reference(x, 10, 40)
        assert abs(u[0] - Uc) < 1e-15 and u[1] == 0.0 and u[2] == 0.0
    # near the virtual origin the centreline velocity is capped at U_J
    P.set_jet_reference(48.0, 48.0, U, D, 130.0, B, S)
    assert abs(P.sponge_reference(141, 48, 48)[0] - U) < 1e-15


def test_momentum_flux_is_the_same_in_every_cross_section():
    """The plane is wide enough that the cut tail of (1 + a eta^2)^-4 is below
    1e-3 of the flux at every x."""
    import ctypes as C
    n = 220
    P = _problem(n=(260, n, n), W=120)
    U, D, x0 = 0.1, 6.0, 20.0
    P.set_jet_reference((n - 1) / 2, (n - 1) / 2, U, D, x0)
    s = P._struct()
    u = np.zeros(3)
    up = u.ctypes.data_as(C.POINTER(C.c_double))
    fluxes = []
    for x in (150, 190, 230):
        tot = 0.0
        for z in range(n):
            for y in range(n):
                oracle.lib().orc_sponge_reference(C.byref(s), x, y, z, up)
                tot += u[0] * u[0]
        fluxes.append(tot)
    fluxes = np.array(fluxes)
    # (a centreline decay of another power, or a spreading that is not linear
    # in x - x0, changes the flux between these planes by tens of per cent)
    assert np.abs(fluxes / fluxes[0] - 1).max() < 1e-3, fluxes


def test_uniform_reference_outside_the_outflow_layer():
    P = _problem()
    P.set_jet_reference(48.0, 48.0, 0.1, 6.0, -5.0)
    assert np.array_equal(P.sponge_reference(139, 48, 48), [0.01, 0.0, 0.0])  # layer starts at x = 140
    assert P.sponge_reference(140, 48, 48)[0] > 0.01
    P.set_jet_reference(48.0, 48.0, 0.1, 0.0, -5.0)  # D = 0: no jet reference
    assert np.array_equal(P.sponge_reference(180, 48, 48), [0.01, 0.0, 0.0])
