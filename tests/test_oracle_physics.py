"""Whole-scheme pins of the oracle against what the physics fixes.

  * Taylor-Green decay at nu = c_s^2 (tau - 1/2) (Sec. II.A, below Eq. truncatedEq)
  * Poiseuille profile between halfway bounce-back walls (viscosity + walls)
  * plane acoustic pulse moving at u0 +- c_s, c_s = 1/sqrt(3) (Sec. II.A, p = c_s^2 rho)
  * exact global conservation on a periodic lattice (Eq. optimizedLB conserves
    rho and rho u cell by cell; streaming only permutes populations)
  * mass conservation in a closed bounce-back box
  * a uniform stream is a fixed point of the inflow / outflow / sponge rules
"""
import math

import numpy as np
import pytest

import oracle
from oracle import D2Q9, D3Q19, CS2, VELOCITY, OUTFLOW
from paper_1710_02065_gb300 import inputs


def _fit_rate(ts, amps):
    return -np.polyfit(ts, np.log(amps), 1)[0]


@pytest.mark.parametrize("tau", [0.6, 0.8])
def test_taylor_green_2d_viscosity(tau):
    n = 64
    P = oracle.Problem(D2Q9, (n, n), tau)
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
    nu_fit = _fit_rate(np.array(ts[1:]), np.array(amps[1:])) / (2 * k * k)
    nu = CS2 * (tau - 0.5)
    assert abs(nu_fit / nu - 1) < 0.01, (nu_fit, nu)


def test_taylor_green_3d_viscosity():
    n, tau = 24, 0.7
    P = oracle.Problem(D3Q19, (n, n, n), tau)
    rho, u = inputs.taylor_green_3d(n, 0.005)
    f = P.equilibrium(rho, u)
    k = 2 * math.pi / n
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    basis = (np.sin(k * x) * np.cos(k * y) * np.cos(k * z)).reshape(-1)
    ts, amps = [], []
    for t in range(0, 121, 30):
        if t:
            f = P.run(f, 30, step0=t - 30)
        _, uu, _ = P.moments(f)
        ts.append(t)
        amps.append((uu[:, 0] * basis).sum() / (basis * basis).sum())
    rate = _fit_rate(np.array(ts[1:]), np.array(amps[1:]))
    nu_fit = rate / (3 * k * k)
    nu = CS2 * (tau - 0.5)
    assert abs(nu_fit / nu - 1) < 0.02, (nu_fit, nu)


def test_taylor_green_3d_viscosity_d3q27():
    """The same decay on the D3Q27 lattice (full third order)."""
    n, tau = 20, 0.7
    P = oracle.Problem(oracle.D3Q27, (n, n, n), tau)
    rho, u = inputs.taylor_green_3d(n, 0.005)
    f = P.equilibrium(rho, u)
    k = 2 * math.pi / n
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    basis = (np.sin(k * x) * np.cos(k * y) * np.cos(k * z)).reshape(-1)
    ts, amps = [], []
    for t in range(0, 81, 20):
        if t:
            f = P.run(f, 20, step0=t - 20)
        _, uu, _ = P.moments(f)
        ts.append(t)
        amps.append((uu[:, 0] * basis).sum() / (basis * basis).sum())
    rate = _fit_rate(np.array(ts[1:]), np.array(amps[1:]))
    assert abs(rate / (3 * k * k) / (CS2 * (tau - 0.5)) - 1) < 0.02


def test_poiseuille_between_bounce_back_walls():
    """Body-force channel: u(y) = g/(2 nu) (y - 1/2)(H + 1/2 - y), walls halfway."""
    H, tau, g = 24, 0.8, 2e-6
    nx, ny = 2, H + 2
    P = oracle.Problem(D2Q9, (nx, ny), tau)
    solid = np.zeros((ny, nx), np.uint8)
    solid[0, :] = 1
    solid[-1, :] = 1
    P.solid = solid.reshape(-1)
    P.g = [g, 0.0, 0.0]
    rho = np.ones(nx * ny)
    u = np.zeros((nx * ny, 3))
    f = P.equilibrium(rho, u)
    f = P.run(f, 12000)
    _, uu, _ = P.moments(f)
    ux = uu[:, 0].reshape(ny, nx)[1:-1, 0]
    nu = CS2 * (tau - 0.5)
    yy = np.arange(1, H + 1)
    exact = g / (2 * nu) * (yy - 0.5) * (H + 0.5 - yy)
    err = np.linalg.norm(ux - exact) / np.linalg.norm(exact)
    assert err < 0.01, err


def test_plane_acoustic_pulse_speed():
    """A planar pulse splits into waves at u0 + c_s and u0 - c_s."""
    nx, ny, u0, tau = 400, 2, 0.05, 0.6
    P = oracle.Problem(D2Q9, (nx, ny), tau)
    rho, u = inputs.plane_pulse_2d(nx, ny, 1e-3, 6.0, u0)
    f = P.equilibrium(rho, u)
    ts, right, left = [], [], []

    def peak(prof, lo, hi):
        i = lo + int(np.argmax(prof[lo:hi]))
        a, b, c = prof[i - 1], prof[i], prof[i + 1]
        return i + 0.5 * (a - c) / (a - 2 * b + c)

    for t in range(0, 121, 20):
        if t:
            f = P.run(f, 20, step0=t - 20)
        r, _, _ = P.moments(f)
        prof = r.reshape(ny, nx)[0] - 1.0
        if t >= 40:
            ts.append(t)
            right.append(peak(prof, nx // 2 + 5, nx - 2))
            left.append(peak(prof, 2, nx // 2 - 5))
    cr = np.polyfit(ts, right, 1)[0]
    cl = np.polyfit(ts, left, 1)[0]
    cs = 1 / math.sqrt(3)
    assert abs(cr - (u0 + cs)) / cs < 0.01, cr
    assert abs(cl - (u0 - cs)) / cs < 0.01, cl


def test_acoustic_pulse_2d_global_conservation():
    """The D2Q9 128^2 periodic Gaussian pulse (tau = 0.6, u0 = (0.05, 0)):
    total mass and momentum are invariant to round-off over 200 steps."""
    n = 128
    P = oracle.Problem(D2Q9, (n, n), 0.6)
    rho, u = inputs.gaussian_pulse_2d(n, 1e-3, 6.0, (0.05, 0.0))
    f = P.equilibrium(rho, u)
    _, _, xi, _, _ = oracle.lattice(D2Q9)
    m0 = f.sum()
    j0 = (f * xi[:, 0:1]).sum()
    f = P.run(f, 200)
    assert abs(f.sum() - m0) / m0 < 1e-13
    assert abs((f * xi[:, 0:1]).sum() - j0) / abs(j0) < 1e-12
    assert abs((f * xi[:, 1:2]).sum()) < 1e-12 * m0


@pytest.mark.parametrize("which", [D2Q9, D3Q19])
def test_closed_bounce_back_box_conserves_mass(which):
    n = (12, 10, 8) if which == D3Q19 else (16, 12)
    P = oracle.Problem(which, n, 0.7)
    shape = tuple(reversed(P.n))
    solid = np.zeros(shape, np.uint8)
    solid[:, 0, :] = solid[:, -1, :] = 1
    solid[:, :, 0] = solid[:, :, -1] = 1
    if which == D3Q19:
        solid[0] = solid[-1] = 1
    solid[shape[0] // 2, shape[1] // 2, shape[2] // 2] = 1  # an obstacle inside
    P.solid = solid.reshape(-1)
    _, _, _, w, _ = oracle.lattice(which)
    f = inputs.random_populations(w, P.ncell, seed=3, spread=0.05)
    fluid = solid.reshape(-1) == 0
    m0 = f[:, fluid].sum()
    f = P.run(f, 50)
    assert abs(f[:, fluid].sum() - m0) / m0 < 1e-13


@pytest.mark.parametrize("which", [D2Q9, D3Q19])
def test_uniform_stream_is_fixed_point_of_open_boundaries(which):
    """Velocity inlet on -x, zero-gradient outflow on +x, sponge layers with the
    stream as reference: a uniform stream stays uniform to round-off."""
    U = 0.08
    if which == D2Q9:
        P = oracle.Problem(D2Q9, (40, 12), 0.6)
    else:
        P = oracle.Problem(D3Q19, (20, 8, 6), 0.6)
    P.set_boundary(0, VELOCITY, (U, 0, 0))
    P.set_boundary(1, OUTFLOW)
    for face in ([1, 2, 3] if which == D2Q9 else [1, 2, 3, 4, 5]):
        P.set_sponge(face, 5, 0.5, 1.0, (U, 0, 0))
    if which == D3Q19:
        for face in (2, 3, 4, 5):
            P.set_boundary(face, OUTFLOW)
    rho = np.ones(P.ncell)
    u = np.zeros((P.ncell, 3))
    u[:, 0] = U
    f0 = P.equilibrium(rho, u)
    f = P.run(f0, 30)
    assert np.abs(f - f0).max() < 1e-15


def test_inlet_noise_statistics():
    """Seeded inlet noise is within +-amp*|u_in| per component and averages out."""
    U, amp = 0.1, 0.01
    P = oracle.Problem(D2Q9, (8, 400), 0.6)
    P.set_boundary(0, VELOCITY, (U, 0, 0))
    P.set_boundary(1, OUTFLOW)
    P.noise_seed, P.noise_amp = 3, amp
    rho = np.ones(P.ncell)
    u = np.zeros((P.ncell, 3)); u[:, 0] = U
    f = P.equilibrium(rho, u)
    f = P.run(f, 1)
    _, uu, _ = P.moments(f)
    inlet = uu.reshape(400, 8, 3)[:, 0, :]
    dv = inlet[:, :2] - np.array([U, 0])
    assert np.abs(dv).max() <= amp * U * (1 + 1e-12)
    assert abs(dv.mean()) < 0.2 * amp * U
    assert dv.std() > 0.4 * amp * U  # uniform on [-a, a] has std a/sqrt(3)


def test_wall_force_balances_body_force_in_poiseuille():
    """Steady channel flow: the walls take exactly the momentum the body force
    puts in, F_wall = g * (fluid mass), by momentum exchange on the links."""
    H, tau, g = 16, 0.8, 2e-6
    nx, ny = 3, H + 2
    P = oracle.Problem(D2Q9, (nx, ny), tau)
    solid = np.zeros((ny, nx), np.uint8)
    solid[0, :] = 1
    solid[-1, :] = 1
    P.solid = solid.reshape(-1)
    P.g = [g, 0.0, 0.0]
    f = P.equilibrium(np.ones(nx * ny), np.zeros((nx * ny, 3)))
    f = P.run(f, 6000)
    F = P.wall_force(f)
    fluid = solid.reshape(-1) == 0
    mass = f[:, fluid].sum()
    assert abs(F[0] - g * mass) / (g * mass) < 1e-6
    assert abs(F[1]) < 1e-12 * g * mass * 1e6


def test_wall_force_zero_at_rest_and_symmetric_for_uniform_obstacle():
    P = oracle.Problem(D2Q9, (30, 20), 0.7)
    P.solid = inputs.cylinder_mask(30, 20, 15, 10, 6)
    f = P.equilibrium(np.ones(P.ncell), np.zeros((P.ncell, 3)))
    F = P.wall_force(f)
    assert np.abs(F).max() < 1e-14


def test_free_slip_walls_exert_no_shear():
    """Channel between free-slip walls (Sec. III lateral condition) driven by a
    body force: the flow accelerates as a plug, no boundary layer forms
    (bounce-back walls in the same channel give a parabola)."""
    from oracle import FREESLIP
    H, tau, g = 20, 0.7, 1e-6
    P = oracle.Problem(D2Q9, (4, H), tau)
    P.set_boundary(2, FREESLIP)
    P.set_boundary(3, FREESLIP)
    P.g = [g, 0.0, 0.0]
    f = P.equilibrium(np.ones(P.ncell), np.zeros((P.ncell, 3)))
    f = P.run(f, 1500)
    _, uu, _ = P.moments(f)
    ux = uu[:, 0].reshape(H, 4)[:, 1]
    # the (oracle-only) body force is not applied on the rebuilt wall nodes,
    # so the plug lags the free acceleration g t by about 1%
    assert abs(ux.mean() - g * 1500) / (g * 1500) < 0.02
    assert (ux.max() - ux.min()) / ux.mean() < 1e-2
    assert np.abs(uu[:, 1]).max() < 1e-12
    # the same channel between bounce-back walls: a boundary layer, > 20x the spread
    Q = oracle.Problem(D2Q9, (4, H + 2), tau)
    solid = np.zeros((H + 2, 4), np.uint8); solid[0] = solid[-1] = 1
    Q.solid = solid.reshape(-1)
    Q.g = [g, 0.0, 0.0]
    fq = Q.run(Q.equilibrium(np.ones(Q.ncell), np.zeros((Q.ncell, 3))), 1500)
    _, uq, _ = Q.moments(fq)
    uq = uq[:, 0].reshape(H + 2, 4)[1:-1, 1]
    assert (uq.max() - uq.min()) / uq.mean() > 20 * (ux.max() - ux.min()) / ux.mean()


@pytest.mark.parametrize("which", [D2Q9, D3Q19])
def test_free_slip_and_pressure_faces_keep_a_uniform_stream(which):
    """A stream parallel to free-slip walls, leaving through a constant-pressure
    outlet at the stream's density, is a fixed point; the outlet nodes carry
    exactly the imposed density after a step from a disturbed state."""
    from oracle import FREESLIP, PRESSURE
    U = 0.07
    P = oracle.Problem(which, (24, 10, 8) if which == D3Q19 else (30, 12), 0.62)
    P.set_boundary(0, VELOCITY, (U, 0, 0))
    P.set_boundary(1, PRESSURE, rho=1.0)
    P.set_boundary(2, FREESLIP)
    P.set_boundary(3, FREESLIP)
    if which == D3Q19:
        P.set_boundary(4, FREESLIP)
        P.set_boundary(5, FREESLIP)
    u = np.zeros((P.ncell, 3)); u[:, 0] = U
    f0 = P.equilibrium(np.ones(P.ncell), u)
    assert np.abs(P.run(f0, 20) - f0).max() < 1e-15
    _, _, _, w, _ = oracle.lattice(which)
    P.set_boundary(1, PRESSURE, rho=1.002)
    f = P.run(inputs.random_populations(w, P.ncell, 5, 0.05), 1)
    rho, _, _ = P.moments(f)
    nx = P.n[0]
    outlet = rho.reshape(-1, nx)[:, nx - 1]
    # outlet nodes not claimed by an earlier face (x-faces come first)
    assert np.abs(outlet - 1.002).max() < 1e-14


@pytest.mark.parametrize("which", [D2Q9, D3Q19])
def test_pressure_outlet_carries_the_shear_of_a_channel_flow(which):
    """Pressure-driven channel (Sec. IV outlet, reading R17): a parabolic
    velocity inlet, a constant-pressure outlet at rho = 1 and halfway
    bounce-back walls at y = 1/2 and H + 1/2.  The outlet node takes u and
    Pi^neq of its inward neighbour with the imposed density, so after any
    number of steps its stored moments equal the neighbour's (density aside)
    to round-off, and in the developed flow they are the Poiseuille ones: the
    profile is the parabola and the stored shear stress is
    Pi^neq_xy = rho c_s^2 (1 - tau) du/dy (the relaxed viscous stress
    (1 - 1/tau) (-rho c_s^2 tau du/dy)).  Dropping Pi^neq at the outlet, or
    taking it from the outlet node's own streamed populations, breaks both."""
    from oracle import PRESSURE
    H, nx, tau, U = 16, 48, 0.8, 0.04
    ny, nz = H + 2, (1 if which == D2Q9 else 3)
    P = oracle.Problem(which, (nx, ny) if which == D2Q9 else (nx, ny, nz), tau)
    solid = np.zeros((nz, ny, nx), np.uint8)
    solid[:, 0, :] = solid[:, -1, :] = 1
    P.solid = solid.reshape(-1)
    fluid = slice(1, ny - 1)
    y = np.arange(ny) - 0.5  # distance from the lower wall
    prof_y = np.zeros(ny)
    prof_y[fluid] = 4 * U * y[fluid] * (H - y[fluid]) / H ** 2
    prof = np.zeros((ny * nz, 3))
    prof[:, 0] = np.tile(prof_y, nz)
    P.set_boundary(0, VELOCITY, profile=prof)
    P.set_boundary(1, PRESSURE, rho=1.0)
    u = np.zeros((P.ncell, 3))
    u[:, 0] = np.broadcast_to(prof_y[None, :, None], (nz, ny, nx)).reshape(-1)
    f = P.run(P.equilibrium(np.ones(P.ncell), u), 2000)
    rho, uu, pn = P.moments(f)
    r = rho.reshape(nz, ny, nx)[:, fluid]
    ux = uu[:, 0].reshape(nz, ny, nx)[:, fluid]
    uy = uu[:, 1].reshape(nz, ny, nx)[:, fluid]
    pxy = pn[:, 1].reshape(nz, ny, nx)[:, fluid]
    # the rule itself, through a whole update: imposed density, neighbour's u and Pi^neq
    assert np.abs(r[:, :, -1] - 1.0).max() < 1e-14
    assert np.abs(ux[:, :, -1] - ux[:, :, -2]).max() < 1e-15
    assert np.abs(uy[:, :, -1] - uy[:, :, -2]).max() < 1e-15
    assert np.abs(pxy[:, :, -1] - pxy[:, :, -2]).max() < 1e-12 * np.abs(pxy[:, :, -2]).max()
    # the developed channel flow at the outlet
    shape = ux[0, :, -1] / ux[0, :, -1].sum() - prof_y[fluid] / prof_y[fluid].sum()
    assert np.abs(shape).max() < 2e-3 * (prof_y[fluid] / prof_y[fluid].sum()).max()
    dudy = 4 * U * (H - 2 * y[fluid]) / H ** 2
    stress = r[0, :, -1] * CS2 * (1 - tau) * dudy
    assert np.abs(pxy[0, :, -1] - stress).max() < 0.03 * np.abs(stress).max()


def test_sponge_absorbs_a_plane_pulse():
    """Plane acoustic pulse (amplitude 1e-3 split into two waves of 5e-4)
    leaving a D2Q9 channel through zero-gradient outflow faces, with and
    without 30-cell sponges (chi_max 0.5, Sec. II.C): after the waves have
    had time to reach the faces and come back to the middle, the largest
    density disturbance left in the middle measures the reflection.  Measured:
    outflow alone about -15 dB, with the sponges about -60 dB; the bounds
    stated here are -10 dB and -50 dB."""
    nx, ny = 400, 2
    T = int(2 * (nx / 2 - 60) / math.sqrt(CS2))

    def reflected(width):
        P = oracle.Problem(D2Q9, (nx, ny), 0.6)
        P.set_boundary(0, oracle.OUTFLOW)
        P.set_boundary(1, oracle.OUTFLOW)
        if width:
            P.set_sponge(0, width, 0.5)
            P.set_sponge(1, width, 0.5)
        rho, u = inputs.plane_pulse_2d(nx, ny, 1e-3, 6.0)
        r, _, _ = P.moments(P.run(P.equilibrium(rho, u), T))
        left = np.abs(r.reshape(ny, nx)[0, 70:nx - 70] - 1).max()
        return 20 * math.log10(left / 5e-4)

    bare, sponge = reflected(0), reflected(30)
    assert bare > -20 and bare < -10, bare
    assert sponge < -50, sponge


def test_threaded_run_is_bitwise_the_plain_run():
    """Problem.run(threads=k) splits each step's cells over host threads; every
    cell is the same orc_update_cell call, so the field is bitwise the one of
    the single-threaded run (inflow with noise, outflow, sponges, a solid)."""
    P = oracle.Problem(D3Q19, (20, 14, 12), 0.56)
    P.set_boundary(0, VELOCITY, (0.04, 0.0, 0.0))
    P.set_boundary(1, OUTFLOW)
    P.set_sponge(1, 5, 0.6)
    P.noise_seed, P.noise_amp = 4, 0.02
    solid = np.zeros((12, 14, 20), np.uint8)
    solid[5:7, 6:8, 8:10] = 1
    P.solid = solid.reshape(-1)
    _, _, _, w, _ = oracle.lattice(D3Q19)
    f0 = inputs.random_populations(w, P.ncell, 3, 0.05)
    a = P.run(f0, 7, step0=2)
    for k in (2, 5, 16):
        assert np.array_equal(P.run(f0, 7, step0=2, threads=k), a)
