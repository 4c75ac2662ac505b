"""Parity of the GPU two-level grid (Sec. II.B) with the oracle's TwoLevel.

Tolerances as in test_gpu_parity: FP64 1e-12 normwise in rho and u on each
level, FP32 1e-5.
"""
import numpy as np
import pytest

import oracle
from cases import cylinder_two_level, to_oracle, VELOCITY

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_02065_gb300 import build
    build.build()


def _normwise(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _gpu_two_level(c, patch, rho_f, u_f, solid_f, prec):
    from cases import to_gpu
    from paper_1710_02065_gb300 import lbm
    s = to_gpu(c, prec)
    X0, Y0, Wc, Hc = patch
    lbm.lbm_add_refinement_patch(s.h, (X0, Y0, 0), (Wc, Hc, 1))
    lbm.lbm_set_geometry_level(s.h, 1, solid_f)
    lbm.lbm_set_state_level(s.h, 1, rho_f, u_f)
    lbm.lbm_set_state(s.h, c.rho0, c.u0)  # refresh interface moments from the coarse state
    return s


def _oracle_two_level(c, patch, rho_f, u_f, solid_f):
    P, _ = to_oracle(c)
    T = oracle.TwoLevel(P, *patch)
    T.set_fine_solid(solid_f)
    T.init(c.rho0, c.u0, rho_f, u_f)
    return T


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_two_level_cylinder_parity(prec, tol):
    from paper_1710_02065_gb300 import lbm
    c, patch, rho_f, u_f, solid_f = cylinder_two_level()
    T = _oracle_two_level(c, patch, rho_f, u_f, solid_f)
    s = _gpu_two_level(c, patch, rho_f, u_f, solid_f, prec)
    ext, tau_f = lbm.lbm_level_info(s.h, 1)
    assert ext == (T.Pf.n[0], T.Pf.n[1], 1)
    assert abs(tau_f - T.Pf.tau) < 1e-15
    steps = 40
    T.run(steps)
    s.step(steps)
    rc, uc, _ = T.Pc.moments(T.fc)
    rf, uf, _ = T.Pf.moments(T.ff)
    grc = np.zeros(T.Pc.ncell); guc = np.zeros((T.Pc.ncell, 3))
    grf = np.zeros(T.Pf.ncell); guf = np.zeros((T.Pf.ncell, 3))
    lbm.lbm_moments_level(s.h, 0, grc, guc, None)
    lbm.lbm_moments_level(s.h, 1, grf, guf, None)
    X0, Y0, Wc, Hc = patch
    nxc, nyc = T.Pc.n[0], T.Pc.n[1]
    live = np.ones((nyc, nxc), bool)
    live[Y0 + 2:Y0 + Hc - 1, X0 + 2:X0 + Wc - 1] = False  # frozen covered coarse cells
    live = live.reshape(-1)
    fluid_f = solid_f == 0
    assert _normwise(grc[live], rc[live]) <= tol
    assert _normwise(guc[live], uc[live]) <= tol
    assert _normwise(grf[fluid_f], rf[fluid_f]) <= tol
    assert _normwise(guf[fluid_f], uf[fluid_f]) <= tol
    F = lbm.lbm_force(s.h, 1)
    F_ref = T.Pf.wall_force(T.ff)
    assert np.abs(F - F_ref).max() <= tol * np.abs(F_ref).max() * 10


def test_two_level_uniform_stream_exact():
    """A uniform stream crosses the GPU interface unchanged (FP64 round-off)."""
    from paper_1710_02065_gb300 import lbm
    from cases import Case
    U = (0.05, -0.02, 0.0)
    c = Case("uniform2", 0, (40, 30, 1), 0.6, rho0=np.ones(1200), u0=np.tile(U, (1200, 1)))
    patch = (10, 8, 16, 12)
    nf = 33 * 25
    s = _gpu_two_level(c, patch, np.ones(nf), np.tile(U, (nf, 1)), np.zeros(nf, np.uint8), 0)
    f0c = s.populations()
    f0f = np.zeros((9, nf))
    lbm.lbm_get_populations_level(s.h, 1, f0f)
    s.step(6)
    f1f = np.zeros((9, nf))
    lbm.lbm_get_populations_level(s.h, 1, f1f)
    assert np.abs(s.populations() - f0c).max() < 1e-15
    assert np.abs(f1f - f0f).max() < 1e-15


def test_two_level_full_size_few_steps():
    """The two-level cylinder at full size (coarse 800x400, fine 641x321),
    FP32, 3 coarse steps: both levels equal the oracle within 1e-5."""
    from paper_1710_02065_gb300 import lbm
    c, patch, rho_f, u_f, solid_f = cylinder_two_level(800, 400, (160, 120, 320, 160), diameter_c=20.0,
                                                       xc=40, yc=80, sponge=50)
    T = _oracle_two_level(c, patch, rho_f, u_f, solid_f)
    s = _gpu_two_level(c, patch, rho_f, u_f, solid_f, 1)
    T.run(3)
    s.step(3)
    rc, uc, _ = T.Pc.moments(T.fc)
    rf, uf, _ = T.Pf.moments(T.ff)
    grc = np.zeros(T.Pc.ncell); guc = np.zeros((T.Pc.ncell, 3))
    grf = np.zeros(T.Pf.ncell); guf = np.zeros((T.Pf.ncell, 3))
    lbm.lbm_moments_level(s.h, 0, grc, guc, None)
    lbm.lbm_moments_level(s.h, 1, grf, guf, None)
    fluid_f = solid_f == 0
    assert _normwise(grc, rc) <= 1e-5 and _normwise(guc, uc) <= 1e-5
    assert _normwise(grf[fluid_f], rf[fluid_f]) <= 1e-5 and _normwise(guf[fluid_f], uf[fluid_f]) <= 1e-5


def _case_3d(lattice=oracle.D3Q19):
    """D3Q19 (or D3Q27) box 24x20x18: inflow on -x, outflow behind a sponge on
    +x, y/z periodic; smooth density pulse and shear on a uniform stream; a
    fine patch over coarse [6, 16] x [5, 13] x [5, 12] holding a small solid
    sphere on the fine level."""
    from cases import Case
    n = (24, 20, 18)
    c = Case("two_level_3d", lattice, n, 0.6)
    U = 0.04
    c.faces = {0: (VELOCITY, (U, 0, 0), None), 1: (oracle.OUTFLOW, (0, 0, 0), None)}
    c.sponges = {1: (4, 0.3)}
    c.rho_ref, c.u_ref = 1.0, (U, 0.0, 0.0)

    def fields(X, Y, Z):
        r2 = (X - 11.0) ** 2 + (Y - 9.0) ** 2 + (Z - 8.5) ** 2
        rho = 1.0 + 2e-3 * np.exp(-r2 / 8.0)
        u = np.zeros(X.shape + (3,))
        u[..., 0] = U
        u[..., 1] = 0.01 * np.sin(2 * np.pi * Z / n[2])
        u[..., 2] = 0.008 * np.cos(2 * np.pi * Y / n[1])
        return rho.reshape(-1), u.reshape(-1, 3)

    z, y, x = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    c.rho0, c.u0 = fields(x.astype(float), y.astype(float), z.astype(float))
    patch = (6, 5, 5, 10, 8, 7)
    X0, Y0, Z0, Wc, Hc, Dc = patch
    nf = (2 * Wc + 1, 2 * Hc + 1, 2 * Dc + 1)
    k, j, i = np.meshgrid(np.arange(nf[2]), np.arange(nf[1]), np.arange(nf[0]), indexing="ij")
    rho_f, u_f = fields(X0 + i / 2, Y0 + j / 2, Z0 + k / 2)
    solid_f = (((i - 9) ** 2 + (j - 8) ** 2 + (k - 7) ** 2) <= 6).astype(np.uint8).reshape(-1)
    return c, patch, rho_f, u_f, solid_f


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
@pytest.mark.parametrize("lattice", [oracle.D3Q19, oracle.D3Q27])
def test_two_level_3d_parity(prec, tol, lattice):
    """D3Q19 / D3Q27 patch (fine shell from the coarse planes, covered coarse
    shell from the fine level) against the oracle's TwoLevel3 on both levels."""
    from cases import to_gpu
    from paper_1710_02065_gb300 import lbm
    c, patch, rho_f, u_f, solid_f = _case_3d(lattice)
    P, _ = to_oracle(c)
    T = oracle.TwoLevel3(P, *patch)
    T.set_fine_solid(solid_f)
    T.init(c.rho0, c.u0, rho_f, u_f)
    s = to_gpu(c, prec)
    X0, Y0, Z0, Wc, Hc, Dc = patch
    lbm.lbm_add_refinement_patch(s.h, (X0, Y0, Z0), (Wc, Hc, Dc))
    lbm.lbm_set_geometry_level(s.h, 1, solid_f)
    lbm.lbm_set_state_level(s.h, 1, rho_f, u_f)
    lbm.lbm_set_state(s.h, c.rho0, c.u0)
    ext, tau_f = lbm.lbm_level_info(s.h, 1)
    assert ext == tuple(T.Pf.n) and abs(tau_f - T.Pf.tau) < 1e-15
    steps = 10
    T.run(steps)
    s.step(steps)
    rc, uc, _ = T.Pc.moments(T.fc)
    rf, uf, _ = T.Pf.moments(T.ff)
    grc = np.zeros(T.Pc.ncell); guc = np.zeros((T.Pc.ncell, 3))
    grf = np.zeros(T.Pf.ncell); guf = np.zeros((T.Pf.ncell, 3))
    lbm.lbm_moments_level(s.h, 0, grc, guc, None)
    lbm.lbm_moments_level(s.h, 1, grf, guf, None)
    nxc, nyc, nzc = T.Pc.n
    live = np.ones((nzc, nyc, nxc), bool)
    live[Z0 + 2:Z0 + Dc - 1, Y0 + 2:Y0 + Hc - 1, X0 + 2:X0 + Wc - 1] = False  # frozen covered coarse cells
    live = live.reshape(-1)
    fluid_f = solid_f == 0
    assert _normwise(grc[live], rc[live]) <= tol
    assert _normwise(guc[live], uc[live]) <= tol
    assert _normwise(grf[fluid_f], rf[fluid_f]) <= tol
    assert _normwise(guf[fluid_f], uf[fluid_f]) <= tol
    F = lbm.lbm_force(s.h, 1)
    F_ref = T.Pf.wall_force(T.ff)
    assert np.abs(F - F_ref).max() <= tol * np.abs(F_ref).max() * 10
    s.close()


@pytest.mark.parametrize("lattice", [oracle.D3Q19, oracle.D3Q27])
def test_two_level_3d_uniform_stream_exact(lattice):
    from paper_1710_02065_gb300 import lbm
    s = lbm.Solver(lattice, (20, 18, 16), 0.6, 0)
    lbm.lbm_add_refinement_patch(s.h, (5, 4, 4), (8, 8, 6))
    U = (0.04, -0.02, 0.01)
    ext, _ = lbm.lbm_level_info(s.h, 1)
    nf = int(np.prod(ext))
    lbm.lbm_set_state_level(s.h, 1, np.ones(nf), np.tile(U, (nf, 1)))
    s.set_state(np.ones(s.ncell), np.tile(U, (s.ncell, 1)))
    f0 = s.populations()
    s.step(4)
    assert np.abs(s.populations() - f0).max() < 1e-15
    rf = np.zeros(nf); uf = np.zeros((nf, 3))
    lbm.lbm_moments_level(s.h, 1, rf, uf, None)
    assert np.abs(uf - np.array(U)).max() < 1e-15 and np.abs(rf - 1).max() < 1e-15
    s.close()


def _nested_case(lattice):
    """Three levels: coarse box with inflow / outflow / sponge, two nested
    patches (each inside the previous one), a solid on the finest level;
    smooth initial state on every level (positions in coarse units)."""
    from cases import Case
    if lattice == oracle.D2Q9:
        n, patches = (48, 40, 1), [((8, 7), (26, 22)), ((10, 9), (24, 20))]
    else:
        n, patches = (28, 24, 22), [((5, 5, 4), (14, 12, 12)), ((6, 5, 5), (12, 10, 10))]
    d = 2 if lattice == oracle.D2Q9 else 3
    c = Case("nested", lattice, n, 0.58)
    U = 0.04
    c.faces = {0: (VELOCITY, (U, 0, 0), None), 1: (oracle.OUTFLOW, (0, 0, 0), None)}
    c.sponges = {1: (5, 0.3)}
    c.rho_ref, c.u_ref = 1.0, (U, 0.0, 0.0)

    def fields(pos):
        X, Y = pos[:, 0], pos[:, 1]
        Z = pos[:, 2] if d == 3 else 0.0 * X
        rho = 1.0 + 1e-3 * np.exp(-((X - 20) ** 2 + (Y - 18) ** 2 + (Z - 11) ** 2 * (d == 3)) / 30.0)
        u = np.zeros((len(X), 3))
        u[:, 0] = U + 0.01 * np.sin(0.3 * Y)
        u[:, 1] = 0.008 * np.cos(0.25 * X)
        if d == 3:
            u[:, 2] = 0.005 * np.sin(0.2 * Y + 0.1 * X)
        return rho, u

    def positions(shape, origin, scale):
        idx = np.stack(np.meshgrid(*[np.arange(v) for v in reversed(shape[:d])], indexing="ij"), -1)
        idx = idx.reshape(-1, d)[:, ::-1].astype(float)
        pos = np.zeros((len(idx), 3))
        pos[:, :d] = np.asarray(origin[:d]) + idx * scale
        return pos

    c.rho0, c.u0 = fields(positions(n, (0, 0, 0), 1.0))
    states, origin, scale, shape = [], np.zeros(3), 1.0, n
    for o, e in patches:
        origin = origin + np.array(list(o) + [0] * (3 - len(o)), float) * scale
        scale /= 2
        shape = tuple(2 * v + 1 for v in e)
        states.append(fields(positions(shape, origin, scale)))
    nf = shape
    if d == 2:
        j, i = np.meshgrid(np.arange(nf[1]), np.arange(nf[0]), indexing="ij")
        solid = ((i - nf[0] // 2) ** 2 + (j - nf[1] // 2) ** 2 <= 9).astype(np.uint8).reshape(-1)
    else:
        k, j, i = np.meshgrid(np.arange(nf[2]), np.arange(nf[1]), np.arange(nf[0]), indexing="ij")
        solid = ((i - nf[0] // 2) ** 2 + (j - nf[1] // 2) ** 2 + (k - nf[2] // 2) ** 2 <= 4).astype(np.uint8).reshape(-1)
    return c, patches, states, solid


@pytest.mark.parametrize("lattice", [oracle.D2Q9, oracle.D3Q19])
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_three_nested_levels_parity(lattice, prec, tol):
    """Three levels (two nested patches, a solid on the finest) against the
    oracle's recursive MultiLevel, every level, wall force on the finest."""
    from cases import to_gpu
    from paper_1710_02065_gb300 import lbm
    c, patches, states, solid = _nested_case(lattice)
    P, _ = to_oracle(c)
    M = oracle.MultiLevel(P, patches)
    M.set_solid(2, solid)
    M.init([(c.rho0, c.u0)] + states)
    s = to_gpu(c, prec)
    for o, e in patches:
        lbm.lbm_add_refinement_patch(s.h, tuple(o) + (0,) * (3 - len(o)), tuple(e) + (1,) * (3 - len(e)))
    lbm.lbm_set_geometry_level(s.h, 2, solid)
    for k in (2, 1):
        lbm.lbm_set_state_level(s.h, k, *states[k - 1])
    lbm.lbm_set_state(s.h, c.rho0, c.u0)
    for k in range(3):
        ext, tau = lbm.lbm_level_info(s.h, k)
        assert ext[:2] == tuple(M.P[k].n[:2]) and abs(tau - M.P[k].tau) < 1e-15
    steps = 6
    M.run(steps)
    s.step(steps)
    for k in range(3):
        r_ref, u_ref, _ = M.P[k].moments(M.f[k])
        n = M.P[k].ncell
        r, u = np.zeros(n), np.zeros((n, 3))
        lbm.lbm_moments_level(s.h, k, r, u, None)
        live = M.P[k].solid == 0 if M.P[k].solid is not None else np.ones(n, bool)
        assert _normwise(r[live], r_ref[live]) <= tol, k
        assert _normwise(u[live], u_ref[live]) <= tol, k
    F = lbm.lbm_force(s.h, 2)
    F_ref = M.P[2].wall_force(M.f[2])
    assert np.abs(F - F_ref).max() <= tol * np.abs(F_ref).max() * 10
    s.close()


@pytest.mark.parametrize("three", [False, True])
def test_refined_checkpoint_resumes_bit_identically(tmp_path, three):
    """lbm_save / lbm_load carry every level's field and the interface moments
    (and the pressure-mean accumulator): a refined run saved after a few coarse
    steps and continued on a fresh handle matches the uninterrupted run bit
    for bit on both levels."""
    from cases import to_gpu
    from paper_1710_02065_gb300 import lbm

    def build():
        if three:
            c, patch, rho_f, u_f, solid_f = _case_3d()
            X0, Y0, Z0, Wc, Hc, Dc = patch
            s = to_gpu(c, 1)
            lbm.lbm_add_refinement_patch(s.h, (X0, Y0, Z0), (Wc, Hc, Dc))
        else:
            c, patch, rho_f, u_f, solid_f = cylinder_two_level()
            X0, Y0, Wc, Hc = patch
            s = to_gpu(c, 1)
            lbm.lbm_add_refinement_patch(s.h, (X0, Y0, 0), (Wc, Hc, 1))
        lbm.lbm_set_geometry_level(s.h, 1, solid_f)
        lbm.lbm_set_state_level(s.h, 1, rho_f, u_f)
        lbm.lbm_set_state(s.h, c.rho0, c.u0)
        return s

    def fine(s):
        ext, _ = lbm.lbm_level_info(s.h, 1)
        f = np.zeros((19 if three else 9, int(np.prod(ext))))
        lbm.lbm_get_populations_level(s.h, 1, f)
        return f

    a = build()
    a.step(3)
    lbm.lbm_pressure_mean(a.h, lbm.LBM_MEAN_ACCUMULATE)
    path = str(tmp_path / "refined.ck")
    lbm.lbm_save(a.h, path)
    a.step(5)
    lbm.lbm_pressure_mean(a.h, lbm.LBM_MEAN_ACCUMULATE)
    b = build()
    b.step(1)  # a different state and level parity before loading
    lbm.lbm_load(b.h, path)
    assert b.info()["step"] == 3
    b.step(5)
    lbm.lbm_pressure_mean(b.h, lbm.LBM_MEAN_ACCUMULATE)
    assert np.array_equal(a.populations(), b.populations())
    assert np.array_equal(fine(a), fine(b))
    n = a.ncell
    da, ma = np.zeros(n), np.zeros(n)
    db, mb = np.zeros(n), np.zeros(n)
    lbm.lbm_pressure_fluctuation(a.h, da, ma)
    lbm.lbm_pressure_fluctuation(b.h, db, mb)
    assert np.array_equal(ma, mb) and np.array_equal(da, db)
    a.close()
    b.close()


@pytest.mark.parametrize("case", ["2d", "3d", "nested3"])
def test_level_streams_concurrent_equals_in_order(case):
    """The refined levels' part of a step on a second stream, concurrent with
    the level-0 update (the default), leaves every level bitwise as running
    everything in order on one stream; also through captured step graphs
    (a non-default stream)."""
    import torch
    from cases import to_gpu
    from paper_1710_02065_gb300 import lbm
    stream = torch.cuda.Stream()

    def build(concurrent, on_stream):
        if case == "2d":
            c, patch, rho_f, u_f, solid_f = cylinder_two_level()
            X0, Y0, Wc, Hc = patch
            pl = [((X0, Y0, 0), (Wc, Hc, 1))]
            states, solid, finest = [(rho_f, u_f)], solid_f, 1
        elif case == "3d":
            c, patch, rho_f, u_f, solid_f = _case_3d()
            X0, Y0, Z0, Wc, Hc, Dc = patch
            pl = [((X0, Y0, Z0), (Wc, Hc, Dc))]
            states, solid, finest = [(rho_f, u_f)], solid_f, 1
        else:
            c, patches, states, solid = _nested_case(oracle.D3Q19)
            pl = [(tuple(o) + (0,) * (3 - len(o)), tuple(e) + (1,) * (3 - len(e))) for o, e in patches]
            finest = 2
        s = to_gpu(c, 1) if not on_stream else None
        if on_stream:
            s = lbm.Solver(c.lattice, c.n, c.tau, 1, stream=stream.cuda_stream)
            for face, spec in c.faces.items():
                lbm.lbm_set_boundary(s.h, face, spec[0], spec[1], spec[2])
            for face, (w, chi) in c.sponges.items():
                lbm.lbm_set_sponge(s.h, face, w, chi, c.rho_ref, c.u_ref)
            if c.solid is not None:
                lbm.lbm_set_geometry(s.h, c.solid)
        lbm.lbm_set_level_streams(s.h, concurrent)
        for o, e in pl:
            lbm.lbm_add_refinement_patch(s.h, o, e)
        lbm.lbm_set_geometry_level(s.h, finest, solid)
        for k in range(len(states), 0, -1):
            lbm.lbm_set_state_level(s.h, k, *states[k - 1])
        lbm.lbm_set_state(s.h, c.rho0, c.u0)
        return s, len(pl) + 1

    ref, nlev = build(0, False)
    ref.step(9)
    for concurrent, on_stream in ((1, False), (1, True), (0, True)):
        s, _ = build(concurrent, on_stream)
        s.step(4)
        s.step(5)
        torch.cuda.synchronize()
        for k in range(nlev):
            ext, _ = lbm.lbm_level_info(ref.h, k)
            q = 9 if ext[2] == 1 else 19
            n = ext[0] * ext[1] * ext[2]
            fa, fb = np.zeros((q, n)), np.zeros((q, n))
            lbm.lbm_get_populations_level(ref.h, k, fa)
            lbm.lbm_get_populations_level(s.h, k, fb)
            assert np.array_equal(fa, fb), (concurrent, on_stream, k)
        s.close()
    with pytest.raises(lbm.LBMError):
        lbm.lbm_set_level_streams(ref.h, 2)
    ref.close()
