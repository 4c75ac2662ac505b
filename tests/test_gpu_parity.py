"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances
  * FP64 storage/compute: 1e-12 normwise relative in rho and u, and
    populations within 1e-13 absolute after a few steps (round-off only).
  * FP32: 1e-5 normwise relative in rho and u; populations within 1e-5 of
    max |f| (FP32 round-off of sums of O(Q) terms of size <= 1).
  * FP16 / BF16 shifted storage: each stored value g = f - w is rounded to a
    10-bit / 7-bit mantissa, so one step may err by 2^-11 / 2^-8 of max |g|;
    the bound used is (steps + 1) * 2^-10 (FP16) or 2^-7 (BF16) of max |g|.
"""
import math

import numpy as np
import pytest

import oracle
from cases import (Case, D2Q9, D3Q19, FREESLIP, OUTFLOW, PERIODIC, PRESSURE, VELOCITY, acoustic_pulse, cylinder,
                   round_jet, taylor_green_3d, to_gpu, to_oracle, with_random_state)
from paper_1710_02065_gb300 import inputs

pytestmark = pytest.mark.gpu

PRECS = {"fp64": 0, "fp32": 1, "fp16": 2, "bf16": 3}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_02065_gb300 import build
    build.build()


def _pop_tol(prec, f_ref, w, steps):
    g = np.abs(f_ref - w[:, None]).max()
    if prec == "fp64":
        return 1e-13
    if prec == "fp32":
        return 1e-5 * np.abs(f_ref).max()
    bits = 10 if prec == "fp16" else 7
    return (steps + 1) * 2.0 ** -bits * g + 1e-7


# Update kernels: the row-staged kernel (bulk copies into shared memory; FP32,
# FP16, BF16) and the register kernels, one or V cells per thread.
KERNELS = {"fp64": ["cell", "vec2"], "fp32": ["rows", "cell", "vec2", "vec4"],
           "fp16": ["rows", "cell", "vec2", "vec4"], "bf16": ["rows", "cell", "vec2", "vec4"]}


def use_kernel(s, kind, block=64):
    """Select one update kernel (and streaming pattern, 'aa-' prefix) on
    solver s; 'rows' must then be active."""
    from paper_1710_02065_gb300 import autotune, lbm
    if kind == "rows":
        lbm.lbm_set_streaming(s.h, lbm.LBM_STREAM_PULL)
        lbm.lbm_set_staging(s.h, 1, 0, 0)
        assert lbm.lbm_get_staging(s.h)[0] == 1, "row-staged kernel not eligible"
    else:
        assert autotune.apply(s.h, (kind, block))


def _normwise(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _boxed_case(lattice, seed=5):
    """Small ragged box exercising every boundary rule at once: velocity
    inflow with a profile and noise, zero-gradient outflow, sponges, a solid
    obstacle, periodic axes, random off-equilibrium populations."""
    if lattice == D2Q9:
        n = (37, 23, 1)
    else:
        n = (19, 13, 11)
    ncell = int(np.prod(n))
    c = Case("boxed", lattice, n, 0.58)
    U = 0.06
    nf = n[1] * n[2]
    prof = np.zeros((nf, 3))
    prof[:, 0] = U * (0.5 + np.random.default_rng(seed).random(nf))
    if lattice == D3Q19:
        prof[:, 2] = 0.01
    c.faces = {0: (VELOCITY, (0, 0, 0), prof), 1: (OUTFLOW, (0, 0, 0), None)}
    if lattice == D3Q19:
        c.faces[4] = (OUTFLOW, (0, 0, 0), None)
        c.faces[5] = (OUTFLOW, (0, 0, 0), None)
        c.sponges = {1: (6, 0.6), 5: (4, 0.9), 3: (3, 0.3)}
    else:
        c.sponges = {1: (8, 0.7), 3: (5, 0.4)}
    c.rho_ref, c.u_ref = 1.01, (0.02, -0.01, 0.0)
    c.noise = (7, 0.05)
    solid = np.zeros(n[::-1], np.uint8)
    if lattice == D2Q9:
        solid[0, 9:12, 14:18] = 1
    else:
        solid[4:7, 5:8, 8:11] = 1
    c.solid = solid.reshape(-1)
    return with_random_state(c, seed=seed, spread=0.08)


@pytest.mark.parametrize("prec", list(PRECS))
@pytest.mark.parametrize("lattice", [D2Q9, D3Q19])
def test_equilibrium_initialisation(lattice, prec):
    n = (13, 7, 1) if lattice == D2Q9 else (9, 7, 5)
    ncell = int(np.prod(n))
    rng = np.random.default_rng(1)
    rho = 1 + 0.01 * rng.normal(size=ncell)
    u = 0.1 * rng.normal(size=(ncell, 3))
    if lattice == D2Q9:
        u[:, 2] = 0
    c = Case("eq", lattice, n, 0.7, rho0=rho, u0=u)
    P, f_ref = to_oracle(c)
    s = to_gpu(c, PRECS[prec])
    f = s.populations()
    _, _, _, w, _ = oracle.lattice(lattice)
    assert np.abs(f - f_ref).max() <= _pop_tol(prec, f_ref, w, 0)


@pytest.mark.parametrize("prec", list(PRECS))
@pytest.mark.parametrize("lattice", [D2Q9, D3Q19])
def test_all_boundary_rules_few_steps(lattice, prec):
    c = _boxed_case(lattice)
    P, f = to_oracle(c)
    s = to_gpu(c, PRECS[prec])
    _, _, _, w, _ = oracle.lattice(lattice)
    f_gpu0 = s.populations()
    assert np.abs(f_gpu0 - f).max() <= _pop_tol(prec, f, w, 0)
    t = 0
    for steps in (1, 2):
        f = P.run(f, steps, step0=t)
        s.step(steps)
        t += steps
        got = s.populations()
        err = np.abs(got - f).max()
        assert err <= _pop_tol(prec, f, w, t), (t, err)
    assert s.info()["step"] == t


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_acoustic_pulse_128_parity_200_steps(prec, tol):
    """D2Q9 128^2 periodic Gaussian pulse, tau 0.6, 200 steps."""
    c = acoustic_pulse(128)
    P, f = to_oracle(c)
    f = P.run(f, 200)
    r_ref, u_ref, _ = P.moments(f)
    s = to_gpu(c, PRECS[prec])
    s.step(200)
    r, u, _ = s.moments()
    assert _normwise(r, r_ref) <= tol
    assert _normwise(u, u_ref) <= tol
    # GPU FP64 totals: mass and momentum conserved over 200 steps
    m, j, rc = s.reduce()
    assert rc == 0
    if prec == "fp64":
        r0 = c.rho0.sum()
        assert abs(m - r0) / r0 < 1e-13
        assert abs(j[0] - (c.rho0 * 0.05).sum()) / abs(j[0]) < 1e-12


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_taylor_green_3d_parity(prec, tol):
    c = taylor_green_3d(24, 0.7, 0.02)
    P, f = to_oracle(c)
    f = P.run(f, 40)
    r_ref, u_ref, pn_ref = P.moments(f)
    s = to_gpu(c, PRECS[prec])
    s.step(40)
    r, u, pn = s.moments()
    assert _normwise(r, r_ref) <= tol
    assert _normwise(u, u_ref) <= tol
    assert np.abs(pn - pn_ref).max() <= tol * np.abs(pn_ref).max() * 10


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_cylinder_scaled_parity(prec, tol):
    """The cylinder workload scaled to 200 x 100 (D = 10), 300 steps."""
    c = cylinder(200, 100, diameter=10.0, sponge=25)
    P, f = to_oracle(c)
    f = P.run(f, 300)
    r_ref, u_ref, _ = P.moments(f)
    s = to_gpu(c, PRECS[prec])
    s.step(300)
    r, u, _ = s.moments()
    fluid = c.solid == 0
    assert _normwise(r[fluid], r_ref[fluid]) <= tol
    assert _normwise(u[fluid], u_ref[fluid]) <= tol
    # momentum-exchange force on the cylinder
    from paper_1710_02065_gb300 import lbm
    F = lbm.lbm_force(s.h, 0)
    F_ref = P.wall_force(f)
    assert np.abs(F - F_ref).max() <= tol * np.abs(F_ref).max() * 10


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_round_jet_scaled_parity(prec, tol):
    """The round jet scaled to 48 x 32 x 32 (D = 6, sponges 8), 60 steps, seeded inlet noise."""
    c = round_jet(48, 32, 32, diameter=6.0, sponge=8, Re=2500.0)
    P, f = to_oracle(c)
    f = P.run(f, 60)
    r_ref, u_ref, _ = P.moments(f)
    s = to_gpu(c, PRECS[prec])
    s.step(60)
    r, u, _ = s.moments()
    assert _normwise(r, r_ref) <= tol
    assert _normwise(u, u_ref) <= tol


def test_edge_sizes_and_zero_steps():
    """Tiny and ragged boxes: 1x1 periodic, 3x3 with open faces, 129 wide (one
    cell past a block), n = 0 steps."""
    for n, faces in [((1, 1, 1), {}), ((3, 3, 1), {0: (VELOCITY, (0.05, 0, 0), None), 1: (OUTFLOW, (0, 0, 0), None),
                                                   2: (OUTFLOW, (0, 0, 0), None), 3: (OUTFLOW, (0, 0, 0), None)}),
                     ((129, 2, 1), {})]:
        c = with_random_state(Case("edge", D2Q9, n, 0.8), seed=2)
        c.faces = faces
        P, f = to_oracle(c)
        s = to_gpu(c, PRECS["fp64"])
        s.step(0)
        assert np.abs(s.populations() - f).max() < 1e-15
        f = P.run(f, 3)
        s.step(3)
        assert np.abs(s.populations() - f).max() < 1e-13
    c = with_random_state(Case("edge3", D3Q19, (3, 3, 3), 0.8), seed=2)
    c.faces = {k: (OUTFLOW, (0, 0, 0), None) for k in range(6)}
    P, f = to_oracle(c)
    s = to_gpu(c, PRECS["fp64"])
    f = P.run(f, 2)
    s.step(2)
    assert np.abs(s.populations() - f).max() < 1e-13


def test_moments_probe_and_reduce_match_oracle():
    c = _boxed_case(D3Q19, seed=9)
    P, f = to_oracle(c)
    f = P.run(f, 2)
    s = to_gpu(c, PRECS["fp64"])
    s.step(2)
    r, u, pn = s.moments()
    r0, u0, pn0 = P.moments(f)
    assert np.abs(r - r0).max() < 1e-14
    assert np.abs(u - u0).max() < 1e-13
    assert np.abs(pn - pn0).max() < 1e-14
    from paper_1710_02065_gb300 import lbm
    cells = [0, 17, 400, c.ncell - 1]
    p = lbm.lbm_probe(s.h, cells)
    assert np.abs(p - (r0[cells] - c.rho_ref) / 3.0).max() < 1e-15
    m, j, rc = s.reduce()
    fluid = c.solid == 0
    assert rc == 0
    assert abs(m - r0[fluid].sum()) < 1e-11
    assert np.abs(j - (r0[fluid, None] * u0[fluid]).sum(0)).max() < 1e-11


def test_non_finite_state_is_reported():
    from paper_1710_02065_gb300 import lbm
    c = with_random_state(Case("nan", D2Q9, (16, 8, 1), 0.8), seed=2)
    c.f0[3, 5] = np.nan
    s = to_gpu(c, PRECS["fp32"])
    _, _, rc = s.reduce()
    assert rc == lbm.LBM_EUNSTABLE


@pytest.mark.parametrize("ux,rho,unstable", [(0.55, 1.0, False), (0.60, 1.0, True), (0.0, -0.1, True)])
def test_supersonic_or_negative_density_is_reported(ux, rho, unstable):
    """|u| >= c_s = 0.577 or rho <= 0 in one fluid cell makes lbm_reduce
    return LBM_EUNSTABLE; a subsonic state passes."""
    from paper_1710_02065_gb300 import lbm
    n = (16, 8, 1)
    r = np.ones(int(np.prod(n)))
    u = np.zeros((r.size, 3))
    r[37], u[37, 0] = abs(rho), ux
    c = Case("sonic", D2Q9, n, 0.8, rho0=r, u0=u)
    if rho <= 0:  # lbm_set_state rejects rho <= 0: write the populations
        _, c.f0 = to_oracle(c)
        c.f0[:, 37] *= rho / abs(rho)
    s = to_gpu(c, PRECS["fp64"])
    _, _, rc = s.reduce()
    assert rc == (lbm.LBM_EUNSTABLE if unstable else lbm.LBM_OK)


@pytest.mark.parametrize("lattice", [D2Q9, D3Q19])
def test_chunked_host_transfers_match_whole_field(lattice):
    """A staging bound of a few KB moves every field in many chunks with a
    ragged last one: state, populations and moments must equal those moved
    whole (bit for bit: the same kernels see the same values)."""
    n = (37, 23, 1) if lattice == D2Q9 else (13, 11, 9)
    outs = []
    for bound in (256 << 20, 1024, 3000):
        c = with_random_state(Case("chunks", lattice, n, 0.7), seed=6)
        rng = np.random.default_rng(3)
        ncell = int(np.prod(n))
        rho = 1 + 0.01 * rng.normal(size=ncell)
        u = 0.05 * rng.normal(size=(ncell, 3))
        if lattice == D2Q9:
            u[:, 2] = 0
        from paper_1710_02065_gb300 import lbm
        s = lbm.Solver(lattice, n, 0.7, PRECS["fp32"])
        lbm.lbm_set_transfer_staging(s.h, bound)
        s.set_state(rho, u)
        s.step(3)
        r1, u1, p1 = s.moments()
        s.set_populations(c.f0)
        s.step(2)
        f2 = s.populations()
        outs.append((r1, u1, p1, f2))
        s.close()
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("lattice", [D2Q9, D3Q19])
def test_page_locked_host_transfers_match_staged(lattice):
    """Page-locked host buffers (torch pinned memory) are read and written by
    the kernels directly; pageable ones go through the staging buffer.  State
    uploads and moment read-backs, FP64 and FP32 host arrays, must agree bit
    for bit, and a bad value in a page-locked upload is still named."""
    import torch
    from paper_1710_02065_gb300 import lbm
    n = (70, 33, 1) if lattice == D2Q9 else (40, 21, 13)
    ncell = int(np.prod(n))
    rng = np.random.default_rng(8)
    rho = 1 + 0.01 * rng.normal(size=ncell)
    u = 0.05 * rng.normal(size=(ncell, 3))
    if lattice == D2Q9:
        u[:, 2] = 0
    for dt, prec in ((np.float64, "fp64"), (np.float32, "fp32"), (np.float32, "fp16")):
        outs = []
        for pinned in (False, True):
            def buf(shape):
                if pinned:
                    return torch.zeros(shape, dtype=torch.float64 if dt == np.float64 else torch.float32).pin_memory().numpy()
                return np.zeros(shape, dtype=dt)
            r_in, u_in = buf(ncell), buf((ncell, 3))
            r_in[:] = rho
            u_in[:] = u
            ro, uo, po = buf(ncell), buf((ncell, 3)), buf((ncell, 6))
            s = lbm.Solver(lattice, n, 0.7, PRECS[prec])
            if dt == np.float64:
                lbm.lbm_set_state(s.h, r_in, u_in)
            else:
                lbm.lbm_set_state_f32(s.h, r_in, u_in)
            s.step(3)
            if dt == np.float64:
                lbm.lbm_moments(s.h, ro, uo, po)
            else:
                lbm.lbm_moments_f32(s.h, ro, uo, po)
            outs.append((ro.copy(), uo.copy(), po.copy(), s.populations()))
            if pinned:
                r_in[77] = -1.0
                with pytest.raises(lbm.LBMError) as e:
                    (lbm.lbm_set_state if dt == np.float64 else lbm.lbm_set_state_f32)(s.h, r_in, u_in)
                assert e.value.code == lbm.LBM_EINVAL and "rho[77]" in lbm.lbm_last_error(s.h)
            s.close()
        for a, b in zip(outs[0], outs[1]):
            assert np.array_equal(a, b), prec


def test_invalid_state_is_rejected_with_its_cell():
    from paper_1710_02065_gb300 import lbm
    n = (20, 10, 1)
    ncell = 200
    s = lbm.Solver(D2Q9, n, 0.7, PRECS["fp64"])
    lbm.lbm_set_transfer_staging(s.h, 1024)  # the bad cell sits in a later chunk
    rho, u = np.ones(ncell), np.zeros((ncell, 3))
    rho[150] = 0.0
    rho[170] = np.nan
    with pytest.raises(lbm.LBMError) as e:
        s.set_state(rho, u)
    assert e.value.code == lbm.LBM_EINVAL and "rho[150]" in lbm.lbm_last_error(s.h)
    rho[150] = rho[170] = 1.0
    u[33, 2] = 1e-3
    with pytest.raises(lbm.LBMError) as e:
        s.set_state(rho, u)
    assert "cell 33" in lbm.lbm_last_error(s.h)
    u[33, 2] = 0.0
    s.set_state(rho, u)  # a valid state afterwards is taken as usual
    r, _, _ = s.moments()
    assert np.allclose(r, 1.0, atol=1e-15)
    s.close()


def test_async_force_and_probe_match_synchronous_calls():
    """lbm_force_async / lbm_probe_async record into device memory without a
    sync; their values equal lbm_force / lbm_probe (an out-of-range index
    gives NaN)."""
    torch = pytest.importorskip("torch")
    from paper_1710_02065_gb300 import lbm, inputs
    nx, ny = 96, 64
    s = lbm.Solver(D2Q9, (nx, ny, 1), 0.6, PRECS["fp64"])
    lbm.lbm_set_boundary(s.h, 0, lbm.LBM_BC_VELOCITY, (0.05, 0, 0))
    lbm.lbm_set_boundary(s.h, 1, lbm.LBM_BC_OUTFLOW)
    lbm.lbm_set_sponge(s.h, 1, 16, 0.5, 1.0, (0.05, 0, 0))
    solid = inputs.cylinder_mask(nx, ny, 30, 32, 10.0)
    lbm.lbm_set_geometry(s.h, solid)
    rho, u = np.ones(nx * ny), np.zeros((nx * ny, 3))
    u[:, 0] = 0.05
    u[solid == 1] = 0
    s.set_state(rho, u)
    cells = np.array([5 + nx * 7, 60 + nx * 40, nx * ny - 1], dtype=np.int64)
    cd = torch.tensor(list(cells) + [nx * ny], dtype=torch.int64, device="cuda")
    Fd = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    pd = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    F_ref, p_ref = [], []
    for k in range(4):
        s.step(5)
        F_ref.append(lbm.lbm_force(s.h, 0))
        p_ref.append(lbm.lbm_probe(s.h, cells))
        lbm.lbm_force_async(s.h, 0, Fd[k].data_ptr())
        lbm.lbm_probe_async(s.h, 4, cd.data_ptr(), pd[k].data_ptr())
    s.sync()
    torch.cuda.synchronize()
    assert np.abs(Fd.cpu().numpy() - np.array(F_ref)).max() == 0.0
    assert np.abs(F_ref[-1]).max() > 0
    p = pd.cpu().numpy()
    assert np.abs(p[:, :3] - np.array(p_ref)).max() <= 1e-17
    assert np.isnan(p[:, 3]).all()
    s.close()


def test_checkpoint_resume_is_bit_identical(tmp_path):
    c = _boxed_case(D2Q9, seed=4)
    a = to_gpu(c, PRECS["fp32"])
    a.step(5)
    from paper_1710_02065_gb300 import lbm
    path = str(tmp_path / "ck.bin")
    lbm.lbm_save(a.h, path)
    a.step(7)
    b = to_gpu(c, PRECS["fp32"])
    lbm.lbm_load(b.h, path)
    assert b.info()["step"] == 5
    b.step(7)
    assert np.array_equal(a.populations(), b.populations())


def test_full_size_cylinder_one_step():
    """1600 x 800 cylinder workload at full size, FP32, one step from a random
    off-equilibrium state, every cell compared with the oracle."""
    c = with_random_state(cylinder(), seed=21, spread=0.05)
    P, f = to_oracle(c)
    s = to_gpu(c, PRECS["fp32"])
    s.step(1)
    got = s.populations()
    ref = P.run(f, 1)
    _, _, _, w, _ = oracle.lattice(D2Q9)
    assert np.abs(got - ref).max() <= _pop_tol("fp32", ref, w, 1)


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
def test_full_size_round_jet_sampled_cells(prec):
    """384 x 256 x 256 round jet at full size, in every launch configuration
    the benchmark's autotuner may pick for the precision (one cell per thread,
    the vectorised kernel with 2 and 4 cells per thread, the row-staged
    kernel; two-lattice pull and in-place AA): one step from a random state
    (for AA a gather-push step, read back through the layout conversion);
    6000 sampled cells (random, plus every face, edge, sponge and inlet class)
    checked cell by cell."""
    from paper_1710_02065_gb300 import autotune
    c = round_jet()
    _, _, _, w, _ = oracle.lattice(D3Q19)
    c.f0 = inputs.random_populations(w, c.ncell, seed=31, spread=0.05)
    s = to_gpu(c, PRECS[prec])
    f0 = s.populations()  # the stored (possibly rounded) state is the oracle's input
    P = oracle.Problem(D3Q19, c.n, c.tau)
    for face, (kind, u, prof) in c.faces.items():
        P.set_boundary(face, kind, u, prof)
    for face, (wd, chi) in c.sponges.items():
        P.set_sponge(face, wd, chi, c.rho_ref, c.u_ref)
    P.noise_seed, P.noise_amp = c.noise
    nx, ny, nz = c.n
    rng = np.random.default_rng(5)
    cells = list(rng.integers(0, c.ncell, 4000))
    for x in (0, 1, 2, 3, nx - 1, nx - 2, nx - 3, nx - 20):
        for y in (0, 1, ny // 2, ny - 2, ny - 1, 3):
            for z in (0, 1, nz // 2, nz - 2, nz - 1, 250):
                cells.append(x + nx * (y + ny * z))
    # inlet disc cells
    for dy in range(-12, 13, 3):
        for dz in range(-12, 13, 3):
            cells.append(0 + nx * ((ny // 2 + dy) + ny * (nz // 2 + dz)))
    cells = np.unique(np.array(cells, dtype=np.int64))
    ref = P.update_cells(f0, cells, step=0)
    g = np.abs(ref - w[None, :]).max()
    ulp = {"fp16": 2.0 ** -10, "bf16": 2.0 ** -7}.get(prec)
    tol = 1e-5 * np.abs(ref).max() if prec == "fp32" else 2 * ulp * g + 1e-7
    s.close()
    kinds = sorted({k for k, _ in autotune.CANDIDATES[PRECS[prec]]} | {"cell", "vec2", "vec4", "aa-vec2"})
    for kind in kinds:
        s = to_gpu(c, PRECS[prec])  # a fresh handle: step 0 (the inlet noise is keyed by the step)
        use_kernel(s, kind)
        s.step(1)
        got = s.populations()
        s.close()
        err = np.abs(got[:, cells].T - ref).max()
        assert err <= tol, (kind, err, tol)


def _open_box(lattice, n, seed, rest=False):
    """Box without a mask: velocity inflow (profile + noise) on -x, outflow on
    +x, open or periodic y/z, sponges; random off-equilibrium state.  rest:
    the sponges relax to the rest state (the vectorised kernel's closed
    form; a moving reference runs the general kernel)."""
    c = Case("open", lattice, n, 0.56)
    nf = n[1] * n[2]
    prof = np.zeros((nf, 3))
    prof[:, 0] = 0.05 * (0.5 + np.random.default_rng(seed).random(nf))
    c.faces = {0: (VELOCITY, (0, 0, 0), prof), 1: (OUTFLOW, (0, 0, 0), None)}
    c.sponges = {1: (5, 0.8)}
    if lattice == D3Q19:
        c.faces[2] = (OUTFLOW, (0, 0, 0), None)
        c.faces[3] = (VELOCITY, (0.01, -0.02, 0.0), None)
        c.sponges[4] = (3, 0.5)
    else:
        c.faces[2] = (VELOCITY, (0.0, 0.01, 0.0), None)
        c.faces[3] = (OUTFLOW, (0, 0, 0), None)
    c.noise = (9, 0.05)
    c.rho_ref, c.u_ref = 1.0, ((0.0, 0.0, 0.0) if rest else (0.01, 0.0, 0.0))
    return with_random_state(c, seed=seed, spread=0.08)


@pytest.mark.parametrize("prec", list(PRECS))
@pytest.mark.parametrize("lattice", [D2Q9, D3Q19])
def test_launch_shapes_match_oracle(lattice, prec):
    """Scalar and vectorised kernels, several block sizes, partial warps
    (nx/V not a multiple of 32), periodic and open x, sponges relaxing to the
    rest state (the vectorised kernel) and to a moving state (the general
    kernel): all equal the oracle."""
    from paper_1710_02065_gb300 import lbm
    _, _, _, w, _ = oracle.lattice(lattice)
    vecs = {"fp64": [1, 2], "fp32": [1, 2, 4], "fp16": [1, 2, 4], "bf16": [1, 2, 4]}[prec]
    sizes = [(40, 12, 1), (136, 7, 1)] if lattice == D2Q9 else [(24, 10, 6), (136, 5, 4)]
    for n, rest in [(n, r) for n in sizes for r in (True, False)]:
        c = _open_box(lattice, n, seed=n[0], rest=rest)
        P, f = to_oracle(c)
        ref = P.run(f, 3)
        tol = _pop_tol(prec, ref, w, 3)
        for vec in vecs:
            for block in (32, 128, 256):
                s = to_gpu(c, PRECS[prec])
                lbm.lbm_set_staging(s.h, 0, 0, 0)
                lbm.lbm_set_launch(s.h, block, vec)
                assert lbm.lbm_get_launch(s.h) == (block, vec)
                s.step(3)
                err = np.abs(s.populations() - ref).max()
                assert err <= tol, (n, vec, block, err)
                s.close()
        # periodic x (vectorised kernel wraps through lane 0 / lane 31 loads)
        cp = with_random_state(Case("periodic", lattice, n, 0.7), seed=3)
        P, f = to_oracle(cp)
        ref = P.run(f, 2)
        for vec in vecs:
            s = to_gpu(cp, PRECS[prec])
            lbm.lbm_set_staging(s.h, 0, 0, 0)
            lbm.lbm_set_launch(s.h, 64, vec)
            s.step(2)
            assert np.abs(s.populations() - ref).max() <= _pop_tol(prec, ref, w, 2)
            s.close()


def test_graph_replay_matches_direct_launches():
    """lbm_step on a non-default stream replays captured step pairs; the result
    is bitwise that of launching every step (single level with walls, open
    jet, and the two-level grid), and a configuration change recaptures."""
    import torch
    from paper_1710_02065_gb300 import lbm
    from cases import cylinder_two_level
    stream = torch.cuda.Stream()

    def pair(c, setup=None):
        a = to_gpu(c, PRECS["fp32"])                     # legacy stream: direct launches
        b = lbm.Solver(c.lattice, c.n, c.tau, PRECS["fp32"], stream=stream.cuda_stream)
        for face, spec in c.faces.items():
            lbm.lbm_set_boundary(b.h, face, spec[0], spec[1], spec[2])
        for face, (w, chi) in c.sponges.items():
            lbm.lbm_set_sponge(b.h, face, w, chi, c.rho_ref, c.u_ref)
        if c.solid is not None:
            lbm.lbm_set_geometry(b.h, c.solid)
        b.set_state(c.rho0, c.u0) if c.f0 is None else b.set_populations(c.f0)
        if setup:
            setup(a)
            setup(b)
        return a, b

    c = cylinder(120, 60, diameter=8.0, sponge=20)
    a, b = pair(c)
    a.step(11)
    b.step(7)
    b.step(4)
    torch.cuda.synchronize()
    assert np.array_equal(a.populations(), b.populations())
    assert a.info()["step"] == b.info()["step"] == 11
    # configuration change between calls: recaptured graph
    lbm.lbm_set_sponge(a.h, 1, 10, 0.9, c.rho_ref, c.u_ref)
    lbm.lbm_set_sponge(b.h, 1, 10, 0.9, c.rho_ref, c.u_ref)
    a.step(6)
    b.step(6)
    assert np.array_equal(a.populations(), b.populations())
    # a long call: one graph of 16 step pairs replayed, the rest direct
    a.step(41)
    b.step(41)
    b.step(41)
    a.step(41)
    assert np.array_equal(a.populations(), b.populations())
    assert a.info()["step"] == b.info()["step"] == 11 + 6 + 82
    # calls of varying length, odd and even, at both parities: the cached
    # graphs of 16, 8, 4, 2 and 1 pairs, and direct odd last steps
    for n in (63, 7, 30, 1, 63, 2, 17):
        b.step(n)
    a.step(63 + 7 + 30 + 1 + 63 + 2 + 17)
    assert np.array_equal(a.populations(), b.populations())
    assert a.info()["step"] == b.info()["step"] == 11 + 6 + 82 + 183

    cj = round_jet(32, 24, 24, diameter=6.0, sponge=6, Re=1000.0, noise=0.0)
    a, b = pair(cj)
    a.step(9)
    b.step(9)
    assert np.array_equal(a.populations(), b.populations())

    c2, patch, rho_f, u_f, solid_f = cylinder_two_level(100, 60, (20, 16, 40, 24), diameter_c=5.0, sponge=10)

    def refine(s):
        lbm.lbm_add_refinement_patch(s.h, (patch[0], patch[1], 0), (patch[2], patch[3], 1))
        lbm.lbm_set_geometry_level(s.h, 1, solid_f)
        lbm.lbm_set_state_level(s.h, 1, rho_f, u_f)
        lbm.lbm_set_state(s.h, c2.rho0, c2.u0)

    a, b = pair(c2, refine)
    a.step(10)
    b.step(5)
    b.step(5)
    torch.cuda.synchronize()
    assert np.array_equal(a.populations(), b.populations())
    fa = np.zeros((9, 81 * 49)); fb = np.zeros((9, 81 * 49))
    lbm.lbm_get_populations_level(a.h, 1, fa)
    lbm.lbm_get_populations_level(b.h, 1, fb)
    assert np.array_equal(fa, fb)


def _slip_box(lattice, n, seed):
    """Velocity inflow, constant-pressure outlet, free-slip lateral walls,
    a sponge; random off-equilibrium state."""
    c = Case("slip", lattice, n, 0.57)
    c.faces = {0: (VELOCITY, (0.05, 0.0, 0.0), None), 1: (PRESSURE, None, None, 1.003),
               2: (FREESLIP, None, None), 3: (FREESLIP, None, None)}
    if lattice == D3Q19:
        c.faces[4] = (FREESLIP, None, None)
        c.faces[5] = (PRESSURE, None, None, 0.998)
    c.sponges = {1: (4, 0.4)}
    c.rho_ref, c.u_ref = 1.0, (0.05, 0.0, 0.0)
    return with_random_state(c, seed=seed, spread=0.08)


@pytest.mark.parametrize("prec", list(PRECS))
@pytest.mark.parametrize("lattice", [D2Q9, D3Q19])
def test_free_slip_and_pressure_faces_match_oracle(lattice, prec):
    from paper_1710_02065_gb300 import lbm
    _, _, _, w, _ = oracle.lattice(lattice)
    n = (40, 14, 1) if lattice == D2Q9 else (24, 12, 10)
    c = _slip_box(lattice, n, seed=8)
    P, f = to_oracle(c)
    ref = P.run(f, 3)
    for kind in KERNELS[prec]:
        s = to_gpu(c, PRECS[prec])
        use_kernel(s, kind)
        s.step(3)
        err = np.abs(s.populations() - ref).max()
        assert err <= _pop_tol(prec, ref, w, 3), (kind, err)
        s.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
@pytest.mark.parametrize("lattice", [D2Q9, D3Q19])
def test_radial_sponge_matches_oracle(lattice, prec):
    """Circular / spherical sponge combined with a planar one, open faces."""
    from paper_1710_02065_gb300 import lbm
    _, _, _, w, _ = oracle.lattice(lattice)
    n = (48, 40, 1) if lattice == D2Q9 else (32, 24, 20)
    c = Case("radial", lattice, n, 0.6)
    c.faces = {0: (VELOCITY, (0.04, 0.0, 0.0), None), 1: (OUTFLOW, None, None)}
    c.sponges = {1: (5, 0.3)}
    center = (n[0] / 2, n[1] / 2, n[2] / 2 if lattice == D3Q19 else 0)
    c.radial = (center, 6.0, 8.0, 0.7)
    c.rho_ref, c.u_ref = 1.0, (0.04, 0.0, 0.0)
    c = with_random_state(c, seed=12, spread=0.06)
    P, f = to_oracle(c)
    ref = P.run(f, 3)
    for kind in KERNELS[prec]:
        s = to_gpu(c, PRECS[prec])
        use_kernel(s, kind)
        s.step(3)
        assert np.abs(s.populations() - ref).max() <= _pop_tol(prec, ref, w, 3), kind
        s.close()


def _staged_cases(lattice):
    """Shapes for the row-staged kernel: whole-plane tiles, several rows per
    tile with a ragged last tile in y, one row per tile; open y/z (boundary
    rows stream from their inward neighbour) and periodic y/z (wrapped
    source rows split a tile's copies into runs)."""
    if lattice == D2Q9:
        return [(40, 12, 1), (512, 7, 1), (64, 9, 1)]
    return [(24, 10, 6), (192, 10, 5), (96, 7, 9)]


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("lattice", [D2Q9, D3Q19])
def test_staged_kernel_matches_oracle(lattice, prec):
    """Row-staged kernel against the oracle: tile shapes, stage counts,
    threads per CTA below and above a tile's cell count, open and periodic
    axes with inflow profile + noise, outflow and sponges."""
    from paper_1710_02065_gb300 import lbm
    _, _, _, w, _ = oracle.lattice(lattice)
    for n in _staged_cases(lattice):
        for periodic in (False, True):
            c = _open_box(lattice, n, seed=n[0] + n[1])
            if periodic:
                for f in range(2, 6 if lattice == D3Q19 else 4):
                    c.faces.pop(f, None)
                c.sponges = {1: (5, 0.8)}
            P, f = to_oracle(c)
            ref = P.run(f, 3)
            tol = _pop_tol(prec, ref, w, 3)
            for stages, block in ((0, 0), (3, 32), (5, 384), (2, 96)):
                s = to_gpu(c, PRECS[prec])
                lbm.lbm_set_staging(s.h, 1, stages, block)
                active, ns, b, R, grid = lbm.lbm_get_staging(s.h)
                assert active == 1 and ns == max(stages, 2) and R >= 1 and grid >= 1
                assert b == block or block == 0
                s.step(3)
                err = np.abs(s.populations() - ref).max()
                assert err <= tol, (n, periodic, stages, block, R, err)
                s.sync()
                s.close()


def test_staged_kernel_bounded_wait_reports_and_recovers():
    """Failure path of the row-staged kernel's bounded wait for a tile's bulk
    copies, without any copy failing: with the wait limit at 0 every wait is
    one non-blocking test, so the copies of a tile just issued count as late.
    The kernel sets the handle's error word and each CTA awaits its copies in
    flight (2 s limit) before returning; lbm_sync reports LBM_ECUDA and clears
    the condition, and the handle stays usable: with the limit restored and
    the state set again, the steps match the oracle."""
    from paper_1710_02065_gb300 import lbm
    _, _, _, w, _ = oracle.lattice(D3Q19)
    c = _open_box(D3Q19, (32, 12, 6), seed=9)
    c.noise = (0, 0.0)  # steps keyed by their count would differ after the failed one
    P, f = to_oracle(c)
    ref = P.run(f, 2)
    s = to_gpu(c, PRECS["fp32"])
    lbm.lbm_set_staging(s.h, 1, 3, 0)
    assert lbm.lbm_get_staging(s.h)[0] == 1
    lbm.lbm_set_staging_wait(s.h, 0)
    s.step(1)
    with pytest.raises(lbm.LBMError) as e:
        s.sync()
    assert e.value.code == lbm.LBM_ECUDA
    assert "did not arrive" in lbm.lbm_last_error(s.h)
    s.sync()  # the error word was cleared; the context is intact
    lbm.lbm_set_staging_wait(s.h, 2_000_000_000)
    s.set_populations(f)
    s.step(2)
    s.sync()
    assert np.abs(s.populations() - ref).max() <= _pop_tol("fp32", ref, w, 2)
    s.close()


def test_staged_kernel_eligibility_and_fallback():
    """Rows that are not a multiple of 16 bytes, a cell-type mask, or FP64
    storage leave the row-staged kernel inactive and lbm_step falls back to
    the register kernels with the same results."""
    from paper_1710_02065_gb300 import lbm
    _, _, _, w, _ = oracle.lattice(D3Q19)
    for n, prec, masked in (((22, 9, 5), "fp32", False), ((36, 8, 5), "fp16", False),
                            ((32, 8, 5), "fp32", True), ((32, 8, 5), "fp64", False)):
        c = _open_box(D3Q19, n, seed=4)
        if masked:
            solid = np.zeros(n[::-1], np.uint8)
            solid[2:4, 3:5, 10:14] = 1
            c.solid = solid.reshape(-1)
        P, f = to_oracle(c)
        ref = P.run(f, 2)
        s = to_gpu(c, PRECS[prec])
        lbm.lbm_set_staging(s.h, 1, 0, 0)
        assert lbm.lbm_get_staging(s.h)[0] == 0, (n, prec, masked)
        s.step(2)
        assert np.abs(s.populations() - ref).max() <= _pop_tol(prec, ref, w, 2)
        s.close()


@pytest.mark.parametrize("prec", list(PRECS))
@pytest.mark.parametrize("lattice", [D2Q9, D3Q19])
def test_plain_bgk_matches_oracle(lattice, prec):
    """Plain LBM-BGK (Eq. standardLB, quadratic equilibrium): every boundary
    rule (inflow profile + noise, outflow, sponges, bounce-back solid) and the
    free-slip / constant-pressure faces, against the oracle's BGK."""
    from paper_1710_02065_gb300 import lbm
    _, _, _, w, _ = oracle.lattice(lattice)
    n = (40, 14, 1) if lattice == D2Q9 else (24, 12, 10)
    for c in (_boxed_case(lattice, seed=6), _slip_box(lattice, n, seed=9)):
        P, f = to_oracle(c)
        P.collision = oracle.BGK
        ref = P.run(f, 3)
        s = to_gpu(c, PRECS[prec])
        lbm.lbm_set_collision(s.h, lbm.LBM_COLLISION_BGK)
        s.step(3)
        err = np.abs(s.populations() - ref).max()
        assert err <= _pop_tol(prec, ref, w, 3), (c.name, err)
        # the two collision models differ on this state by far more than the
        # FP64 / FP32 tolerances (and more than the 16-bit ones)
        P.collision = oracle.RR
        assert np.abs(P.run(f, 3) - ref).max() > 5 * _pop_tol(prec, ref, w, 3)
        s.close()


def test_collision_model_and_refinement_exclude_each_other():
    from paper_1710_02065_gb300 import lbm
    s = lbm.Solver(D2Q9, (40, 30, 1), 0.6, PRECS["fp32"])
    lbm.lbm_set_collision(s.h, lbm.LBM_COLLISION_BGK)
    with pytest.raises(lbm.LBMError):
        lbm.lbm_add_refinement_patch(s.h, (10, 8, 0), (16, 12, 1))
    lbm.lbm_set_collision(s.h, lbm.LBM_COLLISION_RR)
    lbm.lbm_add_refinement_patch(s.h, (10, 8, 0), (16, 12, 1))
    with pytest.raises(lbm.LBMError):
        lbm.lbm_set_collision(s.h, lbm.LBM_COLLISION_BGK)
    with pytest.raises(lbm.LBMError):
        lbm.lbm_set_collision(s.h, 7)
    s.close()


@pytest.mark.parametrize("prec", list(PRECS))
def test_jet_similarity_sponge_reference_matches_oracle(prec):
    """Outflow sponge with the round-jet similarity reference (Sec. IV), a
    jet inflow profile, outflow and lateral sponges; every kernel."""
    from paper_1710_02065_gb300 import lbm
    _, _, _, w, _ = oracle.lattice(D3Q19)
    n = (48, 24, 24)
    c = Case("jetref", D3Q19, n, 0.56)
    prof = inputs.top_hat_profile(n[1], n[2], n[1] / 2, n[2] / 2, 4.0, 0.08, 1.0)
    c.faces = {0: (VELOCITY, (0, 0, 0), prof), 1: (OUTFLOW, (0, 0, 0), None)}
    c.sponges = {1: (16, 0.6), 3: (4, 0.3)}
    c.rho_ref, c.u_ref = 1.0, (0.0, 0.0, 0.0)
    c = with_random_state(c, seed=21, spread=0.05)
    jet = (n[1] / 2 - 0.5, n[2] / 2 - 0.5, 0.08, 3.0, 18.0, 5.8, 0.094)  # capped for x < 35.4, decaying beyond
    P, f = to_oracle(c)
    P.set_jet_reference(*jet)
    ref = P.run(f, 3)
    P0, _ = to_oracle(c)
    assert np.abs(P0.run(f, 3) - ref).max() > 1e-6  # the reference changes the result
    for kind in KERNELS[prec]:
        s = to_gpu(c, PRECS[prec])
        lbm.lbm_set_sponge_jet_reference(s.h, *jet)
        use_kernel(s, kind)
        s.step(3)
        err = np.abs(s.populations() - ref).max()
        assert err <= _pop_tol(prec, ref, w, 3), (kind, err)
        s.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 5e-7)])
def test_pressure_fluctuation_matches_oracle(prec, tol):
    """Delta p~ = c_s^2 (rho - temporal mean rho) (Sec. III) over 12 sampled
    steps of the D2Q9 acoustic pulse, and the mean Delta p, against the same
    averages of the oracle's fields (absolute tolerances: FP64 round-off; FP32
    storage keeps rho - 1 to about 1e-7)."""
    from paper_1710_02065_gb300 import lbm
    c = acoustic_pulse(64)
    P, f = to_oracle(c)
    s = to_gpu(c, PRECS[prec])
    with pytest.raises(lbm.LBMError):
        lbm.lbm_pressure_fluctuation(s.h, np.zeros(s.ncell), None)
    rhos = []
    for t in range(12):
        f = P.run(f, 1, step0=t)
        rhos.append(P.moments(f)[0])
        s.step(1)
        lbm.lbm_pressure_mean(s.h, lbm.LBM_MEAN_ACCUMULATE)
    mean = np.mean(rhos, axis=0)
    dp, dpm = np.zeros(s.ncell), np.zeros(s.ncell)
    lbm.lbm_pressure_fluctuation(s.h, dp, dpm)
    assert np.abs(dp - (rhos[-1] - mean) / 3).max() <= tol
    assert np.abs(dpm - (mean - 1) / 3).max() <= tol
    # reset: a single new sample makes Delta p~ vanish
    lbm.lbm_pressure_mean(s.h, lbm.LBM_MEAN_RESET)
    lbm.lbm_pressure_mean(s.h, lbm.LBM_MEAN_ACCUMULATE)
    lbm.lbm_pressure_fluctuation(s.h, dp, None)
    assert np.abs(dp).max() <= tol
    s.close()


D3Q27 = 2


@pytest.mark.parametrize("prec", list(PRECS))
def test_d3q27_all_boundary_rules_match_oracle(prec):
    """D3Q27 (full third order, H_xyz included): inflow profile + noise,
    outflow, sponges, a bounce-back solid and random off-equilibrium
    populations, general and two-cell kernels, plain BGK as well."""
    from paper_1710_02065_gb300 import lbm
    _, _, _, w, _ = oracle.lattice(D3Q27)
    c = _boxed_case(D3Q27, seed=13)
    assert c.q == 27
    P, f = to_oracle(c)
    ref = P.run(f, 3)
    tol = _pop_tol(prec, ref, w, 3)
    s = to_gpu(c, PRECS[prec])
    s.step(3)
    assert np.abs(s.populations() - ref).max() <= tol
    s.close()
    for rest in (True, False):
        co = _open_box(D3Q27, (24, 10, 6), seed=31, rest=rest)
        P, f = to_oracle(co)
        ref = P.run(f, 3)
        for kind in ("cell", "vec2"):
            s = to_gpu(co, PRECS[prec])
            use_kernel(s, kind)
            s.step(3)
            assert np.abs(s.populations() - ref).max() <= _pop_tol(prec, ref, w, 3), (kind, rest)
            s.close()
    P.collision = oracle.BGK
    ref = P.run(f, 3)
    s = to_gpu(co, PRECS[prec])
    lbm.lbm_set_collision(s.h, lbm.LBM_COLLISION_BGK)
    s.step(3)
    assert np.abs(s.populations() - ref).max() <= _pop_tol(prec, ref, w, 3)
    s.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_d3q27_taylor_green_parity(prec, tol):
    c = taylor_green_3d(16, lattice=D3Q27)
    P, f = to_oracle(c)
    ref = P.run(f, 60)
    r_ref, u_ref, _ = P.moments(ref)
    s = to_gpu(c, PRECS[prec])
    s.step(60)
    r, u, _ = s.moments()
    assert _normwise(r, r_ref) <= tol and _normwise(u, u_ref) <= tol
    s.close()


@pytest.mark.parametrize("prec", list(PRECS))
def test_d2q9_fourth_order_matches_oracle(prec):
    """Optional fourth-order D2Q9 term (H_xxyy): every boundary rule, a solid,
    noise, sponges, random populations, on every kernel; a 200-step acoustic
    pulse started from the order-4 equilibrium."""
    from paper_1710_02065_gb300 import lbm
    _, _, _, w, _ = oracle.lattice(D2Q9)
    c = _boxed_case(D2Q9, seed=17)
    P, f = to_oracle(c)
    P.order4 = 1
    ref = P.run(f, 3)
    P.order4 = 0
    assert np.abs(P.run(f, 3) - ref).max() > 1e-8  # the term is active on this state
    s = to_gpu(c, PRECS[prec])
    lbm.lbm_set_hermite_order(s.h, 4)
    s.step(3)
    assert np.abs(s.populations() - ref).max() <= _pop_tol(prec, ref, w, 3)
    s.close()
    co = _open_box(D2Q9, (40, 12, 1), seed=23)
    P, f = to_oracle(co)
    P.order4 = 1
    ref = P.run(f, 3)
    for kind in KERNELS[prec]:
        s = to_gpu(co, PRECS[prec])
        lbm.lbm_set_hermite_order(s.h, 4)
        use_kernel(s, kind)
        s.step(3)
        assert np.abs(s.populations() - ref).max() <= _pop_tol(prec, ref, w, 3), kind
        s.close()
    if prec in ("fp64", "fp32"):
        tol = 1e-12 if prec == "fp64" else 1e-5
        cp = acoustic_pulse(96)
        P, _ = to_oracle(cp)
        P.order4 = 1
        f0 = P.equilibrium(cp.rho0, cp.u0)
        ref = P.run(f0, 200)
        r_ref, u_ref, _ = P.moments(ref)
        s = lbm.Solver(D2Q9, cp.n, cp.tau, PRECS[prec])
        lbm.lbm_set_hermite_order(s.h, 4)
        s.set_state(cp.rho0, cp.u0)
        s.step(200)
        r, u, _ = s.moments()
        assert _normwise(r, r_ref) <= tol and _normwise(u, u_ref) <= tol
        with pytest.raises(lbm.LBMError):
            lbm.lbm_add_refinement_patch(s.h, (10, 10, 0), (20, 20, 1))
        s.close()


@pytest.mark.parametrize("lattice", [D2Q9, D3Q19])
def test_sponge_changed_between_steps_matches_oracle(lattice):
    """Sponge layers set, widened and removed between steps (the per-axis
    strength tables are re-uploaded in stream order, after the steps already
    queued) give the oracle's result with the same sequence of settings."""
    from paper_1710_02065_gb300 import lbm
    c = with_random_state(Case("responge", lattice, (40, 24, 1) if lattice == D2Q9 else (24, 16, 12), 0.7),
                          seed=9, spread=0.02)
    c.faces = {0: (OUTFLOW, (0, 0, 0), None), 1: (OUTFLOW, (0, 0, 0), None)}
    P, f = to_oracle(c)
    s = to_gpu(c, PRECS["fp64"])
    plan = [(3, {1: (8, 0.5)}), (4, {1: (12, 0.8), 0: (5, 0.3)}), (3, {1: (0, 0.0)}), (2, {})]
    step = 0
    for nsteps, changes in plan:
        for face, (w, chi) in changes.items():
            P.set_sponge(face, w, chi, 1.0, (0, 0, 0))
            lbm.lbm_set_sponge(s.h, face, w, chi, 1.0, (0.0, 0.0, 0.0))
        f = P.run(f, nsteps, step0=step)
        s.step(nsteps)  # queued without a sync: the next table upload must wait for these steps
        step += nsteps
    r_ref, u_ref, _ = P.moments(f)
    r, u, _ = s.moments()
    assert _normwise(r, r_ref) <= 1e-12
    assert _normwise(u, u_ref) <= 1e-12
    s.close()
