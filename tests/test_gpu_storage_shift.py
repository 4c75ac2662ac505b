"""Storage shifted by a reference equilibrium (lbm_set_storage_shift): the
populations are stored as f_i - feqH_i(1, u_s) instead of f_i - w_i.

On a mean flow u_s the stored values are then the acoustic and off-equilibrium
parts only, so the 16-bit formats round them at that scale.  The update is the
same arithmetic (the shift is added on load and removed on store), so the
results must match the FP64 oracle with the rounding bound taken on the
shifted magnitude max |f - feqH(1, u_s)|, and be far more accurate than the
default shift for 16-bit storage.
"""
import numpy as np
import pytest

import oracle
from cases import D2Q9, acoustic_pulse, cylinder, to_gpu, to_oracle
from test_gpu_parity import PRECS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_02065_gb300 import build
    build.build()


def _shifted_pulse(prec, u_s, n=64):
    from paper_1710_02065_gb300 import lbm
    c = acoustic_pulse(n)
    s = lbm.Solver(c.lattice, c.n, c.tau, PRECS[prec])
    lbm.lbm_set_storage_shift(s.h, u_s)
    s.set_state(c.rho0, c.u0)
    return c, s


def _bound(prec, ref, base, steps):
    if prec == "fp64":
        return 1e-13
    if prec == "fp32":
        return 1e-5 * np.abs(ref).max()
    bits = 10 if prec == "fp16" else 7
    return (steps + 1) * 2.0 ** -bits * np.abs(ref - base[:, None]).max() + 1e-9


@pytest.mark.parametrize("prec", list(PRECS))
def test_shifted_pulse_matches_oracle(prec):
    """D2Q9 pulse of amplitude 1e-3 on u0 = (0.05, 0): with u_s = u0 every
    precision matches the oracle within the rounding of the shifted values;
    16-bit storage is at least 10x more accurate than with the default shift."""
    u0 = (0.05, 0.0, 0.0)
    c, s = _shifted_pulse(prec, u0)
    P, f = to_oracle(c)
    ref = P.run(f, 40)
    s.step(40)
    got = s.populations()
    s.close()
    feq = oracle.feqH(D2Q9, 1.0, u0)
    err = np.abs(got - ref).max()
    assert err <= _bound(prec, ref, feq, 40), err
    if prec in ("fp16", "bf16"):
        plain = to_gpu(c, PRECS[prec])
        plain.step(40)
        err_plain = np.abs(plain.populations() - ref).max()
        plain.close()
        assert err_plain > 10 * err, (err_plain, err)


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_shifted_cylinder_with_walls_inflow_and_sponge_matches_oracle(prec):
    """Cylinder (halfway bounce-back, velocity inflow, outflow, sponge relaxing
    to (1, U)), stored shifted by the inflow equilibrium: bounced populations
    carry the shift of the array they are read from."""
    from paper_1710_02065_gb300 import lbm
    c = cylinder(96, 48, diameter=10.0, sponge=16)
    P, f = to_oracle(c)
    ref = P.run(f, 12)
    s = lbm.Solver(c.lattice, c.n, c.tau, PRECS[prec])
    lbm.lbm_set_storage_shift(s.h, c.u_ref)
    for face, (kind, u, prof) in c.faces.items():
        lbm.lbm_set_boundary(s.h, face, kind, u, prof)
    for face, (w, chi) in c.sponges.items():
        lbm.lbm_set_sponge(s.h, face, w, chi, c.rho_ref, c.u_ref)
    lbm.lbm_set_geometry(s.h, c.solid)
    s.set_state(c.rho0, c.u0)
    s.step(12)
    err = np.abs(s.populations() - ref).max()
    s.close()
    assert err <= _bound(prec, ref, oracle.feqH(D2Q9, 1.0, c.u_ref), 12), err


def test_shift_change_mid_run_and_checkpoints(tmp_path):
    """FP64: changing the shift re-expresses the stored field exactly enough
    that the run continues on the oracle's trajectory; a checkpoint records
    the shift and loads only into a handle with the same one."""
    from paper_1710_02065_gb300 import lbm
    c = acoustic_pulse(48)
    P, f = to_oracle(c)
    s = to_gpu(c, PRECS["fp64"])
    s.step(7)
    lbm.lbm_set_storage_shift(s.h, (0.05, 0.0, 0.0))
    s.step(6)
    assert np.abs(s.populations() - P.run(f, 13)).max() <= 1e-13
    path = str(tmp_path / "shift.bin")
    lbm.lbm_save(s.h, path)
    lbm.lbm_set_storage_shift(s.h, None)
    s.step(5)
    assert np.abs(s.populations() - P.run(f, 18)).max() <= 1e-13
    b = lbm.Solver(c.lattice, c.n, c.tau, PRECS["fp64"])
    with pytest.raises(lbm.LBMError):
        lbm.lbm_load(b.h, path)
    lbm.lbm_set_storage_shift(b.h, (0.05, 0.0, 0.0))
    lbm.lbm_load(b.h, path)
    b.step(5)
    assert np.abs(b.populations() - P.run(f, 18)).max() <= 1e-13
    with pytest.raises(lbm.LBMError):
        lbm.lbm_set_streaming(b.h, lbm.LBM_STREAM_AA)
    s.close()
    b.close()
