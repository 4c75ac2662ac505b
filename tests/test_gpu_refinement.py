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
