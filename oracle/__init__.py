"""FP64 CPU oracle for the recursive Hermite-regularized LBM (arXiv:1710.02065).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product library never calls it, and nothing here imports the product package.

The arithmetic lives in ``rrlbm_oracle.c`` (plain loops, FP64); this module
compiles it with the host C compiler and wraps it with ctypes/numpy.

Each function cites the part of the paper it follows:
  * ``feqH``      -- Eq. eqH with Eq. recursive1 (Sec. II.A)
  * ``fneqH``     -- Eq. neqH with Eq. recursive2 at n = 3 (Sec. II.A)
  * ``collide``   -- Eq. optimizedLB, and Eq. spongeLB / Eq. dampingLBM (Sec. II.C)
  * ``Problem.step`` -- pull streaming (left side of Eq. optimizedLB) plus the
    boundary rules of Sec. III (velocity inflow, zero-gradient outflow,
    bounce-back walls) and the sponge layers of Sec. II.C.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rrlbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

D2Q9, D3Q19, D3Q27 = 0, 1, 2
_Q = {D2Q9: 9, D3Q19: 19, D3Q27: 27}
PERIODIC, VELOCITY, OUTFLOW, FREESLIP, PRESSURE = 0, 1, 2, 3, 4
RR, BGK = 0, 1  # collision models
CS2 = 1.0 / 3.0


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (host C compiler)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cc = os.environ.get("CC", "gcc")
        subprocess.check_call([cc, "-O2", "-std=c99", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(C.Structure):
    _fields_ = [
        ("lattice", C.c_int),
        ("n", C.c_int * 3),
        ("tau", C.c_double),
        ("face_kind", C.c_int * 6),
        ("u_face", (C.c_double * 3) * 6),
        ("rho_face", C.c_double * 6),
        ("u_profile", C.POINTER(C.c_double) * 6),
        ("noise_seed", C.c_uint64),
        ("noise_amp", C.c_double),
        ("sponge_width", C.c_int * 6),
        ("sponge_chi", C.c_double * 6),
        ("rho_ref", C.c_double),
        ("u_ref", C.c_double * 3),
        ("radial", C.c_double * 6),
        ("solid", C.POINTER(C.c_uint8)),
        ("g", C.c_double * 3),
        ("collision", C.c_int),
        ("jet_ref", C.c_double * 7),
        ("order4", C.c_int),
    ]


class _Patch(C.Structure):
    _fields_ = [("X0", C.c_int), ("Y0", C.c_int), ("Wc", C.c_int), ("Hc", C.c_int)]


class _Patch3(C.Structure):
    _fields_ = [("X0", C.c_int), ("Y0", C.c_int), ("Z0", C.c_int), ("Wc", C.c_int), ("Hc", C.c_int),
                ("Dc", C.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            P = C.POINTER(_Problem)
            _lib.orc_lattice.argtypes = [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                         C.POINTER(C.c_int), dp, C.POINTER(C.c_int)]
            _lib.orc_feqH.argtypes = [C.c_int, C.c_double, dp, dp]
            _lib.orc_fneqH.argtypes = [C.c_int, dp, dp, dp]
            _lib.orc_collide.argtypes = [C.c_int, dp, C.c_double, C.c_double, C.c_double, dp, dp, C.c_int, dp]
            _lib.orc_step.argtypes = [P, dp, dp, C.c_int64]
            _lib.orc_run.argtypes = [P, dp, dp, C.c_int64, C.c_int64]
            _lib.orc_run_threads.argtypes = [P, dp, dp, C.c_int64, C.c_int64, C.c_int]
            _lib.orc_update_cell.argtypes = [P, dp, C.c_int64, C.c_int64, dp]
            _lib.orc_update_cells.argtypes = [P, dp, C.c_int64, C.POINTER(C.c_int64), C.c_int64, dp]
            _lib.orc_field_moments.argtypes = [P, dp, dp, dp, dp]
            _lib.orc_init_equilibrium.argtypes = [P, dp, dp, dp]
            _lib.orc_wall_force.argtypes = [P, dp, dp]
            _lib.orc_chi_at.argtypes = [P, C.c_int, C.c_int, C.c_int]
            _lib.orc_chi_at.restype = C.c_double
            _lib.orc_sigma.argtypes = [C.c_double, C.c_double]
            _lib.orc_sigma.restype = C.c_double
            _lib.orc_splitmix64.argtypes = [C.c_uint64]
            _lib.orc_splitmix64.restype = C.c_uint64
            _lib.orc_u01.argtypes = [C.c_uint64]
            _lib.orc_u01.restype = C.c_double
            G = C.POINTER(_Patch)
            _lib.orc_refined_init_moments.argtypes = [P, G, dp, dp]
            _lib.orc_refined_step.argtypes = [P, P, G, dp, dp, dp, dp, dp, dp, C.c_int64]
            G3 = C.POINTER(_Patch3)
            _lib.orc_refined3_init_moments.argtypes = [P, G3, dp, dp]
            _lib.orc_refined3_step.argtypes = [P, P, G3, dp, dp, dp, dp, dp, dp, C.c_int64]
            _lib.orc_refine3_interp.argtypes = [P, G3, dp, dp, C.c_double, C.c_int, C.c_int, C.c_int, dp]
            _lib.orc_refine3_filter.argtypes = [dp, dp]
            _lib.orc_sponge_reference.argtypes = [P, C.c_int, C.c_int, C.c_int, dp]
            _lib.orc_refine2_line_moments.argtypes = [P, G, dp, dp]
            _lib.orc_refine2_fill.argtypes = [P, P, G, dp, dp, C.c_double, dp]
            _lib.orc_refine2_restrict.argtypes = [P, P, G, dp, dp]
            _lib.orc_refine3_plane_moments.argtypes = [P, G3, dp, dp]
            _lib.orc_refine3_fill.argtypes = [P, P, G3, dp, dp, C.c_double, dp]
            _lib.orc_refine3_restrict.argtypes = [P, P, G3, dp, dp]
        return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def lattice(which: int):
    """(d, q, xi[q,3] int, w[q], opp[q]) of D2Q9 (0), D3Q19 (1) or D3Q27 (2)."""
    d, q = C.c_int(), C.c_int()
    xi = np.zeros(27 * 3, dtype=np.int32)
    w = np.zeros(27)
    opp = np.zeros(27, dtype=np.int32)
    rc = lib().orc_lattice(which, C.byref(d), C.byref(q), xi.ctypes.data_as(C.POINTER(C.c_int)),
                           _dp(w), opp.ctypes.data_as(C.POINTER(C.c_int)))
    assert rc == 0
    q = q.value
    return d.value, q, xi.reshape(27, 3)[:q].copy(), w[:q].copy(), opp[:q].copy()


def feqH(which: int, rho: float, u) -> np.ndarray:
    """Hermite-regularized equilibrium, Eq. eqH (order 3, lattice-supported terms)."""
    q = _Q[which]
    out = np.zeros(q)
    lib().orc_feqH(which, float(rho), _dp(np.ascontiguousarray(u, dtype=np.float64)), _dp(out))
    return out


def fneqH(which: int, u, pi_neq) -> np.ndarray:
    """Hermite-regularized off-equilibrium part, Eq. neqH with Eq. recursive2."""
    q = _Q[which]
    out = np.zeros(q)
    pn = np.ascontiguousarray(np.asarray(pi_neq, dtype=np.float64).reshape(9))
    lib().orc_fneqH(which, _dp(np.ascontiguousarray(u, dtype=np.float64)), _dp(pn), _dp(out))
    return out


def collide(which: int, f, tau: float, chi: float = 0.0, rho_ref: float = 1.0,
            u_ref=(0.0, 0.0, 0.0), g=(0.0, 0.0, 0.0), order4: bool = False) -> np.ndarray:
    """One cell's rrBGK collision, Eq. optimizedLB (Eq. spongeLB when chi > 0)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros_like(f)
    lib().orc_collide(which, _dp(f), float(tau), float(chi), float(rho_ref),
                      _dp(np.ascontiguousarray(u_ref, dtype=np.float64)),
                      _dp(np.ascontiguousarray(g, dtype=np.float64)), int(bool(order4)), _dp(out))
    return out


def sigma(d: float, width: float) -> float:
    """Sponge profile of Sec. II.C, 3125 (W-d) d^4 / (256 W^5), d from the inner edge."""
    return lib().orc_sigma(float(d), float(width))


def splitmix64(x: int) -> int:
    return int(lib().orc_splitmix64(C.c_uint64(x & (2**64 - 1))))


def u01(counter: int) -> float:
    return float(lib().orc_u01(C.c_uint64(counter & (2**64 - 1))))


class Problem:
    """A single-level lattice with its boundary rules, mirroring the C struct."""

    def __init__(self, lattice: int, extents, tau: float):
        self.lattice = lattice
        n = list(extents) + [1] * (3 - len(extents))
        if lattice == D2Q9:
            n[2] = 1
        self.n = tuple(int(v) for v in n)
        self.q = _Q[lattice]
        self.tau = float(tau)
        self.face_kind = [PERIODIC] * 6
        self.u_face = [[0.0, 0.0, 0.0] for _ in range(6)]
        self.rho_face = [1.0] * 6
        self.u_profile = [None] * 6
        self.noise_seed = 0
        self.noise_amp = 0.0
        self.sponge_width = [0] * 6
        self.sponge_chi = [0.0] * 6
        self.rho_ref = 1.0
        self.u_ref = [0.0, 0.0, 0.0]
        self.solid = None
        self.g = [0.0, 0.0, 0.0]
        self.radial = [0.0] * 6
        self.collision = RR  # RR: rrBGK (Eq. optimizedLB); BGK: plain BGK (Eq. standardLB)
        self.jet_ref = [0.0] * 7  # yc, zc, U_J, D, x0, B, S of the +x sponge's jet reference; D = 0: none
        self.order4 = 0  # D2Q9: 1 adds the fourth-order H_xxyy term

    @property
    def ncell(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]

    def set_boundary(self, face: int, kind: int, u=(0.0, 0.0, 0.0), profile=None, rho=1.0):
        """kind PERIODIC, VELOCITY (u or profile), OUTFLOW, FREESLIP or PRESSURE (rho)."""
        self.face_kind[face] = kind
        self.rho_face[face] = float(rho)
        self.u_face[face] = [float(v) for v in (u if u is not None else (0.0, 0.0, 0.0))]
        self.u_profile[face] = None if profile is None else np.ascontiguousarray(profile, dtype=np.float64)

    def set_radial_sponge(self, center, r0: float, width: float, chi_max: float, rho_ref=1.0,
                          u_ref=(0.0, 0.0, 0.0)):
        c = list(center) + [0.0] * (3 - len(center))
        self.radial = [float(c[0]), float(c[1]), float(c[2]), float(r0), float(width), float(chi_max)]
        self.rho_ref = float(rho_ref)
        self.u_ref = [float(v) for v in u_ref]

    def set_jet_reference(self, yc: float, zc: float, U_jet: float, D: float, x0: float, B: float = 5.8,
                          S: float = 0.094):
        """Round-jet similarity reference for the cells of the +x sponge layer."""
        self.jet_ref = [float(yc), float(zc), float(U_jet), float(D), float(x0), float(B), float(S)]

    def sponge_reference(self, x: int, y: int, z: int) -> np.ndarray:
        u = np.zeros(3)
        s = self._struct()
        lib().orc_sponge_reference(C.byref(s), int(x), int(y), int(z), _dp(u))
        return u

    def set_sponge(self, face: int, width: int, chi_max: float, rho_ref=1.0, u_ref=(0.0, 0.0, 0.0)):
        self.sponge_width[face] = int(width)
        self.sponge_chi[face] = float(chi_max)
        self.rho_ref = float(rho_ref)
        self.u_ref = [float(v) for v in u_ref]

    def _struct(self) -> _Problem:
        s = _Problem()
        s.lattice = self.lattice
        for a in range(3):
            s.n[a] = self.n[a]
            s.u_ref[a] = self.u_ref[a]
            s.g[a] = self.g[a]
        s.tau = self.tau
        s.collision = self.collision
        for k in range(7):
            s.jet_ref[k] = self.jet_ref[k]
        s.order4 = int(self.order4)
        for f in range(6):
            s.face_kind[f] = self.face_kind[f]
            s.rho_face[f] = self.rho_face[f]
            for a in range(3):
                s.u_face[f][a] = self.u_face[f][a]
            s.u_profile[f] = _dp(self.u_profile[f]) if self.u_profile[f] is not None else None
            s.sponge_width[f] = self.sponge_width[f]
            s.sponge_chi[f] = self.sponge_chi[f]
        for k in range(6):
            s.radial[k] = self.radial[k]
        s.noise_seed = int(self.noise_seed)
        s.noise_amp = float(self.noise_amp)
        s.rho_ref = self.rho_ref
        if self.solid is not None:
            self._solid_keep = np.ascontiguousarray(self.solid.reshape(-1), dtype=np.uint8)
            s.solid = self._solid_keep.ctypes.data_as(C.POINTER(C.c_uint8))
        else:
            s.solid = None
        return s

    def equilibrium(self, rho: np.ndarray, u: np.ndarray) -> np.ndarray:
        """Field f = feqH(rho, u); rho shape (ncell,), u shape (ncell, 3)."""
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1, 3)
        f = np.zeros(self.q * self.ncell)
        s = self._struct()
        lib().orc_init_equilibrium(C.byref(s), _dp(rho), _dp(u), _dp(f))
        return f.reshape(self.q, self.ncell)

    def run(self, f: np.ndarray, nsteps: int, step0: int = 0, threads: int = 1) -> np.ndarray:
        """Advance a (q, ncell) field nsteps steps; returns the new field.
        threads > 1 splits each step's cells over host threads (bitwise the
        same result)."""
        f = np.array(f, dtype=np.float64, order="C").reshape(self.q, self.ncell)
        work = np.empty_like(f)
        s = self._struct()
        if threads > 1:
            rc = lib().orc_run_threads(C.byref(s), _dp(f), _dp(work), int(step0), int(nsteps), int(threads))
            if rc != 0:
                raise RuntimeError("oracle: could not start its threads")
        else:
            lib().orc_run(C.byref(s), _dp(f), _dp(work), int(step0), int(nsteps))
        return f

    def update_cell(self, f: np.ndarray, cell: int, step: int = 0) -> np.ndarray:
        """Post-collision populations of one cell from the full field f."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        out = np.zeros(self.q)
        s = self._struct()
        lib().orc_update_cell(C.byref(s), _dp(f), int(cell), int(step), _dp(out))
        return out

    def update_cells(self, f: np.ndarray, cells, step: int = 0) -> np.ndarray:
        """Post-collision populations (len(cells), q) of listed cells from the full field f."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        out = np.zeros((len(cells), self.q))
        s = self._struct()
        lib().orc_update_cells(C.byref(s), _dp(f), len(cells), cells.ctypes.data_as(C.POINTER(C.c_int64)),
                               int(step), _dp(out))
        return out

    def moments(self, f: np.ndarray):
        """(rho[ncell], u[ncell,3], pi_neq[ncell,6]) of a stored field."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        rho = np.zeros(self.ncell)
        u = np.zeros(3 * self.ncell)
        pn = np.zeros(6 * self.ncell)
        s = self._struct()
        lib().orc_field_moments(C.byref(s), _dp(f), _dp(rho), _dp(u), _dp(pn))
        return rho, u.reshape(-1, 3), pn.reshape(-1, 6)

    def wall_force(self, f: np.ndarray) -> np.ndarray:
        """Momentum-exchange force on the solid cells from the stored field f."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        F = np.zeros(3)
        s = self._struct()
        lib().orc_wall_force(C.byref(s), _dp(f), _dp(F))
        return F

    def chi(self, x: int, y: int, z: int = 0) -> float:
        s = self._struct()
        return lib().orc_chi_at(C.byref(s), x, y, z)


FLUID, SOLID, FIXED = 0, 1, 2


class TwoLevel:
    """Two-level 2:1 D2Q9 grid (Sec. II.B): a coarse Problem plus a fine patch
    over coarse nodes X0..X0+Wc, Y0..Y0+Hc, with tau_f = 2 tau_c - 1/2.

    The coarse problem carries its own boundaries; the fine one is periodic
    with its boundary ring fixed (rebuilt from coarse data every half step).
    The patch must keep 2 coarse nodes from every coarse face.
    """

    def __init__(self, coarse: Problem, X0: int, Y0: int, Wc: int, Hc: int):
        assert coarse.lattice == D2Q9
        nxc, nyc = coarse.n[0], coarse.n[1]
        assert X0 >= 2 and Y0 >= 2 and X0 + Wc <= nxc - 3 and Y0 + Hc <= nyc - 3 and Wc >= 4 and Hc >= 4
        self.Pc = coarse
        self.patch = (X0, Y0, Wc, Hc)
        self.Pf = Problem(D2Q9, (2 * Wc + 1, 2 * Hc + 1), 2 * coarse.tau - 0.5)
        cmask = np.zeros((nyc, nxc), np.uint8) if coarse.solid is None else coarse.solid.reshape(nyc, nxc).copy()
        cmask[Y0 + 1:Y0 + Hc, X0 + 1:X0 + Wc] = FIXED
        self.Pc.solid = cmask.reshape(-1)
        fmask = np.zeros((2 * Hc + 1, 2 * Wc + 1), np.uint8)
        fmask[0, :] = fmask[-1, :] = FIXED
        fmask[:, 0] = fmask[:, -1] = FIXED
        self.Pf.solid = fmask.reshape(-1)
        self.step_index = 0

    def set_fine_solid(self, solid_fine: np.ndarray):
        m = self.Pf.solid.reshape(self.Pf.n[1], self.Pf.n[0]).copy()
        s = np.asarray(solid_fine, np.uint8).reshape(m.shape)
        m[(s == SOLID) & (m != FIXED)] = SOLID
        self.Pf.solid = m.reshape(-1)

    def init(self, rho_c, u_c, rho_f, u_f):
        self.fc = self.Pc.equilibrium(rho_c, u_c)
        self.ff = self.Pf.equilibrium(rho_f, u_f)
        self.M0 = np.zeros(6 * self.Pc.ncell)
        self.M1 = np.zeros(6 * self.Pc.ncell)
        sc, g = self.Pc._struct(), _Patch(*self.patch)
        lib().orc_refined_init_moments(C.byref(sc), C.byref(g), _dp(self.fc), _dp(self.M0))
        self.step_index = 0

    def run(self, nsteps: int):
        sc, sf, g = self.Pc._struct(), self.Pf._struct(), _Patch(*self.patch)
        wc = np.empty_like(self.fc)
        wf = np.empty_like(self.ff)
        for _ in range(int(nsteps)):
            lib().orc_refined_step(C.byref(sc), C.byref(sf), C.byref(g), _dp(self.fc), _dp(wc),
                                   _dp(self.ff), _dp(wf), _dp(self.M0), _dp(self.M1), self.step_index)
            self.step_index += 1


class TwoLevel3:
    """Two-level 2:1 D3Q19 or D3Q27 grid (Sec. II.B): a coarse Problem plus a fine patch
    over coarse nodes X0..X0+Wc, Y0..Y0+Hc, Z0..Z0+Dc, tau_f = 2 tau_c - 1/2.

    The fine problem is periodic with its boundary shell fixed (rebuilt from
    coarse data every half step); the covered coarse interior is fixed, its
    first shell rebuilt from fine data every coarse step.  The patch must keep
    2 coarse nodes from every coarse face.
    """

    def __init__(self, coarse: Problem, X0: int, Y0: int, Z0: int, Wc: int, Hc: int, Dc: int):
        assert coarse.lattice in (D3Q19, D3Q27)
        nxc, nyc, nzc = coarse.n
        assert min(X0, Y0, Z0) >= 2 and min(Wc, Hc, Dc) >= 4
        assert X0 + Wc <= nxc - 3 and Y0 + Hc <= nyc - 3 and Z0 + Dc <= nzc - 3
        self.Pc = coarse
        self.patch = (X0, Y0, Z0, Wc, Hc, Dc)
        nf = (2 * Wc + 1, 2 * Hc + 1, 2 * Dc + 1)
        self.Pf = Problem(coarse.lattice, nf, 2 * coarse.tau - 0.5)
        shape_c = (nzc, nyc, nxc)
        cmask = np.zeros(shape_c, np.uint8) if coarse.solid is None else coarse.solid.reshape(shape_c).copy()
        cmask[Z0 + 1:Z0 + Dc, Y0 + 1:Y0 + Hc, X0 + 1:X0 + Wc] = FIXED
        self.Pc.solid = cmask.reshape(-1)
        fmask = np.zeros(nf[::-1], np.uint8)
        fmask[0, :, :] = fmask[-1, :, :] = FIXED
        fmask[:, 0, :] = fmask[:, -1, :] = FIXED
        fmask[:, :, 0] = fmask[:, :, -1] = FIXED
        self.Pf.solid = fmask.reshape(-1)
        self.step_index = 0

    def set_fine_solid(self, solid_fine: np.ndarray):
        m = self.Pf.solid.copy()
        s = np.asarray(solid_fine, np.uint8).reshape(-1)
        m[(s == SOLID) & (m != FIXED)] = SOLID
        self.Pf.solid = m

    def init(self, rho_c, u_c, rho_f, u_f):
        self.fc = self.Pc.equilibrium(rho_c, u_c)
        self.ff = self.Pf.equilibrium(rho_f, u_f)
        self.M0 = np.zeros(10 * self.Pc.ncell)
        self.M1 = np.zeros(10 * self.Pc.ncell)
        sc, g = self.Pc._struct(), _Patch3(*self.patch)
        lib().orc_refined3_init_moments(C.byref(sc), C.byref(g), _dp(self.fc), _dp(self.M0))
        self.step_index = 0

    def run(self, nsteps: int):
        sc, sf, g = self.Pc._struct(), self.Pf._struct(), _Patch3(*self.patch)
        wc = np.empty_like(self.fc)
        wf = np.empty_like(self.ff)
        for _ in range(int(nsteps)):
            lib().orc_refined3_step(C.byref(sc), C.byref(sf), C.byref(g), _dp(self.fc), _dp(wc),
                                    _dp(self.ff), _dp(wf), _dp(self.M0), _dp(self.M1), self.step_index)
            self.step_index += 1

    def interp(self, M0: np.ndarray, M1: np.ndarray, a: float, i: int, j: int, k: int) -> np.ndarray:
        """Coarse -> fine interface moments at fine shell node (i, j, k) from
        per-coarse-cell moment arrays (10 per cell), time weight a."""
        m = np.zeros(10)
        sc, g = self.Pc._struct(), _Patch3(*self.patch)
        lib().orc_refine3_interp(C.byref(sc), C.byref(g), _dp(np.ascontiguousarray(M0, dtype=np.float64)),
                                 _dp(np.ascontiguousarray(M1, dtype=np.float64)), float(a), int(i), int(j), int(k),
                                 _dp(m))
        return m

    @staticmethod
    def filter(m27: np.ndarray) -> np.ndarray:
        """Fine -> coarse moments from the 27 neighbours' moments, shape
        (3, 3, 3, 10) indexed [dz, dy, dx] with offsets -1, 0, +1."""
        mc = np.zeros(10)
        lib().orc_refine3_filter(_dp(np.ascontiguousarray(m27, dtype=np.float64).reshape(-1)), _dp(mc))
        return mc


class MultiLevel:
    """Nested 2:1 patches (Sec. II.B applied recursively, as the paper's
    cylinder (4 levels) and jet (5 levels) use it): level 0 is the coarse
    Problem; level k + 1 covers the level-k nodes origin..origin + extent
    (per axis of the lattice), with tau_{k+1} = 2 tau_k - 1/2.  Every level
    above 0 is a periodic box with its boundary ring / shell fixed and rebuilt
    from its parent; every level with a child has the child's covered
    interior fixed and its first ring / shell rebuilt from the child.

    One step of level k: parent-side interface moments at t + 1 (when k has
    a child), the level's own update, then two steps of the child with its
    ring refilled at t + 1/2 and t + 1 from the interface moments, and the
    covered ring of level k restricted from the child at t + 1/2 -- the order
    of orc_refined_step, applied at every level.
    """

    def __init__(self, coarse: Problem, patches):
        self.three = coarse.lattice in (D3Q19, D3Q27)
        self.P = [coarse]
        self.G = []
        for origin, extent in patches:
            parent = self.P[-1]
            d = 3 if self.three else 2
            o, e = [int(v) for v in origin[:d]], [int(v) for v in extent[:d]]
            for a in range(d):
                assert o[a] >= 2 and e[a] >= 4 and o[a] + e[a] <= parent.n[a] - 3
            nf = tuple(2 * v + 1 for v in e)
            fine = Problem(coarse.lattice, nf, 2 * parent.tau - 0.5)
            shape = tuple(reversed(nf))
            fm = np.zeros(shape, np.uint8)
            if self.three:
                fm[0], fm[-1] = FIXED, FIXED
                fm[:, 0], fm[:, -1] = FIXED, FIXED
                fm[:, :, 0], fm[:, :, -1] = FIXED, FIXED
            else:
                fm[0], fm[-1] = FIXED, FIXED
                fm[:, 0], fm[:, -1] = FIXED, FIXED
            fine.solid = fm.reshape(-1)
            pshape = tuple(reversed(parent.n[:d]))
            pm = np.zeros(pshape, np.uint8) if parent.solid is None else parent.solid.reshape(pshape).copy()
            if self.three:
                pm[o[2] + 1:o[2] + e[2], o[1] + 1:o[1] + e[1], o[0] + 1:o[0] + e[0]] = FIXED
                self.G.append(_Patch3(o[0], o[1], o[2], e[0], e[1], e[2]))
            else:
                pm[o[1] + 1:o[1] + e[1], o[0] + 1:o[0] + e[0]] = FIXED
                self.G.append(_Patch(o[0], o[1], e[0], e[1]))
            parent.solid = pm.reshape(-1)
            self.P.append(fine)

    @property
    def levels(self) -> int:
        return len(self.P)

    def set_solid(self, level: int, solid: np.ndarray):
        m = self.P[level].solid.copy()
        s = np.asarray(solid, np.uint8).reshape(-1)
        m[(s == SOLID) & (m != FIXED)] = SOLID
        self.P[level].solid = m

    def init(self, states):
        """states: one (rho, u) per level."""
        self.f = [P.equilibrium(r, u) for P, (r, u) in zip(self.P, states)]
        nm = 10 if self.three else 6
        self.M0 = [np.zeros(nm * self.P[k].ncell) for k in range(len(self.G))]
        self.M1 = [np.zeros(nm * self.P[k].ncell) for k in range(len(self.G))]
        for k, g in enumerate(self.G):
            sc = self.P[k]._struct()
            init = lib().orc_refined3_init_moments if self.three else lib().orc_refined_init_moments
            init(C.byref(sc), C.byref(g), _dp(self.f[k]), _dp(self.M0[k]))
        self.step_index = 0

    def _advance(self, k: int, step: int):
        L = lib()
        P = self.P[k]
        child = k < len(self.G)
        if child:
            g, sc = self.G[k], P._struct()
            (L.orc_refine3_plane_moments if self.three else L.orc_refine2_line_moments)(
                C.byref(sc), C.byref(g), _dp(self.f[k]), _dp(self.M1[k]))
        new = np.empty_like(self.f[k])
        s = P._struct()
        L.orc_step(C.byref(s), _dp(self.f[k]), _dp(new), int(step))
        if child:
            sf = self.P[k + 1]._struct()
            fill = L.orc_refine3_fill if self.three else L.orc_refine2_fill
            restrict = L.orc_refine3_restrict if self.three else L.orc_refine2_restrict
            self._advance(k + 1, 2 * step)
            fill(C.byref(sc), C.byref(sf), C.byref(g), _dp(self.M0[k]), _dp(self.M1[k]), 0.5, _dp(self.f[k + 1]))
            half = self.f[k + 1].copy()
            self._advance(k + 1, 2 * step + 1)
            fill(C.byref(sc), C.byref(sf), C.byref(g), _dp(self.M0[k]), _dp(self.M1[k]), 1.0, _dp(self.f[k + 1]))
            restrict(C.byref(sc), C.byref(sf), C.byref(g), _dp(half), _dp(new))
            self.M0[k][:] = self.M1[k]
        self.f[k] = new

    def run(self, nsteps: int):
        for _ in range(int(nsteps)):
            self._advance(0, self.step_index)
            self.step_index += 1
