"""Thin ctypes binding of liblbm (``include/lbm.h``).

Functions keep the C names and argument order; they only marshal numpy
arrays and raise ``LBMError`` on a negative return code.  Every step of the
computation runs in liblbm's CUDA kernels.  Importing this module loads
``_build/liblbm.so`` and fails loudly if it has not been built: there is no
fallback implementation.

``Solver`` wraps a handle with numpy-friendly helpers for tests and benchmarks.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# LBM_CHECKED=1 loads the checked build (every update index tested before use;
# built by build.build(checked=True)) instead of the release library
LIB_PATH = os.path.join(_HERE, "_build", "liblbm_checked.so" if os.environ.get("LBM_CHECKED") == "1" else "liblbm.so")

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_EIO = 0, -1, -2, -3, -4, -5
LBM_D2Q9, LBM_D3Q19, LBM_D3Q27 = 0, 1, 2
LBM_FP64, LBM_FP32, LBM_FP16_SHIFTED, LBM_BF16_SHIFTED = 0, 1, 2, 3
LBM_FACE_XM, LBM_FACE_XP, LBM_FACE_YM, LBM_FACE_YP, LBM_FACE_ZM, LBM_FACE_ZP = range(6)
LBM_BC_PERIODIC, LBM_BC_VELOCITY, LBM_BC_OUTFLOW, LBM_BC_FREESLIP, LBM_BC_PRESSURE = 0, 1, 2, 3, 4
LBM_CELL_FLUID, LBM_CELL_SOLID = 0, 1
LBM_STREAM_PULL, LBM_STREAM_AA = 0, 1

PRECISIONS = {"fp64": LBM_FP64, "fp32": LBM_FP32, "fp16": LBM_FP16_SHIFTED, "bf16": LBM_BF16_SHIFTED}

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"liblbm.so is not built ({LIB_PATH}); run `python -m paper_1710_02065_gb300.build` "
        "(the CUDA library is the only implementation)")

_lib = C.CDLL(LIB_PATH)
_h = C.c_void_p
_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_i64p = C.POINTER(C.c_int64)


def _sig(name, args, res=C.c_int):
    fn = getattr(_lib, name)
    fn.argtypes = args
    fn.restype = res
    return fn


_sig("lbm_lattice_table", [C.c_int, _ip, _ip, _ip, _dp])
_sig("lbm_create", [C.POINTER(_h), C.c_int, _ip, C.c_double, C.c_int, C.c_double, C.c_int, C.c_void_p])
_sig("lbm_destroy", [_h], None)
_sig("lbm_last_error", [_h], C.c_char_p)
_sig("lbm_set_geometry", [_h, C.POINTER(C.c_uint8)])
_sig("lbm_set_boundary", [_h, C.c_int, C.c_int, _dp, _dp])
_sig("lbm_set_inlet_noise", [_h, C.c_uint64, C.c_double])
_sig("lbm_set_pressure", [_h, C.c_int, C.c_double])
_sig("lbm_set_sponge", [_h, C.c_int, C.c_int, C.c_double, C.c_double, _dp])
_sig("lbm_set_radial_sponge", [_h, _dp, C.c_double, C.c_double, C.c_double, C.c_double, _dp])
_sig("lbm_set_state", [_h, _dp, _dp])
_sig("lbm_set_state_f32", [_h, C.POINTER(C.c_float), C.POINTER(C.c_float)])
_sig("lbm_moments_f32", [_h, C.POINTER(C.c_float), C.POINTER(C.c_float), C.POINTER(C.c_float)])
_sig("lbm_set_populations", [_h, _dp])
_sig("lbm_get_populations", [_h, _dp])
_sig("lbm_step", [_h, C.c_int64])
_sig("lbm_moments", [_h, _dp, _dp, _dp])
_sig("lbm_reduce", [_h, _dp, _dp])
_sig("lbm_probe", [_h, C.c_int, _i64p, _dp])
_sig("lbm_sync", [_h])
_sig("lbm_set_launch", [_h, C.c_int, C.c_int])
_sig("lbm_get_launch", [_h, _ip, _ip])
_sig("lbm_set_staging", [_h, C.c_int, C.c_int, C.c_int])
_sig("lbm_set_transfer_staging", [_h, C.c_size_t])
_sig("lbm_set_collision", [_h, C.c_int])
_sig("lbm_set_hermite_order", [_h, C.c_int])
_sig("lbm_pressure_mean", [_h, C.c_int])
_sig("lbm_pressure_fluctuation", [_h, _dp, _dp])
_sig("lbm_set_sponge_jet_reference", [_h] + [C.c_double] * 7)
_sig("lbm_get_staging", [_h, _ip, _ip, _ip, _ip, _ip])
_sig("lbm_set_staging_wait", [_h, C.c_uint64])
_sig("lbm_set_streaming", [_h, C.c_int])
_sig("lbm_set_storage_shift", [_h, _dp])
_sig("lbm_get_streaming", [_h, _ip])
_sig("lbm_info", [_h, _i64p, _i64p, _dp, _dp])
_sig("lbm_add_refinement_patch", [_h, _ip, _ip])
_sig("lbm_force", [_h, C.c_int, _dp])
_sig("lbm_force_async", [_h, C.c_int, C.c_void_p])
_sig("lbm_probe_async", [_h, C.c_int, C.c_void_p, C.c_void_p])
_sig("lbm_level_info", [_h, C.c_int, _ip, _dp])
_sig("lbm_set_geometry_level", [_h, C.c_int, C.POINTER(C.c_uint8)])
_sig("lbm_set_state_level", [_h, C.c_int, _dp, _dp])
_sig("lbm_set_populations_level", [_h, C.c_int, _dp])
_sig("lbm_get_populations_level", [_h, C.c_int, _dp])
_sig("lbm_moments_level", [_h, C.c_int, _dp, _dp, _dp])
class lbm_request(C.Structure):
    _fields_ = [("lattice", C.c_int), ("precision", C.c_int), ("extents", C.c_int * 3), ("tau", C.c_double),
                ("steps", C.c_int64), ("rho", _dp), ("u", _dp)]


_sig("lbm_server_create", [C.POINTER(C.c_void_p), C.c_size_t, C.c_int, C.c_void_p])
_sig("lbm_server_destroy", [C.c_void_p], None)
_sig("lbm_server_last_error", [C.c_void_p], C.c_char_p)
_sig("lbm_server_submit", [C.c_void_p, C.POINTER(lbm_request), _i64p])
_sig("lbm_server_run", [C.c_void_p, C.c_int64, _ip])
_sig("lbm_server_set_streaming", [C.c_void_p, C.c_int])
_sig("lbm_server_set_launch", [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int])
_sig("lbm_set_level_streams", [C.c_void_p, C.c_int])
_sig("lbm_server_get_launch", [C.c_void_p, C.c_int, C.c_int, _ip, _ip])
_sig("lbm_server_gpu_time", [C.c_void_p, _dp])
_sig("lbm_server_poll", [C.c_void_p, C.c_int64, _ip, _i64p])
_sig("lbm_server_result", [C.c_void_p, C.c_int64, _dp, _dp])
_sig("lbm_server_stats", [C.c_void_p, _ip, _ip, C.POINTER(C.c_size_t), _i64p])
_sig("lbm_reduce_noalloc", [C.c_int, C.c_int, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p])
_sig("lbm_save", [_h, C.c_char_p])
_sig("lbm_load", [_h, C.c_char_p])

EXPORTED = [
    "lbm_lattice_table", "lbm_create", "lbm_destroy", "lbm_last_error", "lbm_set_geometry",
    "lbm_set_boundary", "lbm_set_pressure", "lbm_set_inlet_noise", "lbm_set_sponge", "lbm_set_radial_sponge", "lbm_set_state",
    "lbm_set_populations", "lbm_get_populations", "lbm_step", "lbm_moments", "lbm_reduce",
    "lbm_probe", "lbm_sync", "lbm_info", "lbm_save", "lbm_load", "lbm_set_launch", "lbm_get_launch",
    "lbm_set_staging", "lbm_get_staging", "lbm_set_transfer_staging", "lbm_set_collision", "lbm_set_sponge_jet_reference", "lbm_set_hermite_order",
    "lbm_pressure_mean", "lbm_pressure_fluctuation",
    "lbm_add_refinement_patch", "lbm_level_info", "lbm_force", "lbm_force_async", "lbm_probe_async", "lbm_set_geometry_level", "lbm_set_state_level",
    "lbm_set_populations_level", "lbm_get_populations_level", "lbm_moments_level",
    "lbm_reduce_noalloc", "lbm_server_create", "lbm_server_destroy", "lbm_server_last_error",
    "lbm_server_submit", "lbm_server_run", "lbm_server_poll", "lbm_server_result", "lbm_server_stats",
    "lbm_server_set_streaming", "lbm_set_streaming", "lbm_get_streaming", "lbm_set_storage_shift",
    "lbm_set_staging_wait", "lbm_server_gpu_time", "lbm_set_state_f32", "lbm_moments_f32",
    "lbm_server_set_launch", "lbm_server_get_launch", "lbm_set_level_streams",
]
LBM_REQ_QUEUED, LBM_REQ_RUNNING, LBM_REQ_DONE, LBM_REQ_FAILED = 0, 1, 2, 3


class LBMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"liblbm error {code}: {msg}")
        self.code = code


def _check(rc: int, h=None):
    if rc != LBM_OK:
        msg = _lib.lbm_last_error(h)
        raise LBMError(rc, msg.decode() if msg else "")
    return rc


def _d(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous, "float64 C-contiguous array required"
    return a.ctypes.data_as(_dp)


def _c64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------
# Same-name wrappers of the C ABI
# ---------------------------------------------------------------------------
def lbm_lattice_table(lattice: int):
    q, d = C.c_int(), C.c_int()
    xi = np.zeros(27 * 3, dtype=np.int32)
    w = np.zeros(27)
    _check(_lib.lbm_lattice_table(lattice, C.byref(q), C.byref(d), xi.ctypes.data_as(_ip), _d(w)))
    return q.value, d.value, xi[: 3 * q.value].reshape(q.value, 3).copy(), w[: q.value].copy()


def lbm_create(lattice: int, extents, tau_or_nu: float, value_is_nu: bool = False,
               Ma_ref: float = 0.0, precision: int = LBM_FP32, cuda_stream: int | None = None):
    h = _h()
    ext = (C.c_int * 3)(*[int(v) for v in (list(extents) + [1] * (3 - len(extents)))])
    rc = _lib.lbm_create(C.byref(h), lattice, ext, float(tau_or_nu), int(bool(value_is_nu)),
                         float(Ma_ref), precision, C.c_void_p(cuda_stream or 0))
    _check(rc, None)
    return h


def lbm_destroy(h):
    _lib.lbm_destroy(h)


def lbm_last_error(h) -> str:
    m = _lib.lbm_last_error(h)
    return m.decode() if m else ""


def lbm_set_geometry(h, cell_type):
    if cell_type is None:
        return _check(_lib.lbm_set_geometry(h, None), h)
    a = np.ascontiguousarray(cell_type, dtype=np.uint8).reshape(-1)
    return _check(_lib.lbm_set_geometry(h, a.ctypes.data_as(C.POINTER(C.c_uint8))), h)


def lbm_set_boundary(h, face: int, kind: int, u_in=None, u_profile=None):
    u = _c64(u_in)
    p = _c64(u_profile)
    return _check(_lib.lbm_set_boundary(h, face, kind, _d(u), _d(p)), h)


def lbm_set_pressure(h, face: int, rho_out: float):
    return _check(_lib.lbm_set_pressure(h, face, float(rho_out)), h)


def lbm_set_inlet_noise(h, seed: int, amplitude: float):
    return _check(_lib.lbm_set_inlet_noise(h, C.c_uint64(int(seed)), float(amplitude)), h)


def lbm_set_sponge(h, face: int, width: int, chi_max: float, rho_ref: float = 1.0, u_ref=(0.0, 0.0, 0.0)):
    u = _c64(u_ref)
    return _check(_lib.lbm_set_sponge(h, face, int(width), float(chi_max), float(rho_ref), _d(u)), h)


def lbm_set_radial_sponge(h, center, r0: float, width: float, chi_max: float, rho_ref: float = 1.0,
                          u_ref=(0.0, 0.0, 0.0)):
    c = _c64(list(center) + [0.0] * (3 - len(center)))
    return _check(_lib.lbm_set_radial_sponge(h, _d(c), float(r0), float(width), float(chi_max), float(rho_ref),
                                             _d(_c64(u_ref))), h)


def lbm_set_state(h, rho, u):
    r = _c64(rho).reshape(-1)
    v = _c64(u).reshape(-1)
    return _check(_lib.lbm_set_state(h, _d(r), _d(v)), h)


def _f32p(a):
    """float* of a C-contiguous float32 numpy array (None -> NULL)."""
    if a is None:
        return None
    if a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"]:
        raise ValueError("expected a C-contiguous float32 array")
    return a.ctypes.data_as(C.POINTER(C.c_float))


def lbm_set_state_f32(h, rho, u):
    """lbm_set_state with FP32 host arrays (passed without a copy when they
    are C-contiguous float32 already, e.g. pinned torch buffers' numpy views)."""
    r = np.ascontiguousarray(rho, dtype=np.float32).reshape(-1)
    v = np.ascontiguousarray(u, dtype=np.float32).reshape(-1)
    return _check(_lib.lbm_set_state_f32(h, _f32p(r), _f32p(v)), h)


def lbm_moments_f32(h, rho=None, u=None, pi_neq=None):
    """lbm_moments into FP32 host arrays (C-contiguous float32 or None)."""
    return _check(_lib.lbm_moments_f32(h, _f32p(rho), _f32p(u), _f32p(pi_neq)), h)


def lbm_set_populations(h, f):
    a = _c64(f)
    return _check(_lib.lbm_set_populations(h, _d(a)), h)


def lbm_get_populations(h, out: np.ndarray):
    return _check(_lib.lbm_get_populations(h, _d(out)), h)


def lbm_step(h, n: int):
    return _check(_lib.lbm_step(h, C.c_int64(int(n))), h)


def lbm_moments(h, rho=None, u=None, pi_neq=None):
    return _check(_lib.lbm_moments(h, _d(rho), _d(u), _d(pi_neq)), h)


def lbm_reduce(h):
    m = C.c_double()
    j = np.zeros(3)
    rc = _lib.lbm_reduce(h, C.byref(m), _d(j))
    if rc not in (LBM_OK, LBM_EUNSTABLE):
        _check(rc, h)
    return m.value, j, rc


def lbm_probe(h, cells) -> np.ndarray:
    c = np.ascontiguousarray(cells, dtype=np.int64)
    out = np.zeros(len(c))
    _check(_lib.lbm_probe(h, len(c), c.ctypes.data_as(_i64p), _d(out)), h)
    return out


def lbm_set_level_streams(h, concurrent: int):
    return _check(_lib.lbm_set_level_streams(h, int(concurrent)), h)


def lbm_set_launch(h, block: int = 0, cells_per_thread: int = 0):
    return _check(_lib.lbm_set_launch(h, int(block), int(cells_per_thread)), h)


def lbm_get_launch(h):
    b, v = C.c_int(), C.c_int()
    _check(_lib.lbm_get_launch(h, C.byref(b), C.byref(v)), h)
    return b.value, v.value


LBM_COLLISION_RR, LBM_COLLISION_BGK = 0, 1


def lbm_set_sponge_jet_reference(h, yc: float, zc: float, U_jet: float, D: float, x0: float, B: float = 5.8,
                                 S: float = 0.094):
    return _check(_lib.lbm_set_sponge_jet_reference(h, float(yc), float(zc), float(U_jet), float(D), float(x0),
                                                    float(B), float(S)), h)


LBM_MEAN_RESET, LBM_MEAN_ACCUMULATE = 0, 1


def lbm_pressure_mean(h, op: int):
    return _check(_lib.lbm_pressure_mean(h, int(op)), h)


def lbm_pressure_fluctuation(h, dp_tilde=None, dp_mean=None):
    """Fill host float64 arrays (ncell) with Delta p~ and the mean Delta p."""
    for a in (dp_tilde, dp_mean):
        assert a is None or (a.dtype == np.float64 and a.flags.c_contiguous)
    return _check(_lib.lbm_pressure_fluctuation(h, _d(dp_tilde), _d(dp_mean)), h)


def lbm_set_hermite_order(h, order: int):
    return _check(_lib.lbm_set_hermite_order(h, int(order)), h)


def lbm_set_collision(h, model: int):
    return _check(_lib.lbm_set_collision(h, int(model)), h)


def lbm_set_staging(h, mode: int = -1, stages: int = 0, block: int = 0):
    return _check(_lib.lbm_set_staging(h, int(mode), int(stages), int(block)), h)


def lbm_set_storage_shift(h, u_s=None):
    """Store f_i - feqH_i(1, u_s) instead of f_i - w_i (None: the default)."""
    if u_s is None:
        return _check(_lib.lbm_set_storage_shift(h, None), h)
    a = np.ascontiguousarray(u_s, dtype=np.float64)
    return _check(_lib.lbm_set_storage_shift(h, a.ctypes.data_as(_dp)), h)


def lbm_set_streaming(h, pattern: int):
    """LBM_STREAM_PULL (two lattices) or LBM_STREAM_AA (one lattice in place)."""
    return _check(_lib.lbm_set_streaming(h, int(pattern)), h)


def lbm_get_streaming(h) -> int:
    v = C.c_int()
    _check(_lib.lbm_get_streaming(h, C.byref(v)), h)
    return v.value


def lbm_set_staging_wait(h, limit_ns: int):
    """Limit (ns) of each wait of the row-staged kernel for a tile's copies."""
    return _check(_lib.lbm_set_staging_wait(h, int(limit_ns)), h)


def lbm_set_transfer_staging(h, max_bytes: int):
    """Bound (bytes) on the device staging buffer of host transfers."""
    return _check(_lib.lbm_set_transfer_staging(h, int(max_bytes)), h)


def lbm_get_staging(h):
    """(active, stages, block, rows_per_tile, grid) of the row-staged kernel."""
    v = [C.c_int() for _ in range(5)]
    _check(_lib.lbm_get_staging(h, *[C.byref(x) for x in v]), h)
    return tuple(x.value for x in v)


def lbm_sync(h):
    return _check(_lib.lbm_sync(h), h)


def lbm_info(h):
    s, l = C.c_int64(), C.c_int64()
    b, t = C.c_double(), C.c_double()
    _check(_lib.lbm_info(h, C.byref(s), C.byref(l), C.byref(b), C.byref(t)), h)
    return {"step": s.value, "launches": l.value, "bytes_per_cell": b.value, "tau": t.value}


def lbm_save(h, path: str):
    return _check(_lib.lbm_save(h, path.encode()), h)


def lbm_load(h, path: str):
    return _check(_lib.lbm_load(h, path.encode()), h)


def lbm_add_refinement_patch(h, origin, extent):
    o = (C.c_int * 3)(*[int(v) for v in (list(origin) + [0] * (3 - len(origin)))])
    e = (C.c_int * 3)(*[int(v) for v in (list(extent) + [1] * (3 - len(extent)))])
    return _check(_lib.lbm_add_refinement_patch(h, o, e), h)


def lbm_force(h, level: int = 0) -> np.ndarray:
    F = np.zeros(3)
    _check(_lib.lbm_force(h, level, _d(F)), h)
    return F


def lbm_force_async(h, level: int, F_dev: int):
    """Force of a level into 3 doubles of device memory (address F_dev), no sync."""
    return _check(_lib.lbm_force_async(h, level, C.c_void_p(F_dev)), h)


def lbm_probe_async(h, n: int, cells_dev: int, p_dev: int):
    """p' at n cells (device int64 list at cells_dev) into device doubles at p_dev, no sync."""
    return _check(_lib.lbm_probe_async(h, int(n), C.c_void_p(cells_dev), C.c_void_p(p_dev)), h)


def lbm_level_info(h, level: int):
    e = (C.c_int * 3)()
    t = C.c_double()
    _check(_lib.lbm_level_info(h, level, e, C.byref(t)), h)
    return tuple(e), t.value


def lbm_set_geometry_level(h, level: int, cell_type):
    if cell_type is None:
        return _check(_lib.lbm_set_geometry_level(h, level, None), h)
    a = np.ascontiguousarray(cell_type, dtype=np.uint8).reshape(-1)
    return _check(_lib.lbm_set_geometry_level(h, level, a.ctypes.data_as(C.POINTER(C.c_uint8))), h)


def lbm_set_state_level(h, level: int, rho, u):
    r = _c64(rho).reshape(-1)
    v = _c64(u).reshape(-1)
    return _check(_lib.lbm_set_state_level(h, level, _d(r), _d(v)), h)


def lbm_set_populations_level(h, level: int, f):
    a = _c64(f)
    return _check(_lib.lbm_set_populations_level(h, level, _d(a)), h)


def lbm_get_populations_level(h, level: int, out: np.ndarray):
    return _check(_lib.lbm_get_populations_level(h, level, _d(out)), h)


def lbm_moments_level(h, level: int, rho=None, u=None, pi_neq=None):
    return _check(_lib.lbm_moments_level(h, level, _d(rho), _d(u), _d(pi_neq)), h)


def lbm_reduce_noalloc(lattice: int, precision: int, f_dev: int, ncell: int, cell_type_dev: int | None,
                       out_dev: int, cuda_stream: int | None = None):
    """Device pointers in, device pointer out (6 doubles); no allocation."""
    return _check(_lib.lbm_reduce_noalloc(lattice, precision, C.c_void_p(f_dev), C.c_int64(int(ncell)),
                                          C.c_void_p(cell_type_dev or 0), C.c_void_p(out_dev),
                                          C.c_void_p(cuda_stream or 0)), None)


def _scheck(rc: int, s):
    if rc != LBM_OK:
        msg = _lib.lbm_server_last_error(s)
        raise LBMError(rc, msg.decode() if msg else "")
    return rc


def lbm_server_create(hbm_budget_bytes: int, max_slots: int, cuda_stream: int | None = None):
    s = C.c_void_p()
    rc = _lib.lbm_server_create(C.byref(s), C.c_size_t(int(hbm_budget_bytes)), int(max_slots),
                                C.c_void_p(cuda_stream or 0))
    _check(rc, None)
    return s


def lbm_server_destroy(s):
    _lib.lbm_server_destroy(s)


def lbm_server_last_error(s) -> str:
    m = _lib.lbm_server_last_error(s)
    return m.decode() if m else ""


def lbm_server_submit(s, lattice: int, precision: int, extents, tau: float, steps: int, rho=None, u=None) -> int:
    ext = list(extents) + [1] * (3 - len(extents))
    r = _c64(rho)
    v = _c64(u)
    req = lbm_request(lattice, precision, (C.c_int * 3)(*[int(e) for e in ext]), float(tau), int(steps),
                      _d(r.reshape(-1)) if r is not None else None, _d(v.reshape(-1)) if v is not None else None)
    rid = C.c_int64()
    _scheck(_lib.lbm_server_submit(s, C.byref(req), C.byref(rid)), s)
    return rid.value


def lbm_server_set_streaming(s, pattern: int):
    """Streaming pattern of the requests admitted from now on."""
    return _scheck(_lib.lbm_server_set_streaming(s, int(pattern)), s)


def lbm_server_set_launch(s, lattice: int, precision: int, cells_per_lane: int, warps_per_block: int):
    """Launch shape of a (lattice, precision) group's batched update (0, 0: defaults)."""
    return _scheck(_lib.lbm_server_set_launch(s, int(lattice), int(precision), int(cells_per_lane),
                                              int(warps_per_block)), s)


def lbm_server_get_launch(s, lattice: int, precision: int):
    """(cells_per_lane, warps_per_block) of a group."""
    v, w = C.c_int(0), C.c_int(0)
    _scheck(_lib.lbm_server_get_launch(s, int(lattice), int(precision), C.byref(v), C.byref(w)), s)
    return v.value, w.value


def lbm_server_gpu_time(s) -> float:
    """Device time (ms) of all rounds so far."""
    v = C.c_double()
    _scheck(_lib.lbm_server_gpu_time(s, C.byref(v)), s)
    return v.value


def lbm_server_run(s, steps: int) -> int:
    done = C.c_int()
    _scheck(_lib.lbm_server_run(s, C.c_int64(int(steps)), C.byref(done)), s)
    return done.value


def lbm_server_poll(s, rid: int):
    st, d = C.c_int(), C.c_int64()
    _scheck(_lib.lbm_server_poll(s, C.c_int64(rid), C.byref(st), C.byref(d)), s)
    return st.value, d.value


def lbm_server_result(s, rid: int, rho=None, u=None):
    rc = _lib.lbm_server_result(s, C.c_int64(rid), _d(rho), _d(u))
    if rc not in (LBM_OK, LBM_EUNSTABLE):
        _scheck(rc, s)
    return rc


def lbm_server_stats(s):
    q, r = C.c_int(), C.c_int()
    b = C.c_size_t()
    cu = C.c_int64()
    _scheck(_lib.lbm_server_stats(s, C.byref(q), C.byref(r), C.byref(b), C.byref(cu)), s)
    return {"queued": q.value, "running": r.value, "bytes_in_use": b.value, "cell_updates": cu.value}


# ---------------------------------------------------------------------------
# Convenience wrapper
# ---------------------------------------------------------------------------
class Solver:
    """Owns one liblbm handle; numpy in, numpy out."""

    def __init__(self, lattice: int, extents, tau: float, precision: int = LBM_FP32,
                 Ma_ref: float = 0.0, stream: int | None = None, value_is_nu: bool = False):
        self.lattice = lattice
        ext = list(extents) + [1] * (3 - len(extents))
        self.n = tuple(int(v) for v in ext)
        self.ncell = self.n[0] * self.n[1] * self.n[2]
        self.q = {LBM_D2Q9: 9, LBM_D3Q19: 19, LBM_D3Q27: 27}[lattice]
        self.h = lbm_create(lattice, self.n, tau, value_is_nu, Ma_ref, precision, stream)

    def close(self):
        if self.h:
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_state(self, rho, u):
        lbm_set_state(self.h, rho, u)

    def set_populations(self, f):
        lbm_set_populations(self.h, np.asarray(f, dtype=np.float64).reshape(self.q, self.ncell))

    def populations(self) -> np.ndarray:
        out = np.zeros((self.q, self.ncell))
        lbm_get_populations(self.h, out)
        return out

    def step(self, n: int = 1):
        lbm_step(self.h, n)

    def sync(self):
        lbm_sync(self.h)

    def moments(self):
        rho = np.zeros(self.ncell)
        u = np.zeros((self.ncell, 3))
        pn = np.zeros((self.ncell, 6))
        lbm_moments(self.h, rho, u, pn)
        return rho, u, pn

    def reduce(self):
        return lbm_reduce(self.h)

    def info(self):
        return lbm_info(self.h)
