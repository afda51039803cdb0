"""ctypes binding of ``include/rtlbfs.h`` (argument marshalling only).

Every step of the solver runs in the CUDA library ``_build/librtlbfs.so``;
this module only converts numpy arrays to pointers and status codes to
exceptions.  There is no CPU fallback: if the library cannot be built or
loaded, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

from . import build as _build

OK = 0
ERR_ARG, ERR_OOM, ERR_CUDA, ERR_DIVERGED, ERR_NOT_CONVERGED, ERR_TIMEOUT, ERR_STATE = (
    -1, -2, -3, -4, -5, -6, -7)
FP64, FP32 = 0, 1
RTLBFS, TLBFS = 0, 1  # face stages (set_scheme)
WEST, EAST, SOUTH, NORTH = 0, 1, 2, 3
WALL_DIRICHLET, WALL_ADIABATIC, PERIODIC, HALO = 0, 1, 2, 3
NU_WEST, NU_EAST, NU_SOUTH, NU_NORTH, NU_AVG, NU_HALF = 0, 1, 2, 3, 4, 5

HEADER = os.path.join(_build.ROOT, "include", "rtlbfs.h")
HEADERS = [HEADER, os.path.join(_build.ROOT, "include", "rtlbfs_batch.h"),
           os.path.join(_build.ROOT, "include", "rtlbfs3d.h"),
           os.path.join(_build.ROOT, "include", "rtlbfs_curv.h"),
           os.path.join(_build.ROOT, "include", "rtlbfs_measure.h")]
RATE_FP32, RATE_FP32X2, RATE_FP64 = 0, 1, 2  # kinds of fma_rate
SLOT_EMPTY, SLOT_RUNNING, SLOT_CONVERGED, SLOT_MAX_STEPS, SLOT_DIVERGED = -1, 0, 1, 2, 3


class Request(C.Structure):
    _fields_ = [("t_arrive", C.c_double), ("n", C.c_int), ("Ra", C.c_double), ("Pr", C.c_double)]


class Result(C.Structure):
    _fields_ = [("t_admit", C.c_double), ("t_finish", C.c_double), ("steps", C.c_long),
                ("status", C.c_int), ("nu_hot", C.c_double), ("nu_cold", C.c_double)]


class ServeOpts(C.Structure):
    _fields_ = [("max_slots", C.c_int), ("mem_fraction", C.c_double), ("tol", C.c_double),
                ("max_steps", C.c_long), ("Ma", C.c_double), ("time_limit_s", C.c_double),
                ("chunk_steps", C.c_int), ("precision", C.c_int)]

_lib = None

_dp = C.POINTER(C.c_double)
_vp = C.c_void_p

# name -> (restype, argtypes)
_SIGS = {
    "rtlbfs_tanh_faces": (C.c_int, [C.c_int, C.c_double, C.c_double, _dp]),
    "rtlbfs_create_mesh": (C.c_int, [C.c_int, C.c_int, _dp, _dp, C.c_int, C.POINTER(_vp)]),
    "rtlbfs_set_params": (C.c_int, [_vp, C.c_double, C.c_double, C.c_double, C.c_double]),
    "rtlbfs_create_strip": (C.c_int, [C.c_int, C.c_int, _dp, _dp, C.c_int, C.c_int, C.c_int,
                                      C.POINTER(_vp)]),
    "rtlbfs_strip_get_rows": (C.c_int, [_vp, C.c_int, _dp]),
    "rtlbfs_strip_set_halo": (C.c_int, [_vp, C.c_int, _dp]),
    "rtlbfs_strip_rows": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, C.POINTER(_vp),
                                    C.POINTER(C.c_size_t)]),
    "rtlbfs_current_buffer": (C.c_int, [_vp, C.POINTER(C.c_int)]),
    "rtlbfs_state_raw_bytes": (C.c_size_t, [_vp]),
    "rtlbfs_get_state_raw": (C.c_int, [_vp, _vp, _dp]),
    "rtlbfs_set_state_raw": (C.c_int, [_vp, _vp, C.c_double]),
    "rtlbfs_strip_pack": (C.c_int, [_vp, C.c_int, C.c_int, _vp]),
    "rtlbfs_strip_unpack": (C.c_int, [_vp, C.c_int, C.c_int, _vp]),
    "rtlbfs_residual_sums": (C.c_int, [_vp, _dp, C.POINTER(C.c_long)]),
    "rtlbfs_set_params_ref": (C.c_int, [_vp] + [C.c_double] * 7),
    "rtlbfs_set_lattice": (C.c_int, [_vp, C.c_double]),
    "rtlbfs_set_bc": (C.c_int, [_vp, C.c_int, C.c_int, C.c_double, C.c_double]),
    "rtlbfs_set_body_force": (C.c_int, [_vp, C.c_double, C.c_double]),
    "rtlbfs_set_physics": (C.c_int, [_vp, C.c_double, C.c_double, C.c_double]),
    "rtlbfs_set_state": (C.c_int, [_vp, _dp, _dp, _dp, _dp]),
    "rtlbfs_get_state": (C.c_int, [_vp, _dp, _dp, _dp, _dp]),
    "rtlbfs_step": (C.c_int, [_vp, C.c_long]),
    "rtlbfs_run_to_steady": (C.c_int, [_vp, C.c_double, C.c_long, C.c_double,
                                       C.POINTER(C.c_long), _dp]),
    "rtlbfs_residual": (C.c_int, [_vp, _dp, C.POINTER(C.c_long)]),
    "rtlbfs_nusselt": (C.c_int, [_vp, C.c_int, _dp]),
    "rtlbfs_set_stream": (C.c_int, [_vp, _vp]),
    "rtlbfs_set_schedule": (C.c_int, [_vp, C.c_int, C.c_int]),
    "rtlbfs_debug_withhold_tile": (C.c_int, [_vp, C.c_int]),
    "rtlbfs_autotune": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                  C.POINTER(C.c_double)]),
    "rtlbfs_sync": (C.c_int, [_vp]),
    "rtlbfs_last_error": (C.c_char_p, [_vp]),
    "rtlbfs_destroy": (None, [_vp]),
    "rtlbfs_launch_count": (C.c_longlong, []),
    "rtlbfs_fma_rate": (C.c_int, [C.c_int, C.c_int, _dp, _dp]),
    "rtlbfs_op_counts": (C.c_int, [_dp, _dp, _dp]),
    "rtlbfs_op_counts_scheme": (C.c_int, [C.c_int, _dp, _dp, _dp]),
    "rtlbfs_set_scheme": (C.c_int, [_vp, C.c_int]),
    "rtlbfs_batch_create": (C.c_int, [C.c_int, C.c_int, C.POINTER(_vp)]),
    "rtlbfs_batch_bytes": (C.c_size_t, [C.c_int, C.c_int, C.c_int]),
    "rtlbfs_batch_free_bytes": (C.c_int, [C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]),
    "rtlbfs_batch_add": (C.c_int, [_vp, C.c_int, C.c_int, _dp, _dp, C.c_double, C.c_double,
                                   C.c_double, C.c_double, C.POINTER(C.c_int)]),
    "rtlbfs_batch_set_bc": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double]),
    "rtlbfs_batch_set_lattice": (C.c_int, [_vp, C.c_int, C.c_double]),
    "rtlbfs_batch_set_state": (C.c_int, [_vp, C.c_int, _dp, _dp, _dp, _dp]),
    "rtlbfs_batch_get_state": (C.c_int, [_vp, C.c_int, _dp, _dp, _dp, _dp]),
    "rtlbfs_batch_state_raw_bytes": (C.c_size_t, [_vp, C.c_int]),
    "rtlbfs_batch_get_state_raw": (C.c_int, [_vp, C.c_int, _vp, _dp]),
    "rtlbfs_batch_set_state_raw": (C.c_int, [_vp, C.c_int, _vp, C.c_double]),
    "rtlbfs_batch_get_states_raw": (C.c_int, [_vp, C.c_int, _vp, _vp, _dp]),
    "rtlbfs_batch_arm_many": (C.c_int, [_vp, C.c_int, _vp, C.c_double, C.c_long]),
    "rtlbfs_batch_set_schedule": (C.c_int, [_vp, C.c_int, C.c_int]),
    "rtlbfs_batch_set_states_raw": (C.c_int, [_vp, C.c_int, _vp, _vp, _dp]),
    "rtlbfs_batch_arm": (C.c_int, [_vp, C.c_int, C.c_double, C.c_long]),
    "rtlbfs_batch_step": (C.c_int, [_vp, C.c_long]),
    "rtlbfs_batch_poll": (C.c_int, [_vp, C.POINTER(C.c_int), C.POINTER(C.c_long), _dp]),
    "rtlbfs_batch_nusselt": (C.c_int, [_vp, C.c_int, C.c_int, _dp]),
    "rtlbfs_batch_remove": (C.c_int, [_vp, C.c_int]),
    "rtlbfs_batch_autotune": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                        C.POINTER(C.c_double)]),
    "rtlbfs_batch_set_stream": (C.c_int, [_vp, _vp]),
    "rtlbfs_batch_info": (C.c_int, [_vp, C.POINTER(C.c_longlong), C.POINTER(C.c_int),
                                    C.POINTER(C.c_int)]),
    "rtlbfs_batch_last_error": (C.c_char_p, [_vp]),
    "rtlbfs_batch_destroy": (None, [_vp]),
    "rtlbfs_serve": (C.c_int, [C.POINTER(Request), C.c_int, C.POINTER(ServeOpts),
                               C.POINTER(Result), C.POINTER(C.c_double)]),
    "rtlbfs_stability_map": (C.c_int, [C.c_int, C.POINTER(C.c_int), _dp, _dp, _dp, C.c_double,
                                       C.c_double, C.c_double, C.c_long, C.c_int, C.c_int,
                                       C.POINTER(C.c_int), C.POINTER(C.c_long), _dp]),
    "rtlbfs_nusselt_noalloc": (C.c_int, [C.c_int, C.c_int, _dp, _dp, _vp, _vp, _vp, _vp,
                                         C.c_double, C.c_double, C.c_double, C.c_double,
                                         C.POINTER(C.c_int), _dp, _dp, C.c_int, _vp, _vp]),
    # 3D (include/rtlbfs3d.h)
    "rtlbfs3d_create": (C.c_int, [C.c_int, C.c_int, C.c_int, _dp, _dp, _dp, C.c_int,
                                  C.POINTER(_vp)]),
    "rtlbfs3d_set_params": (C.c_int, [_vp, C.c_double, C.c_double, C.c_double, C.c_double]),
    "rtlbfs3d_set_physics": (C.c_int, [_vp, C.c_double, C.c_double, C.c_double]),
    "rtlbfs3d_set_lattice": (C.c_int, [_vp, C.c_double]),
    "rtlbfs3d_set_gravity_axis": (C.c_int, [_vp, C.c_int]),
    "rtlbfs3d_set_body_force": (C.c_int, [_vp, C.c_double, C.c_double, C.c_double]),
    "rtlbfs3d_set_bc": (C.c_int, [_vp, C.c_int, C.c_int, C.c_double, _dp]),
    "rtlbfs3d_set_state": (C.c_int, [_vp, _dp, _dp, _dp, _dp, _dp]),
    "rtlbfs3d_get_state": (C.c_int, [_vp, _dp, _dp, _dp, _dp, _dp]),
    "rtlbfs3d_step": (C.c_int, [_vp, C.c_long]),
    "rtlbfs3d_run_to_steady": (C.c_int, [_vp, C.c_double, C.c_long, C.c_double,
                                         C.POINTER(C.c_long), _dp]),
    "rtlbfs3d_residual": (C.c_int, [_vp, _dp, C.POINTER(C.c_long)]),
    "rtlbfs3d_nusselt": (C.c_int, [_vp, C.c_int, C.c_int, _dp]),
    "rtlbfs3d_set_schedule": (C.c_int, [_vp, C.c_int, C.c_int]),
    "rtlbfs3d_autotune": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_int), _dp]),
    "rtlbfs3d_set_stream": (C.c_int, [_vp, _vp]),
    "rtlbfs3d_sync": (C.c_int, [_vp]),
    "rtlbfs3d_last_error": (C.c_char_p, [_vp]),
    "rtlbfs3d_op_counts": (C.c_int, [_dp, _dp, _dp]),
    "rtlbfs3d_op_counts_scheme": (C.c_int, [C.c_int, _dp, _dp, _dp]),
    "rtlbfs3d_set_scheme": (C.c_int, [_vp, C.c_int]),
    "rtlbfs3d_destroy": (None, [_vp]),
    # curvilinear 2D (include/rtlbfs_curv.h)
    "rtlbfsc_create": (C.c_int, [C.c_int, C.c_int, _dp, _dp, C.c_int, C.c_int, C.POINTER(_vp)]),
    "rtlbfsc_set_physics": (C.c_int, [_vp, C.c_double, C.c_double, C.c_double, C.c_double]),
    "rtlbfsc_set_lattice": (C.c_int, [_vp, C.c_double]),
    "rtlbfsc_set_gravity": (C.c_int, [_vp, C.c_double, C.c_double, C.c_double]),
    "rtlbfsc_set_body_force": (C.c_int, [_vp, C.c_double, C.c_double]),
    "rtlbfsc_set_bc": (C.c_int, [_vp, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double]),
    "rtlbfsc_set_farfield": (C.c_int, [_vp, C.c_double, C.c_double, C.c_double, C.c_double]),
    "rtlbfsc_set_state": (C.c_int, [_vp, _dp, _dp, _dp, _dp]),
    "rtlbfsc_get_state": (C.c_int, [_vp, _dp, _dp, _dp, _dp]),
    "rtlbfsc_step": (C.c_int, [_vp, C.c_long]),
    "rtlbfsc_run_to_steady": (C.c_int, [_vp, C.c_double, C.c_long, C.c_double,
                                        C.POINTER(C.c_long), _dp]),
    "rtlbfsc_residual": (C.c_int, [_vp, _dp, C.POINTER(C.c_long)]),
    "rtlbfsc_wall_heat": (C.c_int, [_vp, C.c_int, _dp, _dp]),
    "rtlbfsc_set_schedule": (C.c_int, [_vp, C.c_int]),
    "rtlbfsc_set_stream": (C.c_int, [_vp, _vp]),
    "rtlbfsc_sync": (C.c_int, [_vp]),
    "rtlbfsc_last_error": (C.c_char_p, [_vp]),
    "rtlbfsc_op_counts": (C.c_int, [_dp, _dp, _dp]),
    "rtlbfsc_destroy": (None, [_vp]),
}


class RTLBFSError(RuntimeError):
    def __init__(self, rc: int, msg: str):
        super().__init__(f"rtlbfs error {rc}: {msg}")
        self.rc = rc


def lib_path() -> str:
    return _build.LIB


def lib(build_if_needed: bool = True):
    """Load the CUDA library (building it first if stale and nvcc exists)."""
    global _lib
    if _lib is None:
        if build_if_needed and _build.stale():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise ImportError("librtlbfs.so is not built; run paper_2202_13449_gb300.build")
        L = C.CDLL(_build.LIB)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def header_functions(paths=None):
    """Names of the functions declared in the public headers."""
    names = set()
    for path in (paths or HEADERS):
        text = open(path).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(rtlbfs(?:3d|c)?_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _f64(a, n: int) -> np.ndarray:
    out = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    if out.size != n:
        raise ValueError(f"expected {n} values, got {out.size}")
    return out


def _raw_out(out, nbytes: int) -> np.ndarray:
    """`out` as an array the library may write nbytes into: C-contiguous,
    writable and large enough (the library writes through a bare pointer)."""
    a = np.asarray(out)
    if not (a.flags.c_contiguous and a.flags.writeable):
        raise ValueError("the output buffer must be C-contiguous and writable")
    if a.nbytes < nbytes:
        raise ValueError(f"the output buffer holds {a.nbytes} bytes, {nbytes} are needed")
    return a


def tanh_faces(n: int, L: float, phi: float) -> np.ndarray:
    """Eq. 74 face coordinates from the library (host-only entry point)."""
    out = np.empty(n + 1)
    rc = lib().rtlbfs_tanh_faces(int(n), float(L), float(phi), _ptr(out))
    if rc:
        raise RTLBFSError(rc, "rtlbfs_tanh_faces")
    return out


def nusselt_noalloc(xf, yf, rho_ptr, u_ptr, v_ptr, T_ptr, nu, chi, kappa, dT, bc_kind, bc_T,
                    bc_u, which, out_ptr, stream=None):
    """Allocation-free Nusselt number of caller-owned FP64 device fields
    (pointers as ints); the result is written to the device double at
    out_ptr asynchronously on `stream`.  Returns the status code."""
    xf = np.ascontiguousarray(xf, dtype=np.float64)
    yf = np.ascontiguousarray(yf, dtype=np.float64)
    kinds = (C.c_int * 4)(*[int(k) for k in bc_kind])
    bT = np.ascontiguousarray(bc_T, dtype=np.float64)
    bU = np.ascontiguousarray(bc_u, dtype=np.float64)
    st = None if stream is None else int(getattr(stream, "cuda_stream", stream))
    return int(lib().rtlbfs_nusselt_noalloc(len(xf) - 1, len(yf) - 1, _ptr(xf), _ptr(yf), rho_ptr,
                                            u_ptr, v_ptr, T_ptr, nu, chi, kappa, dT, kinds,
                                            _ptr(bT), _ptr(bU), int(which), out_ptr, st))


def launch_count() -> int:
    return int(lib().rtlbfs_launch_count())


def fma_rate(kind: int, reps: int):
    """(FMAs per second, ms) of the current device for RATE_FP32 (FFMA),
    RATE_FP32X2 (FFMA2, two FMAs each) or RATE_FP64, from one timed launch
    of independent FMA chains on every SM (include/rtlbfs_measure.h)."""
    r, ms = C.c_double(), C.c_double()
    rc = lib().rtlbfs_fma_rate(int(kind), int(reps), C.byref(r), C.byref(ms))
    if rc:
        raise RTLBFSError(rc, "rtlbfs_fma_rate")
    return r.value, ms.value


def op_counts(scheme: int = 0):
    """(FP ops per face, FP ops per cell-update, SFU ops per cell-update) of
    the step with face stage `scheme` (RTLBFS or TLBFS), each face and
    gradient evaluated once (host-only)."""
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    rc = lib().rtlbfs_op_counts_scheme(int(scheme), C.byref(a), C.byref(b), C.byref(c))
    if rc:
        raise RTLBFSError(rc, "rtlbfs_op_counts")
    return a.value, b.value, c.value


class Solver:
    """One cavity on the GPU (a handle of ``include/rtlbfs.h``).  With
    ``rows=(j0, j1)`` the handle is the row strip j0 <= j < j1 of the mesh
    (rtlbfs_create_strip): its fields are (j1 - j0) x nx."""

    def __init__(self, xf, yf, precision: int = FP64, rows=None):
        L = lib()
        self.xf = np.ascontiguousarray(xf, dtype=np.float64)
        self.yf = np.ascontiguousarray(yf, dtype=np.float64)
        self.nx, self.ny = len(self.xf) - 1, len(self.yf) - 1
        self.precision = precision
        self.rows = None
        h = _vp()
        if rows is None:
            rc = L.rtlbfs_create_mesh(self.nx, self.ny, _ptr(self.xf), _ptr(self.yf),
                                      int(precision), C.byref(h))
        else:
            j0, j1 = int(rows[0]), int(rows[1])
            rc = L.rtlbfs_create_strip(self.nx, self.ny, _ptr(self.xf), _ptr(self.yf), j0, j1,
                                       int(precision), C.byref(h))
            self.rows = (j0, j1)
            self.ny = j1 - j0
        if rc:
            raise RTLBFSError(rc, "rtlbfs_create_mesh" if rows is None else "rtlbfs_create_strip")
        self._h = h

    # -- row strips (rtlbfs_create_strip)
    def strip_get_rows(self, side: int) -> np.ndarray:
        """The strip's two rows next to `side` as an array (4, 2, nx)."""
        out = np.empty(8 * self.nx)
        self._check(lib().rtlbfs_strip_get_rows(self._h, int(side), _ptr(out)), "strip_get_rows")
        return out.reshape(4, 2, self.nx)

    def strip_set_halo(self, side: int, rows):
        """Set the two halo rows beyond `side` from an array (4, 2, nx)."""
        a = _f64(rows, 8 * self.nx)
        self._check(lib().rtlbfs_strip_set_halo(self._h, int(side), _ptr(a)), "strip_set_halo")

    def strip_rows(self, side: int, halo: bool, buffer: int):
        """(device address, bytes) of the two own (halo=False) or halo rows
        next to `side` in state buffer `buffer`."""
        p, n = _vp(), C.c_size_t()
        self._check(lib().rtlbfs_strip_rows(self._h, int(side), int(bool(halo)), int(buffer),
                                            C.byref(p), C.byref(n)), "strip_rows")
        return int(p.value or 0), int(n.value)

    def strip_pack(self, side: int, buffer: int, dev_ptr: int):
        """Queue a copy of the own rows next to `side` (buffer `buffer`) to
        the device address dev_ptr (strip_rows' bytes)."""
        self._check(lib().rtlbfs_strip_pack(self._h, int(side), int(buffer), _vp(dev_ptr)),
                    "strip_pack")

    def strip_unpack(self, side: int, buffer: int, dev_ptr: int):
        """Queue a copy from device address dev_ptr into the halo rows
        beyond `side` (buffer `buffer`)."""
        self._check(lib().rtlbfs_strip_unpack(self._h, int(side), int(buffer), _vp(dev_ptr)),
                    "strip_unpack")

    def current_buffer(self) -> int:
        b = C.c_int()
        self._check(lib().rtlbfs_current_buffer(self._h, C.byref(b)), "current_buffer")
        return int(b.value)

    def residual_sums(self):
        """(sums of the last step (4,), step count): see rtlbfs_residual_sums."""
        out = np.empty(4)
        steps = C.c_long()
        self._check(lib().rtlbfs_residual_sums(self._h, _ptr(out), C.byref(steps)),
                    "residual_sums")
        return out, int(steps.value)

    # -- helpers
    def _check(self, rc: int, what: str):
        if rc:
            msg = lib().rtlbfs_last_error(self._h)
            raise RTLBFSError(rc, f"{what}: {msg.decode() if msg else ''}")

    def close(self):
        if getattr(self, "_h", None):
            lib().rtlbfs_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- configuration
    def set_params(self, Ra, Pr, Ma, dt):
        self._check(lib().rtlbfs_set_params(self._h, Ra, Pr, Ma, dt), "set_params")

    def set_params_ref(self, Ra, Pr, Ma, dt, L, dT=1.0, T_ref=0.5):
        self._check(lib().rtlbfs_set_params_ref(self._h, Ra, Pr, Ma, dt, L, dT, T_ref),
                    "set_params_ref")

    def set_lattice(self, kappa):
        self._check(lib().rtlbfs_set_lattice(self._h, kappa), "set_lattice")

    def set_bc(self, side, kind, T_wall=0.0, u_wall=0.0):
        self._check(lib().rtlbfs_set_bc(self._h, side, kind, T_wall, u_wall), "set_bc")

    def set_body_force(self, fx, fy):
        self._check(lib().rtlbfs_set_body_force(self._h, fx, fy), "set_body_force")

    def set_physics(self, nu, chi, beta_g):
        self._check(lib().rtlbfs_set_physics(self._h, nu, chi, beta_g), "set_physics")

    def set_scheme(self, scheme: int):
        """Face stage: RTLBFS (0, Section 3.2) or TLBFS (1, Section 2.2)."""
        self._check(lib().rtlbfs_set_scheme(self._h, int(scheme)), "set_scheme")

    def set_schedule(self, kernel: int = 0, chunk_rows: int = 0):
        """kernel 0: warp-marching strips (chunk_rows rows per unit), 1:
        shared-memory tiles (chunk_rows = tile height: 16, 14, 12, 10, 8, 4 or
        2 in FP32; 16, 8, 4 or 2 in FP64), 2: the same tiles in a persistent
        launch (one cavity whose tiles all fit at once); chunk_rows 0 picks
        automatically."""
        self._check(lib().rtlbfs_set_schedule(self._h, int(kernel), int(chunk_rows)),
                    "set_schedule")

    def debug_withhold_tile(self, tile: int):
        """Tests only: the persistent kernel's tile that never reports progress."""
        self._check(lib().rtlbfs_debug_withhold_tile(self._h, int(tile)), "debug_withhold_tile")

    def autotune(self, steps: int = 64):
        """Pick the fastest schedule on a snapshot of the state (restored);
        returns (kernel, chunk_rows, ms_per_step)."""
        k, r, ms = C.c_int(0), C.c_int(0), C.c_double(0)
        self._check(lib().rtlbfs_autotune(self._h, int(steps), C.byref(k), C.byref(r), C.byref(ms)),
                    "autotune")
        return int(k.value), int(r.value), float(ms.value)

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, an int handle, or None."""
        ptr = None if stream is None else int(getattr(stream, "cuda_stream", stream))
        self._check(lib().rtlbfs_set_stream(self._h, ptr), "set_stream")

    # -- state
    def set_state(self, rho, u, v, T):
        n = self.nx * self.ny
        arrs = [_f64(a, n) for a in (rho, u, v, T)]
        self._check(lib().rtlbfs_set_state(self._h, *[_ptr(a) for a in arrs]), "set_state")

    def get_state(self):
        out = [np.empty((self.ny, self.nx)) for _ in range(4)]
        self._check(lib().rtlbfs_get_state(self._h, *[_ptr(a) for a in out]), "get_state")
        return tuple(out)

    def raw_bytes(self) -> int:
        return int(lib().rtlbfs_state_raw_bytes(self._h))

    def get_state_raw(self, out=None):
        """(records, T_unit): the state's cell records as a uint8 array (or
        into `out`, any writable buffer of raw_bytes() bytes, e.g. a pinned
        torch tensor's numpy view) and the temperature unit."""
        nb = self.raw_bytes()
        out = np.empty(nb, dtype=np.uint8) if out is None else _raw_out(out, nb)
        tu = C.c_double()
        self._check(lib().rtlbfs_get_state_raw(self._h, _vp(out.ctypes.data), C.byref(tu)),
                    "get_state_raw")
        return out, tu.value

    def set_state_raw(self, records, T_unit: float = 1.0):
        a = np.ascontiguousarray(records).view(np.uint8).reshape(-1)
        if a.size != self.raw_bytes():
            raise ValueError(f"expected {self.raw_bytes()} bytes, got {a.size}")
        self._check(lib().rtlbfs_set_state_raw(self._h, _vp(a.ctypes.data), float(T_unit)),
                    "set_state_raw")

    # -- stepping
    def step(self, n: int):
        self._check(lib().rtlbfs_step(self._h, int(n)), "step")

    def run_to_steady(self, tol: float, max_steps: int, timeout_s: float = 0.0):
        """Returns (rc, steps_taken, (R_u, R_T)); rc 0 = converged."""
        steps = C.c_long(0)
        res = np.full(2, np.nan)
        rc = lib().rtlbfs_run_to_steady(self._h, float(tol), int(max_steps), float(timeout_s),
                                        C.byref(steps), _ptr(res))
        if rc not in (OK, ERR_NOT_CONVERGED, ERR_TIMEOUT, ERR_DIVERGED):
            self._check(rc, "run_to_steady")
        return rc, int(steps.value), (float(res[0]), float(res[1]))

    def residual(self):
        res = np.full(2, np.nan)
        steps = C.c_long(0)
        self._check(lib().rtlbfs_residual(self._h, _ptr(res), C.byref(steps)), "residual")
        return (float(res[0]), float(res[1])), int(steps.value)

    def nusselt(self, which: int) -> float:
        out = np.empty(1)
        self._check(lib().rtlbfs_nusselt(self._h, int(which), _ptr(out)), "nusselt")
        return float(out[0])

    def sync(self):
        self._check(lib().rtlbfs_sync(self._h), "sync")


class Batch:
    """Many cavities advanced together (a batch of ``include/rtlbfs_batch.h``)."""

    def __init__(self, precision: int = FP32, max_slots: int = 64):
        h = _vp()
        rc = lib().rtlbfs_batch_create(int(precision), int(max_slots), C.byref(h))
        if rc:
            raise RTLBFSError(rc, "rtlbfs_batch_create")
        self._h = h
        self.max_slots = max_slots
        self.precision = precision
        self.shapes = {}
        self._nbytes = {}  # raw_bytes of each slot in use (fixed until it is removed)

    def _check(self, rc, what):
        if rc:
            msg = lib().rtlbfs_batch_last_error(self._h)
            raise RTLBFSError(rc, f"{what}: {msg.decode() if msg else ''}")

    def close(self):
        if getattr(self, "_h", None):
            lib().rtlbfs_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add(self, xf, yf, Ra, Pr, Ma, dt) -> int:
        xf = np.ascontiguousarray(xf, dtype=np.float64)
        yf = np.ascontiguousarray(yf, dtype=np.float64)
        s = C.c_int(-1)
        self._check(lib().rtlbfs_batch_add(self._h, len(xf) - 1, len(yf) - 1, _ptr(xf), _ptr(yf),
                                           Ra, Pr, Ma, dt, C.byref(s)), "batch_add")
        self.shapes[s.value] = (len(yf) - 1, len(xf) - 1)
        self._nbytes.pop(s.value, None)
        return int(s.value)

    def set_bc(self, slot, side, kind, T_wall=0.0, u_wall=0.0):
        self._check(lib().rtlbfs_batch_set_bc(self._h, slot, side, kind, T_wall, u_wall),
                    "batch_set_bc")

    def set_lattice(self, slot, kappa):
        self._check(lib().rtlbfs_batch_set_lattice(self._h, slot, float(kappa)),
                    "batch_set_lattice")

    def set_state(self, slot, rho, u, v, T):
        ny, nx = self.shapes[slot]
        arrs = [_f64(a, nx * ny) for a in (rho, u, v, T)]
        self._check(lib().rtlbfs_batch_set_state(self._h, slot, *[_ptr(a) for a in arrs]),
                    "batch_set_state")

    def get_state(self, slot):
        ny, nx = self.shapes[slot]
        out = [np.empty((ny, nx)) for _ in range(4)]
        self._check(lib().rtlbfs_batch_get_state(self._h, slot, *[_ptr(a) for a in out]),
                    "batch_get_state")
        return tuple(out)

    def raw_bytes(self, slot) -> int:
        nb = self._nbytes.get(slot)
        if nb is None:
            nb = int(lib().rtlbfs_batch_state_raw_bytes(self._h, int(slot)))
            if nb:
                self._nbytes[slot] = nb
        return nb

    def get_state_raw(self, slot, out=None):
        """(records, T_unit) of a slot: its cell records as a uint8 array (or
        into `out`, any writable buffer of raw_bytes(slot) bytes) and the
        temperature unit."""
        nb = self.raw_bytes(slot)  # 0: not a slot in use, refused by the library
        out = np.empty(nb, dtype=np.uint8) if out is None else _raw_out(out, nb)
        tu = C.c_double()
        self._check(lib().rtlbfs_batch_get_state_raw(self._h, int(slot), _vp(out.ctypes.data),
                                                     C.byref(tu)), "batch_get_state_raw")
        return out, tu.value

    def set_state_raw(self, slot, records, T_unit: float = 1.0):
        a = np.ascontiguousarray(records).view(np.uint8).reshape(-1)
        if a.size != self.raw_bytes(slot):
            raise ValueError(f"expected {self.raw_bytes(slot)} bytes, got {a.size}")
        self._check(lib().rtlbfs_batch_set_state_raw(self._h, int(slot), _vp(a.ctypes.data),
                                                     float(T_unit)), "batch_set_state_raw")

    def get_states_raw(self, slots, outs):
        """Records of several slots in one call, into the writable buffers
        outs[k] (raw_bytes(slots[k]) bytes each); returns their T_units."""
        n = len(slots)
        if len(outs) != n:
            raise ValueError(f"{n} slots but {len(outs)} output buffers")
        sl = np.ascontiguousarray(slots, dtype=np.int32)
        arrs = [_raw_out(o, self.raw_bytes(s)) for s, o in zip(slots, outs)]
        ptrs = (_vp * n)(*[_vp(a.ctypes.data) for a in arrs])
        tu = np.empty(n)
        self._check(lib().rtlbfs_batch_get_states_raw(self._h, n, _vp(sl.ctypes.data),
                                                      C.cast(ptrs, _vp), _ptr(tu)),
                    "batch_get_states_raw")
        return tu

    def set_states_raw(self, slots, recs, T_units):
        """Restore several slots' records in one call."""
        n = len(slots)
        if len(recs) != n or len(T_units) != n:
            raise ValueError(f"{n} slots but {len(recs)} record buffers and {len(T_units)} units")
        sl = np.ascontiguousarray(slots, dtype=np.int32)
        arrs = [np.ascontiguousarray(r).view(np.uint8).reshape(-1) for r in recs]
        for s, a in zip(slots, arrs):
            nb = self.raw_bytes(s)  # 0: not a slot in use, refused by the library
            if nb and a.size != nb:
                raise ValueError(f"slot {s}: expected {nb} bytes, got {a.size}")
        ptrs = (_vp * n)(*[_vp(a.ctypes.data) for a in arrs])
        tu = np.ascontiguousarray(T_units, dtype=np.float64)
        self._check(lib().rtlbfs_batch_set_states_raw(self._h, n, _vp(sl.ctypes.data),
                                                      C.cast(ptrs, _vp), _ptr(tu)),
                    "batch_set_states_raw")

    def arm(self, slot, tol, max_steps):
        self._check(lib().rtlbfs_batch_arm(self._h, slot, float(tol), int(max_steps)), "batch_arm")

    def set_schedule(self, kernel: int = 0, chunk_rows: int = 0):
        """Step kernel (0 marching, 1 tiles) and its rows per unit / tile height."""
        self._check(lib().rtlbfs_batch_set_schedule(self._h, int(kernel), int(chunk_rows)),
                    "batch_set_schedule")

    def arm_many(self, slots, tol, max_steps):
        """arm() for several slots in one launch."""
        sl = np.ascontiguousarray(slots, dtype=np.int32)
        self._check(lib().rtlbfs_batch_arm_many(self._h, len(sl), _vp(sl.ctypes.data), float(tol),
                                                int(max_steps)), "batch_arm_many")

    def step(self, nsteps):
        self._check(lib().rtlbfs_batch_step(self._h, int(nsteps)), "batch_step")

    def poll(self):
        st = (C.c_int * self.max_slots)()
        steps = (C.c_long * self.max_slots)()
        res = np.empty(2 * self.max_slots)
        self._check(lib().rtlbfs_batch_poll(self._h, st, steps, _ptr(res)), "batch_poll")
        return list(st), list(steps), res.reshape(-1, 2)

    def nusselt(self, slot, which):
        out = np.empty(1)
        self._check(lib().rtlbfs_batch_nusselt(self._h, slot, int(which), _ptr(out)),
                    "batch_nusselt")
        return float(out[0])

    def remove(self, slot):
        self._check(lib().rtlbfs_batch_remove(self._h, slot), "batch_remove")
        self.shapes.pop(slot, None)
        self._nbytes.pop(slot, None)

    def autotune(self, steps=32):
        k, r, ms = C.c_int(0), C.c_int(0), C.c_double(0)
        self._check(lib().rtlbfs_batch_autotune(self._h, int(steps), C.byref(k), C.byref(r),
                                                C.byref(ms)), "batch_autotune")
        return int(k.value), int(r.value), float(ms.value)

    def set_stream(self, stream):
        ptr = None if stream is None else int(getattr(stream, "cuda_stream", stream))
        self._check(lib().rtlbfs_batch_set_stream(self._h, ptr), "batch_set_stream")

    def info(self):
        cells, slots, units = C.c_longlong(0), C.c_int(0), C.c_int(0)
        self._check(lib().rtlbfs_batch_info(self._h, C.byref(cells), C.byref(slots),
                                            C.byref(units)), "batch_info")
        return int(cells.value), int(slots.value), int(units.value)


def batch_bytes(precision, nx, ny) -> int:
    return int(lib().rtlbfs_batch_bytes(int(precision), int(nx), int(ny)))


def serve(requests, *, max_slots=64, mem_fraction=0.5, tol=1e-8, max_steps=100000, Ma=0.1,
          time_limit_s=0.0, chunk_steps=256, precision=FP32):
    """Replay (t_arrive, n, Ra, Pr) requests through the library's request
    loop; returns (list of result dicts, elapsed seconds)."""
    n = len(requests)
    reqs = (Request * max(n, 1))()
    for k, (t, nn, Ra, Pr) in enumerate(requests):
        reqs[k].t_arrive, reqs[k].n, reqs[k].Ra, reqs[k].Pr = float(t), int(nn), float(Ra), float(Pr)
    out = (Result * max(n, 1))()
    opts = ServeOpts(int(max_slots), float(mem_fraction), float(tol), int(max_steps), float(Ma),
                     float(time_limit_s), int(chunk_steps), int(precision))
    el = C.c_double(0)
    rc = lib().rtlbfs_serve(reqs, n, C.byref(opts), out, C.byref(el))
    if rc:
        raise RTLBFSError(rc, "rtlbfs_serve")
    res = [dict(t_admit=r.t_admit, t_finish=r.t_finish, steps=r.steps, status=r.status,
                nu_hot=r.nu_hot, nu_cold=r.nu_cold) for r in out[:n]]
    return res, float(el.value)


def stability_map(n, Ra, kappa, dt=None, *, Pr=0.71, Ma=0.1, tol=1e-9, max_steps=200000,
                  precision=FP32, chunk_steps=256):
    """Section 3.3's stability test for cases (n[k], Ra[k], kappa[k], dt[k])
    in one batch; returns (status array, steps array, elapsed seconds)."""
    m = len(n)
    nn = (C.c_int * max(m, 1))(*[int(x) for x in n])
    ra = np.ascontiguousarray(Ra, dtype=np.float64)
    ka = np.ascontiguousarray(kappa, dtype=np.float64)
    dd = None if dt is None else np.ascontiguousarray(dt, dtype=np.float64)
    st = (C.c_int * max(m, 1))()
    steps = (C.c_long * max(m, 1))()
    el = C.c_double(0)
    rc = lib().rtlbfs_stability_map(m, nn, _ptr(ra), _ptr(ka), None if dd is None else _ptr(dd),
                                    float(Pr), float(Ma), float(tol), int(max_steps),
                                    int(precision), int(chunk_steps), st, steps, C.byref(el))
    if rc:
        raise RTLBFSError(rc, "rtlbfs_stability_map")
    return np.array(st[:m]), np.array(steps[:m]), float(el.value)


# ---------------------------------------------------------------------------
# 3D (include/rtlbfs3d.h)
# ---------------------------------------------------------------------------
XM, XP, YM, YP, ZM, ZP, MID_X = 0, 1, 2, 3, 4, 5, 6


def op_counts3(scheme: int = 0):
    """(FP ops per face, FP ops per cell-update, SFU ops per cell-update) of
    the 3D step with face stage `scheme` (RTLBFS or TLBFS), each face and
    gradient evaluated once (host-only)."""
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    rc = lib().rtlbfs3d_op_counts_scheme(int(scheme), C.byref(a), C.byref(b), C.byref(c))
    if rc:
        raise RTLBFSError(rc, "rtlbfs3d_op_counts")
    return a.value, b.value, c.value


class Solver3:
    """One 3D mesh on the GPU (a handle of ``include/rtlbfs3d.h``); the state
    is five arrays (rho, u, v, w, T) of shape (nz, ny, nx)."""

    def __init__(self, xf, yf, zf, precision: int = FP64):
        L = lib()
        self.f = [np.ascontiguousarray(a, dtype=np.float64) for a in (xf, yf, zf)]
        self.nx, self.ny, self.nz = (len(a) - 1 for a in self.f)
        self.precision = precision
        h = _vp()
        rc = L.rtlbfs3d_create(self.nx, self.ny, self.nz, *[_ptr(a) for a in self.f],
                               int(precision), C.byref(h))
        if rc:
            raise RTLBFSError(rc, "rtlbfs3d_create")
        self._h = h

    def _check(self, rc: int, what: str):
        if rc:
            msg = lib().rtlbfs3d_last_error(self._h)
            raise RTLBFSError(rc, f"{what}: {msg.decode() if msg else ''}")

    def close(self):
        if getattr(self, "_h", None):
            lib().rtlbfs3d_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    def set_params(self, Ra, Pr, Ma, dt):
        self._check(lib().rtlbfs3d_set_params(self._h, Ra, Pr, Ma, dt), "set_params")

    def set_physics(self, nu, chi, beta_g):
        self._check(lib().rtlbfs3d_set_physics(self._h, nu, chi, beta_g), "set_physics")

    def set_lattice(self, kappa):
        self._check(lib().rtlbfs3d_set_lattice(self._h, kappa), "set_lattice")

    def set_gravity_axis(self, axis):
        self._check(lib().rtlbfs3d_set_gravity_axis(self._h, int(axis)), "set_gravity_axis")

    def set_body_force(self, fx, fy, fz):
        self._check(lib().rtlbfs3d_set_body_force(self._h, fx, fy, fz), "set_body_force")

    def set_bc(self, side, kind, T_wall=0.0, u_wall=(0.0, 0.0, 0.0)):
        uw = np.ascontiguousarray(u_wall, dtype=np.float64)
        self._check(lib().rtlbfs3d_set_bc(self._h, int(side), int(kind), float(T_wall), _ptr(uw)),
                    "set_bc")

    def set_scheme(self, scheme: int):
        """Face stage: RTLBFS (0, Section 3.2) or TLBFS (1, Section 2.2)."""
        self._check(lib().rtlbfs3d_set_scheme(self._h, int(scheme)), "set_scheme")

    def set_schedule(self, tile: int = 0, kchunk: int = 0):
        """tile 0: 32 x 4, 1: 16 x 8, 2: 32 x 8 columns per block; kchunk
        z-planes per work unit (0: automatic)."""
        self._check(lib().rtlbfs3d_set_schedule(self._h, int(tile), int(kchunk)), "set_schedule")

    def autotune(self, steps: int = 32):
        t, ms = C.c_int(0), C.c_double(0)
        self._check(lib().rtlbfs3d_autotune(self._h, int(steps), C.byref(t), C.byref(ms)),
                    "autotune")
        return int(t.value), float(ms.value)

    def set_stream(self, stream):
        ptr = None if stream is None else int(getattr(stream, "cuda_stream", stream))
        self._check(lib().rtlbfs3d_set_stream(self._h, ptr), "set_stream")

    def sync(self):
        self._check(lib().rtlbfs3d_sync(self._h), "sync")

    def set_state(self, rho, u, v, w, T):
        n = self.nx * self.ny * self.nz
        arrs = [_f64(a, n) for a in (rho, u, v, w, T)]
        self._check(lib().rtlbfs3d_set_state(self._h, *[_ptr(a) for a in arrs]), "set_state")

    def get_state(self):
        out = [np.empty(self.shape) for _ in range(5)]
        self._check(lib().rtlbfs3d_get_state(self._h, *[_ptr(a) for a in out]), "get_state")
        return tuple(out)

    def step(self, n: int):
        self._check(lib().rtlbfs3d_step(self._h, int(n)), "step")

    def step_rc(self, n: int) -> int:
        """step() returning the status code instead of raising."""
        return int(lib().rtlbfs3d_step(self._h, int(n)))

    def run_to_steady(self, tol: float, max_steps: int, timeout_s: float = 0.0):
        """Returns (rc, steps_taken, (R_u, R_T)); rc 0 = converged."""
        steps = C.c_long(0)
        res = np.full(2, np.nan)
        rc = lib().rtlbfs3d_run_to_steady(self._h, float(tol), int(max_steps), float(timeout_s),
                                          C.byref(steps), _ptr(res))
        if rc not in (OK, ERR_NOT_CONVERGED, ERR_TIMEOUT, ERR_DIVERGED):
            self._check(rc, "run_to_steady")
        return int(rc), int(steps.value), (float(res[0]), float(res[1]))

    def residual(self):
        res = np.full(2, np.nan)
        steps = C.c_long(0)
        self._check(lib().rtlbfs3d_residual(self._h, _ptr(res), C.byref(steps)), "residual")
        return (float(res[0]), float(res[1])), int(steps.value)

    def nusselt(self, side: int, mid: bool = False) -> float:
        out = C.c_double(0)
        self._check(lib().rtlbfs3d_nusselt(self._h, int(side), int(bool(mid)), C.byref(out)),
                    "nusselt")
        return float(out.value)


# ---------------------------------------------------------------------------
# Curvilinear 2D (include/rtlbfs_curv.h)
# ---------------------------------------------------------------------------
FARFIELD = 3


def op_counts_curv():
    """(FP ops per face, per cell-update, SFU ops per cell-update) of the
    curvilinear step (host-only)."""
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    rc = lib().rtlbfsc_op_counts(C.byref(a), C.byref(b), C.byref(c))
    if rc:
        raise RTLBFSError(rc, "rtlbfsc_op_counts")
    return a.value, b.value, c.value


class SolverC:
    """One body-fitted 2D mesh on the GPU (a handle of include/rtlbfs_curv.h);
    vertices X, Y of shape (nj+1, ni+1), fields of shape (nj, ni)."""

    def __init__(self, X, Y, periodic_i: bool, precision: int = FP64):
        self.X = np.ascontiguousarray(X, dtype=np.float64)
        self.Y = np.ascontiguousarray(Y, dtype=np.float64)
        self.nj, self.ni = self.X.shape[0] - 1, self.X.shape[1] - 1
        h = _vp()
        rc = lib().rtlbfsc_create(self.ni, self.nj, _ptr(self.X), _ptr(self.Y),
                                  int(bool(periodic_i)), int(precision), C.byref(h))
        if rc:
            raise RTLBFSError(rc, "rtlbfsc_create")
        self._h = h

    def _check(self, rc: int, what: str):
        if rc:
            msg = lib().rtlbfsc_last_error(self._h)
            raise RTLBFSError(rc, f"{what}: {msg.decode() if msg else ''}")

    def close(self):
        if getattr(self, "_h", None):
            lib().rtlbfsc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_physics(self, nu, chi, beta_g, dt):
        self._check(lib().rtlbfsc_set_physics(self._h, nu, chi, beta_g, dt), "set_physics")

    def set_lattice(self, kappa):
        self._check(lib().rtlbfsc_set_lattice(self._h, kappa), "set_lattice")

    def set_gravity(self, gx, gy, T_ref=0.5):
        self._check(lib().rtlbfsc_set_gravity(self._h, gx, gy, T_ref), "set_gravity")

    def set_body_force(self, fx, fy):
        self._check(lib().rtlbfsc_set_body_force(self._h, fx, fy), "set_body_force")

    def set_bc(self, side, kind, T_wall=0.0, ux=0.0, uy=0.0):
        self._check(lib().rtlbfsc_set_bc(self._h, int(side), int(kind), float(T_wall), float(ux),
                                         float(uy)), "set_bc")

    def set_farfield(self, rho, u, v, T):
        self._check(lib().rtlbfsc_set_farfield(self._h, rho, u, v, T), "set_farfield")

    def set_schedule(self, tile_rows: int = 0):
        self._check(lib().rtlbfsc_set_schedule(self._h, int(tile_rows)), "set_schedule")

    def set_stream(self, stream):
        ptr = None if stream is None else int(getattr(stream, "cuda_stream", stream))
        self._check(lib().rtlbfsc_set_stream(self._h, ptr), "set_stream")

    def set_state(self, rho, u, v, T):
        n = self.ni * self.nj
        arrs = [_f64(a, n) for a in (rho, u, v, T)]
        self._check(lib().rtlbfsc_set_state(self._h, *[_ptr(a) for a in arrs]), "set_state")

    def get_state(self):
        out = [np.empty((self.nj, self.ni)) for _ in range(4)]
        self._check(lib().rtlbfsc_get_state(self._h, *[_ptr(a) for a in out]), "get_state")
        return tuple(out)

    def step(self, n: int):
        self._check(lib().rtlbfsc_step(self._h, int(n)), "step")

    def step_rc(self, n: int) -> int:
        return int(lib().rtlbfsc_step(self._h, int(n)))

    def run_to_steady(self, tol: float, max_steps: int, timeout_s: float = 0.0):
        steps = C.c_long(0)
        res = np.full(2, np.nan)
        rc = lib().rtlbfsc_run_to_steady(self._h, float(tol), int(max_steps), float(timeout_s),
                                         C.byref(steps), _ptr(res))
        if rc not in (OK, ERR_NOT_CONVERGED, ERR_TIMEOUT, ERR_DIVERGED):
            self._check(rc, "run_to_steady")
        return int(rc), int(steps.value), (float(res[0]), float(res[1]))

    def residual(self):
        res = np.full(2, np.nan)
        steps = C.c_long(0)
        self._check(lib().rtlbfsc_residual(self._h, _ptr(res), C.byref(steps)), "residual")
        return (float(res[0]), float(res[1])), int(steps.value)

    def wall_heat(self, side: int):
        q, per = C.c_double(0), C.c_double(0)
        self._check(lib().rtlbfsc_wall_heat(self._h, int(side), C.byref(q), C.byref(per)),
                    "wall_heat")
        return float(q.value), float(per.value)
