"""FP64 CPU oracle of 3D RTLBFS (arXiv 2202.13449, Section 3.2 with the
D3Q19 lattice of Eqs. 5-6; the cubic cavity of Section 4.4).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``: ctypes marshalling
of ``rtlbfs3d_oracle.c`` (whose header comment lists the equations and the
readings taken).  The state is five arrays (rho, u, v, w, T) of shape
(nz, ny, nx); sides are numbered 0 -x, 1 +x, 2 -y, 3 +y, 4 -z, 5 +z.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

import numpy as np

from . import (DIRICHLET, ADIABATIC, PERIODIC, RTLBFS, TLBFS, lib as _lib2d,  # noqa: F401
               params_from_ra, tanh_faces)

NQ = 5
MID_PLANE_X = 6  # side value of nusselt(): the x-normal face plane at nx/2


class _Problem3(C.Structure):
    _fields_ = [
        ("n", C.c_int * 3),
        ("f", C.POINTER(C.c_double) * 3),
        ("nu", C.c_double), ("chi", C.c_double), ("beta_g", C.c_double),
        ("T_ref", C.c_double), ("dT", C.c_double),
        ("dt", C.c_double), ("kappa", C.c_double),
        ("force", C.c_double * 3),
        ("g_axis", C.c_int),
        ("bc_kind", C.c_int * 6), ("bc_T", C.c_double * 6), ("bc_u", C.c_double * 18),
        ("scheme", C.c_int),
    ]


class FaceOut3(C.Structure):
    _fields_ = [
        ("h", C.c_double), ("tau_f", C.c_double), ("tau_g", C.c_double),
        ("node", C.c_double * (NQ * 19)), ("pred", C.c_double * 5), ("flux", C.c_double * 5),
    ]

    def nodes(self) -> np.ndarray:
        """Primitives at the 19 nodes, shape (5, 19) = [q][D3Q19 index]."""
        return np.array(self.node[:], dtype=np.float64).reshape(NQ, 19)


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = _lib2d()
        dp = C.POINTER(C.c_double)
        pp = C.POINTER(_Problem3)
        st = [dp] * 5
        L.orc3_step.argtypes = [pp, *st, C.c_long, dp]
        L.orc3_run_to_steady.argtypes = [pp, *st, C.c_double, C.c_long, C.POINTER(C.c_long), dp]
        L.orc3_gradients.argtypes = [pp, *st, dp]
        L.orc3_face.argtypes = [pp, *st, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(FaceOut3)]
        L.orc3_face_from_nodes.argtypes = [pp, C.c_int, dp, C.c_double, C.c_int,
                                           C.POINTER(FaceOut3)]
        L.orc3_lattice.argtypes = [C.POINTER(C.c_int)]
        L.orc3_fluxes.argtypes = [pp, *st, dp, dp, dp]
        L.orc3_nusselt.argtypes = [pp, *st, C.c_int, C.c_int, dp]
        for f in ("orc3_step", "orc3_run_to_steady", "orc3_gradients", "orc3_face",
                  "orc3_face_from_nodes", "orc3_lattice", "orc3_fluxes", "orc3_nusselt"):
            getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def lattice() -> np.ndarray:
    """The D3Q19 velocities the oracle uses, shape (19, 3)."""
    out = (C.c_int * 57)()
    lib().orc3_lattice(out)
    return np.array(out[:], dtype=np.int64).reshape(19, 3)


@dataclass
class Problem3:
    """Mesh, physics and boundary conditions of one 3D case (oracle side)."""
    xf: np.ndarray
    yf: np.ndarray
    zf: np.ndarray
    nu: float
    chi: float
    beta_g: float = 0.0
    T_ref: float = 0.5
    dT: float = 1.0
    dt: float = 0.5
    kappa: float = 1.0
    force: tuple = (0.0, 0.0, 0.0)
    g_axis: int = 2
    # Section 4.4: cold -x wall, hot +x wall, the other four adiabatic, no slip
    bc_kind: tuple = (DIRICHLET, DIRICHLET, ADIABATIC, ADIABATIC, ADIABATIC, ADIABATIC)
    bc_T: tuple = (0.0, 1.0, 0.0, 0.0, 0.0, 0.0)
    bc_u: tuple = ((0.0, 0.0, 0.0),) * 6
    scheme: int = 0  # 0 RTLBFS (Section 3.2), 1 TLBFS (Section 2.2)
    _keep: list = field(default_factory=list, repr=False)

    @property
    def shape(self):
        """(nz, ny, nx)"""
        return (len(self.zf) - 1, len(self.yf) - 1, len(self.xf) - 1)

    def c(self) -> _Problem3:
        fs = [np.ascontiguousarray(a, dtype=np.float64) for a in (self.xf, self.yf, self.zf)]
        self._keep = fs
        p = _Problem3()
        for a in range(3):
            p.n[a] = len(fs[a]) - 1
            p.f[a] = _dp(fs[a])
        p.nu, p.chi, p.beta_g = self.nu, self.chi, self.beta_g
        p.T_ref, p.dT, p.dt, p.kappa = self.T_ref, self.dT, self.dt, self.kappa
        p.force[:] = list(self.force)
        p.g_axis = int(self.g_axis)
        p.bc_kind[:] = list(self.bc_kind)
        p.bc_T[:] = list(self.bc_T)
        p.bc_u[:] = [float(x) for uw in self.bc_u for x in uw]
        p.scheme = int(self.scheme)
        return p


def _state(st):
    return [np.ascontiguousarray(a, dtype=np.float64).copy() for a in st]


def step(prob: Problem3, state, nsteps: int):
    """Advance ``nsteps``; returns (new_state, (R_u, R_T) of the last step, rc)."""
    s = _state(state)
    res = np.full(2, np.nan)
    p = prob.c()
    rc = lib().orc3_step(C.byref(p), *map(_dp, s), int(nsteps), _dp(res))
    if rc == -1:
        raise ValueError("orc3_step: bad arguments")
    return tuple(s), (float(res[0]), float(res[1])), rc


def run_to_steady(prob: Problem3, state, tol: float, max_steps: int):
    """Step until max(R_u, R_T) < tol; returns (state, steps, (R_u, R_T), rc)
    with rc 0 converged, -5 max_steps reached, -4 diverged."""
    s = _state(state)
    res = np.full(2, np.nan)
    steps = C.c_long(0)
    p = prob.c()
    rc = lib().orc3_run_to_steady(C.byref(p), *map(_dp, s), float(tol), int(max_steps),
                                  C.byref(steps), _dp(res))
    if rc == -1:
        raise ValueError("orc3_run_to_steady: bad arguments")
    return tuple(s), int(steps.value), (float(res[0]), float(res[1])), rc


def gradients(prob: Problem3, state) -> np.ndarray:
    """Eq. 55 gradients, shape (5, 3, nz, ny, nx): [q][d/dx, d/dy, d/dz]."""
    s = _state(state)
    out = np.empty(15 * int(np.prod(prob.shape)))
    p = prob.c()
    rc = lib().orc3_gradients(C.byref(p), *map(_dp, s), _dp(out))
    if rc:
        raise ValueError(f"orc3_gradients rc={rc}")
    return out.reshape(5, 3, *prob.shape)


def face(prob: Problem3, state, nd: int, i: int, j: int, k: int) -> FaceOut3:
    """One face's nodes, prediction and fluxes: normal axis nd, face position
    (i, j, k) whose index along nd runs over [0, n]."""
    s = _state(state)
    o = FaceOut3()
    p = prob.c()
    rc = lib().orc3_face(C.byref(p), *map(_dp, s), int(nd), int(i), int(j), int(k), C.byref(o))
    if rc:
        raise ValueError(f"orc3_face rc={rc}")
    return o


def face_from_nodes(prob: Problem3, nd: int, nodes, h: float, wall_side: int = -1) -> FaceOut3:
    """Predictor and fluxes (Eqs. 46-48, 57-59) from given node primitives of
    shape (5, 19); the mesh of ``prob`` is unused."""
    nodes = np.ascontiguousarray(nodes, dtype=np.float64).reshape(NQ * 19)
    o = FaceOut3()
    p = prob.c()
    rc = lib().orc3_face_from_nodes(C.byref(p), int(nd), _dp(nodes), float(h), int(wall_side),
                                    C.byref(o))
    if rc:
        raise ValueError(f"orc3_face_from_nodes rc={rc}")
    return o


def fluxes(prob: Problem3, state):
    """All face fluxes: a tuple of three arrays, axis a's of shape
    (5, nz + [a == 2], ny + [a == 1], nx + [a == 0])."""
    s = _state(state)
    nz, ny, nx = prob.shape
    shapes = [(5, nz, ny, nx + 1), (5, nz, ny + 1, nx), (5, nz + 1, ny, nx)]
    outs = [np.empty(int(np.prod(sh))) for sh in shapes]
    p = prob.c()
    rc = lib().orc3_fluxes(C.byref(p), *map(_dp, s), *map(_dp, outs))
    if rc:
        raise ValueError(f"orc3_fluxes rc={rc}")
    return tuple(o.reshape(sh) for o, sh in zip(outs, shapes))


def nusselt(prob: Problem3, state, side: int, mid: bool = False) -> float:
    """Nusselt number through wall ``side`` (Eq. 76), or along the wall's
    middle line (Eq. 75) with ``mid``; side MID_PLANE_X: the plane x = Lx/2."""
    s = _state(state)
    out = np.empty(1)
    p = prob.c()
    rc = lib().orc3_nusselt(C.byref(p), *map(_dp, s), int(side), int(bool(mid)), _dp(out))
    if rc:
        raise ValueError(f"orc3_nusselt rc={rc}")
    return float(out[0])


def cubic_cavity(n: int, Ra: float, Pr: float = 0.71, Ma: float = 0.1, phi: float = 0.0,
                 dt: float | None = None, kappa: float = 1.0, L: float | None = None) -> Problem3:
    """Cubic cavity of Section 4.4: n^3 cells on [0, L]^3 (L = n by default),
    Eq. 74 stretching with factor phi in all three directions, cold wall at
    x = 0 and hot wall at x = L, the other walls adiabatic, gravity along
    -z, no slip everywhere.  dt defaults to half the smallest cell width."""
    L = float(n) if L is None else float(L)
    f = tanh_faces(n, L, phi)
    nu, chi, bg = params_from_ra(Ra, Pr, Ma, L)
    if dt is None:
        dt = 0.5 * float(np.min(np.diff(f)))
    return Problem3(xf=f, yf=f.copy(), zf=f.copy(), nu=nu, chi=chi, beta_g=bg, T_ref=0.5,
                    dT=1.0, dt=dt, kappa=kappa)
