"""FP64 CPU oracle of 2D RTLBFS on structured curvilinear (body-fitted)
quadrilateral meshes (arXiv 2202.13449, Section 3.2 with the local lattice of
each face; the O-meshes of Section 4.3).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``: ctypes marshalling of
``rtlbfs_curv_oracle.c`` (whose header comment lists the steps and the
readings).  Vertices X, Y have shape (nj+1, ni+1); fields (rho, u, v, T)
shape (nj, ni).  Sides: 0 i = 0, 1 i = ni, 2 j = 0, 3 j = nj.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

import numpy as np

from . import lib as _lib2d

DIRICHLET, ADIABATIC, PERIODIC, FARFIELD = 0, 1, 2, 3


class _ProblemC(C.Structure):
    _fields_ = [
        ("ni", C.c_int), ("nj", C.c_int),
        ("X", C.POINTER(C.c_double)), ("Y", C.POINTER(C.c_double)),
        ("nu", C.c_double), ("chi", C.c_double), ("beta_g", C.c_double),
        ("T_ref", C.c_double), ("dT", C.c_double), ("dt", C.c_double), ("kappa", C.c_double),
        ("gdir", C.c_double * 2), ("force", C.c_double * 2),
        ("bc_kind", C.c_int * 4), ("bc_T", C.c_double * 4), ("bc_u", C.c_double * 8),
        ("inf", C.c_double * 4),
    ]


class FaceOutC(C.Structure):
    _fields_ = [
        ("h", C.c_double), ("tau_f", C.c_double), ("tau_g", C.c_double),
        ("n", C.c_double * 2), ("len", C.c_double),
        ("node", C.c_double * 36), ("pred", C.c_double * 4), ("flux", C.c_double * 4),
    ]

    def nodes(self) -> np.ndarray:
        """Frame primitives (rho, u_n, u_t, T) at node (a, b): shape (4, 3, 3)."""
        return np.array(self.node[:], dtype=np.float64).reshape(4, 3, 3)


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = _lib2d()
        dp = C.POINTER(C.c_double)
        pp = C.POINTER(_ProblemC)
        L.orcc_step.argtypes = [pp, dp, dp, dp, dp, C.c_long, dp]
        L.orcc_run_to_steady.argtypes = [pp, dp, dp, dp, dp, C.c_double, C.c_long,
                                         C.POINTER(C.c_long), dp]
        L.orcc_gradients.argtypes = [pp, dp, dp, dp, dp, dp, dp]
        L.orcc_face.argtypes = [pp, dp, dp, dp, dp, C.c_int, C.c_int, C.c_int,
                                C.POINTER(FaceOutC)]
        L.orcc_heat.argtypes = [pp, dp, dp, dp, dp, C.c_int, dp, dp]
        for f in ("orcc_step", "orcc_run_to_steady", "orcc_gradients", "orcc_face", "orcc_heat"):
            getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


@dataclass
class ProblemC:
    """Mesh, physics and boundary conditions of one curvilinear case."""
    X: np.ndarray
    Y: np.ndarray
    nu: float
    chi: float
    beta_g: float = 0.0
    T_ref: float = 0.5
    dT: float = 1.0
    dt: float = 0.5
    kappa: float = 1.0
    gdir: tuple = (0.0, 1.0)
    force: tuple = (0.0, 0.0)
    bc_kind: tuple = (PERIODIC, PERIODIC, DIRICHLET, DIRICHLET)
    bc_T: tuple = (0.0, 0.0, 1.0, 0.0)
    bc_u: tuple = ((0.0, 0.0),) * 4
    inf: tuple = (1.0, 0.0, 0.0, 0.0)
    _keep: list = field(default_factory=list, repr=False)

    @property
    def shape(self):
        return (self.X.shape[0] - 1, self.X.shape[1] - 1)

    def c(self) -> _ProblemC:
        X = np.ascontiguousarray(self.X, dtype=np.float64)
        Y = np.ascontiguousarray(self.Y, dtype=np.float64)
        self._keep = [X, Y]
        p = _ProblemC()
        p.nj, p.ni = X.shape[0] - 1, X.shape[1] - 1
        p.X, p.Y = _dp(X), _dp(Y)
        p.nu, p.chi, p.beta_g, p.T_ref, p.dT = self.nu, self.chi, self.beta_g, self.T_ref, self.dT
        p.dt, p.kappa = self.dt, self.kappa
        p.gdir[:] = list(self.gdir)
        p.force[:] = list(self.force)
        p.bc_kind[:] = list(self.bc_kind)
        p.bc_T[:] = list(self.bc_T)
        p.bc_u[:] = [float(x) for uw in self.bc_u for x in uw]
        p.inf[:] = list(self.inf)
        return p


def _state(st):
    return [np.ascontiguousarray(a, dtype=np.float64).copy() for a in st]


def step(prob: ProblemC, state, nsteps: int):
    s = _state(state)
    res = np.full(2, np.nan)
    p = prob.c()
    rc = lib().orcc_step(C.byref(p), *map(_dp, s), int(nsteps), _dp(res))
    if rc == -1:
        raise ValueError("orcc_step: bad arguments (or a left-handed mesh)")
    return tuple(s), (float(res[0]), float(res[1])), rc


def run_to_steady(prob: ProblemC, state, tol: float, max_steps: int):
    s = _state(state)
    res = np.full(2, np.nan)
    steps = C.c_long(0)
    p = prob.c()
    rc = lib().orcc_run_to_steady(C.byref(p), *map(_dp, s), float(tol), int(max_steps),
                                  C.byref(steps), _dp(res))
    if rc == -1:
        raise ValueError("orcc_run_to_steady: bad arguments")
    return tuple(s), int(steps.value), (float(res[0]), float(res[1])), rc


def gradients(prob: ProblemC, state):
    """(gradients (4, 2, nj, ni), geometry (3, nj, ni): centre x, y, area)."""
    s = _state(state)
    nj, ni = prob.shape
    g = np.empty(8 * ni * nj)
    geo = np.empty(3 * ni * nj)
    p = prob.c()
    rc = lib().orcc_gradients(C.byref(p), *map(_dp, s), _dp(g), _dp(geo))
    if rc:
        raise ValueError(f"orcc_gradients rc={rc}")
    return g.reshape(4, 2, nj, ni), geo.reshape(3, nj, ni)


def face(prob: ProblemC, state, kind: int, i: int, j: int) -> FaceOutC:
    s = _state(state)
    o = FaceOutC()
    p = prob.c()
    rc = lib().orcc_face(C.byref(p), *map(_dp, s), int(kind), int(i), int(j), C.byref(o))
    if rc:
        raise ValueError(f"orcc_face rc={rc}")
    return o


def heat(prob: ProblemC, state, side: int):
    """(sum over the side's faces of the energy flux times the face length,
    along increasing j; the side's length)."""
    s = _state(state)
    out, per = np.empty(1), np.empty(1)
    p = prob.c()
    rc = lib().orcc_heat(C.byref(p), *map(_dp, s), int(side), _dp(out), _dp(per))
    if rc:
        raise ValueError(f"orcc_heat rc={rc}")
    return float(out[0]), float(per[0])
