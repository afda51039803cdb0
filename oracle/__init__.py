"""FP64 CPU oracle of RTLBFS (arXiv 2202.13449, Section 3.2): 2D here, 3D
(D3Q19, Section 4.4) in ``oracle.d3``, 2D curvilinear meshes (Section 4.3)
in ``oracle.curv``.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product package
never imports this module, and the C source here shares no code with the
CUDA path.  ``build()`` compiles ``rtlbfs_oracle.c``, ``rtlbfs3d_oracle.c``
and ``rtlbfs_curv_oracle.c`` with gcc into
``oracle/_build/``; everything else is ctypes marshalling.

Functions mirror the C entry points (see the header comment of
``rtlbfs_oracle.c`` for the paper's equations and the readings taken):

* ``tanh_faces`` -- Eq. 74 mesh faces
* ``params_from_ra`` -- Eq. 63 / Eqs. 9-10 transport coefficients
* ``Problem`` -- mesh, physics and boundary conditions
* ``step`` / ``run_to_steady`` -- explicit RTLBFS steps (Eqs. 55-59, 64), or
  TLBFS steps (Section 2.2, Eqs. 29-43) with ``Problem.scheme = TLBFS``
* ``gradients`` / ``face`` / ``fluxes`` / ``nusselt`` -- intermediate results
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "rtlbfs_oracle.c"), os.path.join(_HERE, "rtlbfs3d_oracle.c"),
         os.path.join(_HERE, "rtlbfs_curv_oracle.c")]
_OUT = os.path.join(_HERE, "_build", "librtlbfs_oracle.so")

W, E, S, N = 0, 1, 2, 3
DIRICHLET, ADIABATIC, PERIODIC = 0, 1, 2
NU_W, NU_E, NU_S, NU_N, NU_A, NU_HALF = 0, 1, 2, 3, 4, 5
RTLBFS, TLBFS = 0, 1  # face stage of Problem.scheme


def build(force: bool = False) -> str:
    """Compile the oracle shared library from the 2D and 3D sources (gcc,
    OpenMP, no fast-math, no FMA contraction so x86 and Arm give the same
    bits)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if (not force and os.path.exists(_OUT)
            and all(os.path.getmtime(_OUT) >= os.path.getmtime(src) for src in _SRCS)):
        return _OUT
    tmp = _OUT + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-Wall", "-o", tmp, *_SRCS, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _OUT)
    return _OUT


class _Problem(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int),
        ("xf", C.POINTER(C.c_double)), ("yf", C.POINTER(C.c_double)),
        ("nu", C.c_double), ("chi", C.c_double), ("beta_g", C.c_double),
        ("T_ref", C.c_double), ("dT", C.c_double),
        ("dt", C.c_double), ("kappa", C.c_double),
        ("fx", C.c_double), ("fy", C.c_double),
        ("bc_kind", C.c_int * 4), ("bc_T", C.c_double * 4), ("bc_u", C.c_double * 4),
        ("scheme", C.c_int),
    ]


class FaceOut(C.Structure):
    _fields_ = [
        ("h", C.c_double), ("tau_f", C.c_double), ("tau_g", C.c_double),
        ("node", C.c_double * 36), ("pred", C.c_double * 4), ("flux", C.c_double * 4),
    ]

    def nodes(self) -> np.ndarray:
        """Primitives at the 9 nodes, shape (4, 3, 3) = [q][a+1][b+1]."""
        return np.array(self.node[:], dtype=np.float64).reshape(4, 3, 3)


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        pp = C.POINTER(_Problem)
        L.orc_tanh_faces.argtypes = [C.c_int, C.c_double, C.c_double, dp]
        L.orc_params.argtypes = [C.c_double] * 5 + [dp]
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_step.argtypes = [pp, dp, dp, dp, dp, C.c_long, dp]
        L.orc_run_to_steady.argtypes = [pp, dp, dp, dp, dp, C.c_double, C.c_long,
                                        C.POINTER(C.c_long), dp]
        L.orc_gradients.argtypes = [pp, dp, dp, dp, dp, dp]
        L.orc_face.argtypes = [pp, dp, dp, dp, dp, C.c_int, C.c_int, C.c_int,
                               C.POINTER(FaceOut)]
        L.orc_fluxes.argtypes = [pp, dp, dp, dp, dp, dp, dp]
        L.orc_face_from_nodes.argtypes = [pp, C.c_int, dp, C.c_double, C.c_int,
                                          C.POINTER(FaceOut)]
        L.orc_nusselt.argtypes = [pp, dp, dp, dp, dp, C.c_int, dp]
        for f in ("orc_tanh_faces", "orc_params", "orc_set_threads", "orc_step",
                  "orc_run_to_steady", "orc_gradients", "orc_face", "orc_fluxes", "orc_face_from_nodes",
                  "orc_nusselt"):
            getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def set_threads(n: int) -> int:
    """Set the OpenMP thread count (n <= 0 queries); returns the count in use."""
    return lib().orc_set_threads(int(n))


def tanh_faces(n: int, L: float, phi: float) -> np.ndarray:
    """Eq. 74 face coordinates (n+1 values); phi <= 0 gives a uniform mesh."""
    out = np.empty(n + 1, dtype=np.float64)
    rc = lib().orc_tanh_faces(int(n), float(L), float(phi), _dp(out))
    if rc:
        raise ValueError(f"orc_tanh_faces rc={rc}")
    return out


def params_from_ra(Ra: float, Pr: float, Ma: float, L: float, dT: float = 1.0):
    """(nu, chi, beta_g) from Eq. 63 with V_c = Ma."""
    out = np.empty(3, dtype=np.float64)
    rc = lib().orc_params(float(Ra), float(Pr), float(Ma), float(L), float(dT), _dp(out))
    if rc:
        raise ValueError(f"orc_params rc={rc}")
    return float(out[0]), float(out[1]), float(out[2])


@dataclass
class Problem:
    """Mesh, physics and boundary conditions of one case (oracle side)."""
    xf: np.ndarray
    yf: np.ndarray
    nu: float
    chi: float
    beta_g: float = 0.0
    T_ref: float = 0.5
    dT: float = 1.0
    dt: float = 0.5
    kappa: float = 1.0
    fx: float = 0.0
    fy: float = 0.0
    bc_kind: tuple = (DIRICHLET, DIRICHLET, ADIABATIC, ADIABATIC)
    bc_T: tuple = (1.0, 0.0, 0.0, 0.0)
    bc_u: tuple = (0.0, 0.0, 0.0, 0.0)
    scheme: int = 0  # 0 RTLBFS (Section 3.2), 1 TLBFS (Section 2.2)
    _keep: list = field(default_factory=list, repr=False)

    @property
    def nx(self) -> int:
        return len(self.xf) - 1

    @property
    def ny(self) -> int:
        return len(self.yf) - 1

    def c(self) -> _Problem:
        xf = np.ascontiguousarray(self.xf, dtype=np.float64)
        yf = np.ascontiguousarray(self.yf, dtype=np.float64)
        self._keep = [xf, yf]
        p = _Problem()
        p.nx, p.ny = self.nx, self.ny
        p.xf, p.yf = _dp(xf), _dp(yf)
        p.nu, p.chi, p.beta_g = self.nu, self.chi, self.beta_g
        p.T_ref, p.dT, p.dt, p.kappa = self.T_ref, self.dT, self.dt, self.kappa
        p.fx, p.fy = self.fx, self.fy
        p.bc_kind[:] = list(self.bc_kind)
        p.bc_T[:] = list(self.bc_T)
        p.bc_u[:] = list(self.bc_u)
        p.scheme = int(self.scheme)
        return p


def _state(st):
    out = [np.ascontiguousarray(a, dtype=np.float64).copy() for a in st]
    return out


def step(prob: Problem, state, nsteps: int):
    """Advance ``nsteps``; returns (new_state, (R_u, R_T) of the last step, rc)."""
    rho, u, v, T = _state(state)
    res = np.full(2, np.nan)
    p = prob.c()
    rc = lib().orc_step(C.byref(p), _dp(rho), _dp(u), _dp(v), _dp(T), int(nsteps), _dp(res))
    if rc == -1:
        raise ValueError("orc_step: bad arguments")
    return (rho, u, v, T), (float(res[0]), float(res[1])), rc


def run_to_steady(prob: Problem, state, tol: float, max_steps: int):
    """Step until max(R_u, R_T) < tol; returns (state, steps, (R_u, R_T), rc)
    with rc 0 converged, -5 max_steps reached, -4 diverged."""
    rho, u, v, T = _state(state)
    res = np.full(2, np.nan)
    steps = C.c_long(0)
    p = prob.c()
    rc = lib().orc_run_to_steady(C.byref(p), _dp(rho), _dp(u), _dp(v), _dp(T), float(tol),
                                 int(max_steps), C.byref(steps), _dp(res))
    if rc == -1:
        raise ValueError("orc_run_to_steady: bad arguments")
    return (rho, u, v, T), int(steps.value), (float(res[0]), float(res[1])), rc


def gradients(prob: Problem, state) -> np.ndarray:
    """Eq. 55 gradients, shape (4, 2, ny, nx): [q][d/dx, d/dy]."""
    rho, u, v, T = _state(state)
    out = np.empty(8 * prob.nx * prob.ny)
    p = prob.c()
    rc = lib().orc_gradients(C.byref(p), _dp(rho), _dp(u), _dp(v), _dp(T), _dp(out))
    if rc:
        raise ValueError(f"orc_gradients rc={rc}")
    return out.reshape(4, 2, prob.ny, prob.nx)


def face(prob: Problem, state, nd: int, i: int, j: int) -> FaceOut:
    """One face's nodes, prediction and fluxes (nd 0: x-face i in [0,nx] of row j)."""
    rho, u, v, T = _state(state)
    o = FaceOut()
    p = prob.c()
    rc = lib().orc_face(C.byref(p), _dp(rho), _dp(u), _dp(v), _dp(T), int(nd), int(i), int(j),
                        C.byref(o))
    if rc:
        raise ValueError(f"orc_face rc={rc}")
    return o


def face_from_nodes(prob: Problem, nd: int, nodes, h: float, wall_side: int = -1) -> FaceOut:
    """Predictor and fluxes (Eqs. 46-48, 57-59) from given node primitives,
    shape (4, 3, 3) = [rho,u,v,T][a+1][b+1]; the mesh of ``prob`` is unused."""
    nodes = np.ascontiguousarray(nodes, dtype=np.float64).reshape(36)
    o = FaceOut()
    p = prob.c()
    rc = lib().orc_face_from_nodes(C.byref(p), int(nd), _dp(nodes), float(h), int(wall_side),
                                   C.byref(o))
    if rc:
        raise ValueError(f"orc_face_from_nodes rc={rc}")
    return o


def fluxes(prob: Problem, state):
    """All face fluxes: (fx (4, ny, nx+1), fy (4, ny+1, nx))."""
    rho, u, v, T = _state(state)
    nx, ny = prob.nx, prob.ny
    fx = np.empty(4 * ny * (nx + 1))
    fy = np.empty(4 * (ny + 1) * nx)
    p = prob.c()
    rc = lib().orc_fluxes(C.byref(p), _dp(rho), _dp(u), _dp(v), _dp(T), _dp(fx), _dp(fy))
    if rc:
        raise ValueError(f"orc_fluxes rc={rc}")
    return fx.reshape(4, ny, nx + 1), fy.reshape(4, ny + 1, nx)


def nusselt(prob: Problem, state, which: int) -> float:
    """Nusselt number: which 0..3 wall W/E/S/N, 4 Nu_a (Eq. 69), 5 Nu_1/2."""
    rho, u, v, T = _state(state)
    out = np.empty(1)
    p = prob.c()
    rc = lib().orc_nusselt(C.byref(p), _dp(rho), _dp(u), _dp(v), _dp(T), int(which), _dp(out))
    if rc:
        raise ValueError(f"orc_nusselt rc={rc}")
    return float(out[0])


def cavity_problem(n: int, Ra: float, Pr: float = 0.71, Ma: float = 0.1, phi: float = 0.0,
                   dt: float | None = None, kappa: float = 1.0, L: float | None = None):
    """Differentially heated square cavity: n x n cells on [0, L]^2 (L = n by
    default, mean width 1), hot west wall T = 1, cold east wall T = 0,
    adiabatic south/north, no-slip everywhere (Section 3.3, Fig. 3).
    dt defaults to half the smallest cell width."""
    L = float(n) if L is None else float(L)
    xf = tanh_faces(n, L, phi)
    nu, chi, bg = params_from_ra(Ra, Pr, Ma, L)
    if dt is None:
        dt = 0.5 * float(np.min(np.diff(xf)))
    return Problem(xf=xf, yf=xf.copy(), nu=nu, chi=chi, beta_g=bg, T_ref=0.5, dT=1.0,
                   dt=dt, kappa=kappa)

