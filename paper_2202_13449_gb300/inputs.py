"""Seeded synthetic inputs shared by the tests, the benchmark and both sides
of every parity check.

This module draws random numbers and lays out initial fields; it holds none
of the solver's arithmetic (no fluxes, no gradients, no parameter mapping),
so the CUDA path and the CPU oracle can both consume its output without
sharing any of the method's code.

Workload recipes (the paper uses no dataset; all inputs are generated):

* ``conduction_state`` -- the cavity's initial state of Section 3.3 / 4.2:
  rho = 1, u = v = 0, T linear between the two isothermal walls.
* ``rb_state`` -- Rayleigh-Benard initial state: T linear in y plus seeded
  uniform noise of a given amplitude on every cell.
* ``batch_specs`` -- the batched-cavity workload: side lengths drawn
  uniformly from {32, 48, 64, 96, 128, 192, 256}, tanh stretching factor
  uniform in [1.0, 2.5], Ra log-uniform in [1e3, 1e6], Pr = 0.71.
* ``serving_trace`` -- request stream: Poisson arrivals, square meshes with
  side log-uniform in [64, 1024], Ra log-uniform in [1e3, 1e8], Pr in
  {0.71, 7.0}.
* ``cylinder_o_mesh`` -- the body-fitted O-mesh of Section 4.3 (vertices
  only): a circle of diameter D, far field at a given radius, first radial
  spacing fixed, geometric growth outward, theta numbered clockwise so the
  mesh is right-handed.
* ``conduction_state3`` / ``perturbed_state3`` -- the 3D counterparts
  (rho, u, v, w, T), arrays of shape (nz, ny, nx): the cubic cavity's
  initial state of Section 4.4 (T linear between the isothermal x walls) and
  a generic seeded state for parity checks.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

BATCH_SIDES = (32, 48, 64, 96, 128, 192, 256)


def rng(seed: int) -> np.random.Generator:
    """Counter-based Philox generator, the same stream on every machine."""
    return np.random.Generator(np.random.Philox(int(seed)))


def uniform_faces(n: int, L: float | None = None) -> np.ndarray:
    """n+1 equally spaced face coordinates on [0, L] (L = n: unit widths)."""
    L = float(n) if L is None else float(L)
    return np.arange(n + 1, dtype=np.float64) * (L / n)


def _centres(f: np.ndarray) -> np.ndarray:
    return 0.5 * (f[1:] + f[:-1])


def conduction_state(xf, yf, T_west: float = 1.0, T_east: float = 0.0):
    """(rho, u, v, T), each ny x nx: rest, unit density, T linear in x."""
    xf = np.asarray(xf, dtype=np.float64)
    yf = np.asarray(yf, dtype=np.float64)
    nx, ny = len(xf) - 1, len(yf) - 1
    s = (_centres(xf) - xf[0]) / (xf[-1] - xf[0])
    T = np.tile(T_west + (T_east - T_west) * s, (ny, 1))
    return (np.ones((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx)), T)


def rb_state(xf, yf, T_south: float = 1.0, T_north: float = 0.0, amp: float = 1e-3,
             seed: int = 0):
    """(rho, u, v, T): rest, unit density, T linear in y plus U(-amp, amp)."""
    xf = np.asarray(xf, dtype=np.float64)
    yf = np.asarray(yf, dtype=np.float64)
    nx, ny = len(xf) - 1, len(yf) - 1
    s = (_centres(yf) - yf[0]) / (yf[-1] - yf[0])
    T = np.tile((T_south + (T_north - T_south) * s)[:, None], (1, nx))
    T = T + rng(seed).uniform(-amp, amp, size=(ny, nx))
    return (np.ones((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx)), T)


def perturbed_state(nx: int, ny: int, seed: int, amp_rho: float = 1e-3, amp_u: float = 1e-2,
                    amp_T: float = 0.1, T_mean: float = 0.5):
    """A generic, non-symmetric state for single-step parity checks:
    rho = 1 + U(-amp_rho, amp_rho), u, v = U(-amp_u, amp_u),
    T = T_mean + U(-amp_T, amp_T)."""
    g = rng(seed)
    rho = 1.0 + g.uniform(-amp_rho, amp_rho, size=(ny, nx))
    u = g.uniform(-amp_u, amp_u, size=(ny, nx))
    v = g.uniform(-amp_u, amp_u, size=(ny, nx))
    T = T_mean + g.uniform(-amp_T, amp_T, size=(ny, nx))
    return (rho, u, v, T)


def random_faces(n: int, seed: int, L: float | None = None, spread: float = 0.5) -> np.ndarray:
    """n+1 ascending faces on [0, L] with widths 1 + U(-spread, spread),
    rescaled to span L (L = n by default): an irregular non-uniform mesh."""
    L = float(n) if L is None else float(L)
    w = 1.0 + rng(seed).uniform(-spread, spread, size=n)
    f = np.concatenate([[0.0], np.cumsum(w)])
    return f * (L / f[-1])


@dataclass
class CavitySpec:
    n: int          # cells per side
    phi: float      # tanh stretching factor (Eq. 74)
    Ra: float
    Pr: float


def batch_specs(count: int = 1024, seed: int = 1234, sides=BATCH_SIDES,
                phi_range=(1.0, 2.5), log_ra=(3.0, 6.0), Pr: float = 0.71):
    """Independent cavities of uneven size for the batched launch."""
    g = rng(seed)
    n = g.choice(np.asarray(sides), size=count)
    phi = g.uniform(phi_range[0], phi_range[1], size=count)
    Ra = 10.0 ** g.uniform(log_ra[0], log_ra[1], size=count)
    return [CavitySpec(int(n[k]), float(phi[k]), float(Ra[k]), float(Pr)) for k in range(count)]


@dataclass
class Request:
    t_arrive: float  # seconds after trace start
    n: int
    Ra: float
    Pr: float


def serving_trace(count: int = 10000, seed: int = 42, rate: float = 200.0,
                  n_range=(64, 1024), log_ra=(3.0, 8.0), prs=(0.71, 7.0)):
    """Poisson arrivals at ``rate`` per second; square uniform meshes."""
    g = rng(seed)
    gaps = g.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps)
    lo, hi = np.log10(n_range[0]), np.log10(n_range[1])
    n = np.rint(10.0 ** g.uniform(lo, hi, size=count)).astype(int)
    Ra = 10.0 ** g.uniform(log_ra[0], log_ra[1], size=count)
    Pr = np.where(g.uniform(size=count) < 0.5, prs[0], prs[1])
    return [Request(float(t[k]), int(n[k]), float(Ra[k]), float(Pr[k])) for k in range(count)]


def conduction_state3(xf, yf, zf, T_west: float = 0.0, T_east: float = 1.0):
    """(rho, u, v, w, T), each nz x ny x nx: rest, unit density, T linear in x
    (cold -x wall, hot +x wall by default, as in the cubic cavity)."""
    xf = np.asarray(xf, dtype=np.float64)
    nx, ny, nz = len(xf) - 1, len(yf) - 1, len(zf) - 1
    s = (_centres(xf) - xf[0]) / (xf[-1] - xf[0])
    T = np.broadcast_to(T_west + (T_east - T_west) * s, (nz, ny, nx)).copy()
    z = np.zeros((nz, ny, nx))
    return (np.ones((nz, ny, nx)), z, z.copy(), z.copy(), T)


def perturbed_state3(nx: int, ny: int, nz: int, seed: int, amp_rho: float = 1e-3,
                     amp_u: float = 1e-2, amp_T: float = 0.1, T_mean: float = 0.5):
    """3D generic state: rho = 1 + U(-amp_rho, amp_rho), u, v, w =
    U(-amp_u, amp_u), T = T_mean + U(-amp_T, amp_T), shape (nz, ny, nx)."""
    g = rng(seed)
    sh = (nz, ny, nx)
    rho = 1.0 + g.uniform(-amp_rho, amp_rho, size=sh)
    u = g.uniform(-amp_u, amp_u, size=sh)
    v = g.uniform(-amp_u, amp_u, size=sh)
    w = g.uniform(-amp_u, amp_u, size=sh)
    T = T_mean + g.uniform(-amp_T, amp_T, size=sh)
    return (rho, u, v, w, T)


def cylinder_o_mesh(ni: int, nj: int, D: float = 1.0, r_far: float = 52.5, first: float = 0.003):
    """Vertices (X, Y), shape (nj+1, ni+1), of an O-mesh around a circle of
    diameter D: radii from D/2 to r_far * D with the first spacing
    first * D and a constant growth ratio (solved by bisection); theta
    decreasing with i so i, j are right-handed; column ni repeats column 0."""
    r0, r1, d0 = 0.5 * D, r_far * D, first * D
    lo, hi = 1.0 + 1e-12, 2.0
    for _ in range(200):
        q = 0.5 * (lo + hi)
        try:
            total = d0 * (q ** nj - 1.0) / (q - 1.0)
        except OverflowError:  # q ** nj beyond the double range: far too long
            total = float("inf")
        if total > r1 - r0:
            hi = q
        else:
            lo = q
    q = 0.5 * (lo + hi)
    r = r0 + d0 * (q ** np.arange(nj + 1) - 1.0) / (q - 1.0)
    r[-1] = r1
    th = -2.0 * np.pi * np.arange(ni + 1) / ni
    X = np.outer(r, np.cos(th))
    Y = np.outer(r, np.sin(th))
    X[:, -1], Y[:, -1] = X[:, 0], Y[:, 0]
    return X, Y
