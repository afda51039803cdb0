"""Whole-step pins of the FP64 oracle: closed forms, invariants and symmetries
that hold for the exact method regardless of how it is coded.

* Ra -> 0 conduction: rest + linear T is a discrete fixed point (uniform and
  stretched meshes).
* Conservation: total mass to round-off (walls and periodic sides); total
  rho*T with all walls adiabatic.
* Symmetries: x-reflection of the heated cavity (gravity along y); x-reflection
  and x<->y transposition without gravity, on irregular meshes.
* Momentum: plane Couette is a fixed point; Poiseuille converges to the
  parabola at second order; the Taylor-Green vortex decays as
  exp(-2 nu k^2 t).
* Energy: the Gaussian hill of Section 4.1 (Eqs. 66-68) against its closed
  form, second-order convergence of E_2 (Fig. 7's claim).
* Nusselt normalisation: on the conduction state every Nusselt number is 1
  on square cavities (uniform and tanh meshes, L, dT, chi away from 1), the
  sign follows the heat flow, and a rectangle's wall numbers count the wall
  length.
* Steady cavity: energy balance Nu_hot = Nu_cold = Nu_1/2, wall number equal
  to Eq. 69's Nu_a to the truncation error, Table 1 at Ra = 1e3 and 1e4.
"""
import json
import os

import numpy as np
import pytest

from helpers import centres
from paper_2202_13449_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


def total(p, a):
    dV = np.outer(np.diff(p.yf), np.diff(p.xf))
    return float(np.sum(a * dV))


# ---------------------------------------------------------------- conduction
@pytest.mark.parametrize("phi", [0.0, 2.0])
def test_conduction_profile_is_a_fixed_point(orc, phi):
    p = orc.cavity_problem(24, 1e4, phi=phi)
    p.beta_g = 0.0  # Ra -> 0: no buoyancy
    st = inputs.conduction_state(p.xf, p.yf)
    st2, res, rc = orc.step(p, st, 20)
    assert rc == 0
    for q in range(4):
        np.testing.assert_allclose(st2[q], st[q], rtol=0, atol=2e-14)


def test_hot_fluid_rises(orc):
    """Buoyancy direction: from rest with the hot wall on the west, the fluid
    next to the hot wall starts to move up (+y) and next to the cold wall down."""
    p = orc.cavity_problem(16, 1e5)
    st, _, rc = orc.step(p, inputs.conduction_state(p.xf, p.yf), 5)
    assert rc == 0
    v = st[2]
    assert v[4:12, :3].min() > 0.0 and v[4:12, -3:].max() < 0.0


# ---------------------------------------------------------------- conservation
def test_mass_conserved_in_heated_cavity(orc):
    p = orc.cavity_problem(20, 1e5, phi=1.5)
    p.yf = inputs.random_faces(17, 4, L=20.0)
    st = inputs.conduction_state(p.xf, p.yf)
    st = (st[0] + 1e-3 * inputs.perturbed_state(20, 17, seed=9)[1], st[1], st[2], st[3])
    m0 = total(p, st[0])
    st2, _, rc = orc.step(p, st, 200)
    assert rc == 0
    assert abs(total(p, st2[0]) - m0) / m0 < 1e-14


def test_mass_and_energy_conserved_periodic_and_adiabatic(orc):
    P, A = orc.PERIODIC, orc.ADIABATIC
    xf = inputs.random_faces(16, 1)
    yf = inputs.random_faces(12, 2)
    p = orc.Problem(xf=xf, yf=yf, nu=0.05, chi=0.07, beta_g=2e-4, dt=0.3, kappa=0.8,
                    bc_kind=(P, P, A, A))
    st = inputs.perturbed_state(16, 12, seed=3)
    m0, e0 = total(p, st[0]), total(p, st[0] * st[3])
    st2, _, rc = orc.step(p, st, 150)
    assert rc == 0
    assert abs(total(p, st2[0]) - m0) / m0 < 1e-14
    assert abs(total(p, st2[0] * st2[3]) - e0) / e0 < 1e-13


# ---------------------------------------------------------------- symmetries
def test_heated_cavity_x_reflection_with_gravity(orc):
    """Gravity acts along y, so reflecting x (u -> -u) and swapping the two
    wall temperatures maps the cavity onto itself.  (Shifting T by a constant
    is not an exact symmetry: the energy equation acts on rho*T, and Eq. 57
    transports rho with the predicted flux while Eq. 59 uses the time-n one.)"""
    p = orc.cavity_problem(18, 1e5, phi=0.0)
    p.xf = inputs.random_faces(18, 41, L=18.0)
    q = orc.cavity_problem(18, 1e5, phi=0.0)
    q.xf = p.xf[-1] - p.xf[::-1]
    q.bc_T = (p.bc_T[1], p.bc_T[0], 0.0, 0.0)
    s = inputs.perturbed_state(18, 18, seed=17, T_mean=0.5)
    refl = lambda st: (st[0][:, ::-1], -st[1][:, ::-1], st[2][:, ::-1], st[3][:, ::-1])
    a, _, rc1 = orc.step(p, s, 40)
    b, _, rc2 = orc.step(q, refl(s), 40)
    assert rc1 == rc2 == 0
    for x, y in zip(refl(a), b):
        np.testing.assert_allclose(x, y, rtol=0, atol=2e-14)


def test_x_reflection_without_gravity(orc):
    D, A = orc.DIRICHLET, orc.ADIABATIC
    xf = inputs.random_faces(13, 5)
    yf = inputs.random_faces(9, 6)
    common = dict(nu=0.04, chi=0.06, beta_g=0.0, dt=0.3, kappa=0.9)
    pa = orc.Problem(xf=xf, yf=yf, bc_kind=(D, A, A, D), bc_T=(0.8, 0.0, 0.0, 0.3),
                     bc_u=(0.01, 0.0, 0.0, 0.02), **common)
    xr = xf[-1] - xf[::-1]
    # the west wall's tangential velocity is v (kept); the lid's is u (negated)
    pb = orc.Problem(xf=xr, yf=yf, bc_kind=(A, D, A, D), bc_T=(0.0, 0.8, 0.0, 0.3),
                     bc_u=(0.0, 0.01, 0.0, -0.02), **common)
    s = inputs.perturbed_state(13, 9, seed=8)
    refl = lambda st: (st[0][:, ::-1], -st[1][:, ::-1], st[2][:, ::-1], st[3][:, ::-1])
    a, _, rc1 = orc.step(pa, s, 25)
    b, _, rc2 = orc.step(pb, refl(s), 25)
    assert rc1 == rc2 == 0
    for x, y in zip(refl(a), b):
        np.testing.assert_allclose(x, y, rtol=0, atol=2e-14)


def test_transpose_without_gravity(orc):
    D, A, P = orc.DIRICHLET, orc.ADIABATIC, orc.PERIODIC
    xf = inputs.random_faces(11, 7)
    yf = inputs.random_faces(14, 8)
    common = dict(nu=0.04, chi=0.03, beta_g=0.0, dt=0.3, kappa=0.7)
    pa = orc.Problem(xf=xf, yf=yf, bc_kind=(P, P, D, A), bc_T=(0, 0, 0.9, 0.0),
                     bc_u=(0, 0, 0.01, 0.0), **common)
    pb = orc.Problem(xf=yf, yf=xf, bc_kind=(D, A, P, P), bc_T=(0.9, 0.0, 0, 0),
                     bc_u=(0.01, 0.0, 0, 0), **common)
    s = inputs.perturbed_state(11, 14, seed=9)
    tr = lambda st: (st[0].T.copy(), st[2].T.copy(), st[1].T.copy(), st[3].T.copy())
    a, _, rc1 = orc.step(pa, s, 25)
    b, _, rc2 = orc.step(pb, tr(s), 25)
    assert rc1 == rc2 == 0
    for x, y in zip(tr(a), b):
        np.testing.assert_allclose(x, y, rtol=0, atol=2e-14)


# ---------------------------------------------------------------- momentum
def channel(orc, n, nu, dt, U_top=0.0, fx=0.0, kappa=1.0):
    P, A = orc.PERIODIC, orc.ADIABATIC
    yf = inputs.uniform_faces(n, 1.0)
    xf = inputs.uniform_faces(4, 4.0 / n)
    return orc.Problem(xf=xf, yf=yf, nu=nu, chi=nu, beta_g=0.0, dt=dt, kappa=kappa, fx=fx,
                       bc_kind=(P, P, A, A), bc_u=(0, 0, 0, U_top))


def test_couette_profile_is_a_fixed_point_and_attracts(orc):
    n, U = 12, 0.02
    p = channel(orc, n, nu=0.05, dt=0.5 / n ** 2 / 0.05 * 0.2, U_top=U)
    yc = centres(p.yf)
    lin = np.tile((U * yc)[:, None], (1, 4))
    st = (np.ones((n, 4)), lin, np.zeros((n, 4)), np.full((n, 4), 0.5))
    st2, _, rc = orc.step(p, st, 50)
    assert rc == 0
    np.testing.assert_allclose(st2[1], lin, rtol=0, atol=1e-16)
    np.testing.assert_allclose(st2[0], 1.0, rtol=0, atol=1e-15)
    rest = (np.ones((n, 4)), np.zeros((n, 4)), np.zeros((n, 4)), np.full((n, 4), 0.5))
    st3, steps, _, rc = orc.run_to_steady(p, rest, 1e-13, 200000)
    assert rc == 0
    np.testing.assert_allclose(st3[1], lin, rtol=0, atol=1e-10 * U / 1e-3)


def test_poiseuille_converges_at_second_order(orc):
    nu, umax = 0.1, 0.01
    fx = 8 * nu * umax  # H = 1
    errs = []
    for n in (8, 16, 32):
        dx = 1.0 / n
        dt = min(0.2 * dx * dx / nu, 0.4 * dx)
        p = channel(orc, n, nu=nu, dt=dt, fx=fx)
        rest = (np.ones((n, 4)), np.zeros((n, 4)), np.zeros((n, 4)), np.full((n, 4), 0.5))
        st, steps, _, rc = orc.run_to_steady(p, rest, 1e-12, 2000000)
        assert rc == 0
        yc = centres(p.yf)
        exact = fx / (2 * nu) * yc * (1.0 - yc)
        errs.append(np.max(np.abs(st[1][:, 0] - exact)) / umax)
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 1e-2
    assert np.all(order > 1.8), (errs, order)


def taylor_green(orc, n, nu=0.02, U=0.01, steps=400, dt=0.5):
    P = orc.PERIODIC
    xf = inputs.uniform_faces(n)
    p = orc.Problem(xf=xf, yf=xf.copy(), nu=nu, chi=nu, beta_g=0.0, dt=dt, kappa=1.0,
                    bc_kind=(P, P, P, P))
    k = 2 * np.pi / n
    X, Y = np.meshgrid(centres(xf), centres(xf))
    u = -U * np.cos(k * X) * np.sin(k * Y)
    v = U * np.sin(k * X) * np.cos(k * Y)
    rho = 1.0 - (U * U / 4) * (np.cos(2 * k * X) + np.cos(2 * k * Y)) * 3.0
    st, _, rc = orc.step(p, (rho, u, v, np.full((n, n), 0.5)), steps)
    assert rc == 0
    mode = np.sin(k * X) * np.cos(k * Y)
    A = np.sum(st[2] * mode) / np.sum(mode * mode)
    rate = -np.log(A / U) / (steps * dt)
    return rate, 2 * nu * k * k


def test_taylor_green_decay_rate(orc):
    errs = []
    for n in (16, 32, 64):
        rate, exact = taylor_green(orc, n, steps=int(0.15 * n * n))
        errs.append(abs(rate - exact) / exact)
    assert errs[-1] < 0.012, errs
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(order > 1.8), (errs, order)


# ---------------------------------------------------------------- energy (Section 4.1)
def gaussian_hill(orc, n, Pe, Fo=0.005, Fo_dx=0.1, dt=1.0, ddt=0.5):
    """Domain [0, 2L]^2 with L = n cells of width 1, periodic, u = (u0, 0);
    chi from Fo_dx = dt chi / dx^2; u0 from Pe = u0 L / chi; end at
    Fo = t chi / L^2; returns E_2 of Eq. 68 against Eq. 67 and the peak."""
    P = orc.PERIODIC
    L = float(n)
    chi = Fo_dx / dt
    u0 = Pe * chi / L
    xf = inputs.uniform_faces(2 * n)
    p = orc.Problem(xf=xf, yf=xf.copy(), nu=chi, chi=chi, beta_g=0.0, dt=dt, kappa=ddt,
                    bc_kind=(P, P, P, P))
    sigma = 0.05 * L
    x0 = np.array([0.5 * L, 0.0])
    X, Y = np.meshgrid(centres(xf), centres(xf))

    def exact(t):
        s2 = 2 * chi * t + sigma ** 2
        T0 = 2 * np.pi * sigma ** 2
        out = np.zeros_like(X)
        for sx in (-2 * L, 0.0, 2 * L):
            for sy in (-2 * L, 0.0, 2 * L):
                d2 = (X - x0[0] - u0 * t - sx) ** 2 + (Y - x0[1] - sy) ** 2
                out += T0 / (2 * np.pi * s2) * np.exp(-d2 / (2 * s2))
        return out

    nsteps = int(round(Fo * L * L / chi / dt))
    st0 = (np.ones_like(X), np.full_like(X, u0), np.zeros_like(X), exact(0.0))
    st, _, rc = orc.step(p, st0, nsteps)
    assert rc == 0
    Ta = exact(nsteps * dt)
    return float(np.sqrt(np.mean((st[3] - Ta) ** 2))), float(Ta.max()), st


def test_gaussian_hill_fig6_setting_matches_closed_form(orc):
    e2, peak, st = gaussian_hill(orc, 50, Pe=100)
    # momentum stays uniform (no force acts on it)
    np.testing.assert_allclose(st[1], st[1][0, 0], rtol=0, atol=1e-15)
    assert e2 / peak < 0.01, (e2, peak)


@pytest.mark.slow
def test_gaussian_hill_second_order(orc):
    errs = [gaussian_hill(orc, n, Pe=10)[0] for n in (40, 80, 120)]
    o1 = np.log(errs[0] / errs[1]) / np.log(2.0)
    o2 = np.log(errs[1] / errs[2]) / np.log(1.5)
    assert o1 > 1.8 and o2 > 1.8, (errs, o1, o2)


# ---------------------------------------------------------------- Nusselt normalisation
def _conduction_x(orc, xf, yf, T_h, T_c, chi):
    """Ra -> 0 cavity: hot west wall T_h, cold east wall T_c, adiabatic south
    and north, at rest with T linear in x (a discrete fixed point, pinned
    above)."""
    p = orc.Problem(xf=xf, yf=yf, nu=0.05, chi=chi, beta_g=0.0, T_ref=0.5 * (T_h + T_c),
                    dT=abs(T_h - T_c), bc_T=(T_h, T_c, 0.0, 0.0))
    return p, inputs.conduction_state(xf, yf, T_west=T_h, T_east=T_c)


@pytest.mark.parametrize("phi", [0.0, 1.7])
def test_conduction_nusselt_numbers_are_one(orc, phi):
    """The Nusselt normalisation against the mathematics of pure conduction.
    A square cavity of side L with the walls at T_h and T_c conducts the heat
    flux chi (T_h - T_c) / L through every vertical line, so the heat through
    a wall, per chi dT, is exactly 1; so is Eq. 69's Nu_a (u = 0, dT/dx =
    -dT / L, integrated over L^2 and divided by chi dT L).  L = 37, dT = 2.5
    and chi = 0.037 are all away from 1, and the tanh meshes (Eq. 74) give
    unequal face areas, so a missing face-area weight, chi or dT fails."""
    L, n = 37.0, 20
    xf = orc.tanh_faces(n, L, phi)
    yf = orc.tanh_faces(n + 6, L, phi)
    p, st = _conduction_x(orc, xf, yf, 3.25, 0.75, 0.037)
    for which in (orc.NU_W, orc.NU_E, orc.NU_HALF, orc.NU_A):
        assert orc.nusselt(p, st, which) == pytest.approx(1.0, rel=1e-13), which
    # no heat crosses the adiabatic walls
    assert orc.nusselt(p, st, orc.NU_S) == 0.0 and orc.nusselt(p, st, orc.NU_N) == 0.0
    # sign: the numbers are heat flow along +x; with the hot wall on the east
    # the heat flows towards -x
    p2, st2 = _conduction_x(orc, xf, yf, 0.75, 3.25, 0.037)
    for which in (orc.NU_W, orc.NU_E, orc.NU_HALF, orc.NU_A):
        assert orc.nusselt(p2, st2, which) == pytest.approx(-1.0, rel=1e-13), which


def test_conduction_nusselt_of_a_rectangle_counts_the_wall_length(orc):
    """On an Lx x Ly rectangle the conducted heat through a vertical wall is
    chi dT Ly / Lx: the wall numbers are the whole wall's heat per chi dT
    (Ly / Lx here), and Eq. 69 divided by Lx gives the same; heated from
    below (Rayleigh-Benard walls, periodic in x) the bottom and top walls
    carry chi dT Lx / Ly."""
    xf = inputs.random_faces(14, 41, L=37.0)
    yf = inputs.random_faces(9, 42, L=23.0)
    p, st = _conduction_x(orc, xf, yf, 1.0, 0.0, 0.21)
    for which in (orc.NU_W, orc.NU_E, orc.NU_HALF, orc.NU_A):
        assert orc.nusselt(p, st, which) == pytest.approx(23.0 / 37.0, rel=1e-13), which
    rb = orc.Problem(xf=xf, yf=yf, nu=0.05, chi=0.21, beta_g=0.0, T_ref=1.5, dT=2.0,
                     bc_kind=(orc.PERIODIC, orc.PERIODIC, orc.DIRICHLET, orc.DIRICHLET),
                     bc_T=(0.0, 0.0, 2.5, 0.5))
    st_rb = inputs.rb_state(xf, yf, T_south=2.5, T_north=0.5, amp=0.0)
    _, res, rc = orc.step(rb, st_rb, 3)  # the profile is a fixed point here too
    assert rc == 0 and res[1] < 1e-14
    for which in (orc.NU_S, orc.NU_N):
        assert orc.nusselt(rb, st_rb, which) == pytest.approx(37.0 / 23.0, rel=1e-13), which


# ---------------------------------------------------------------- steady cavity
def test_steady_cavity_energy_balance(orc):
    p = orc.cavity_problem(24, 1e4, phi=1.0)
    st0 = inputs.conduction_state(p.xf, p.yf)
    st, steps, res, rc = orc.run_to_steady(p, st0, 1e-10, 400000)
    assert rc == 0
    nw, ne, nh = (orc.nusselt(p, st, w) for w in (orc.NU_W, orc.NU_E, orc.NU_HALF))
    assert ne == pytest.approx(nw, rel=1e-6)
    assert nh == pytest.approx(nw, rel=1e-6)
    fx, _ = orc.fluxes(p, st)
    cols = (fx[3] * np.diff(p.yf)[:, None]).sum(axis=0) / p.chi
    np.testing.assert_allclose(cols, nw, rtol=1e-6)
    # no heat leaves through the adiabatic walls
    assert orc.nusselt(p, st, orc.NU_S) == 0.0 and orc.nusselt(p, st, orc.NU_N) == 0.0
    # the wall number and Eq. 69's volume integral are two discretisations of
    # the same steady heat transport: they agree to the mesh's truncation
    # error, and both are within 1 % of Table 1's Nu_a at Ra = 1e4
    gold = json.load(open(os.path.join(HERE, "golden", "table1_nu_a.json")))["Nu_a"]["1e4"]
    na = orc.nusselt(p, st, orc.NU_A)
    assert abs(nw - na) < 2e-3 * na, (nw, na)
    assert nw == pytest.approx(gold, rel=0.01)
    assert na == pytest.approx(gold, rel=0.01)


@pytest.mark.slow
def test_cavity_ra1e3_against_table1(orc):
    gold = json.load(open(os.path.join(HERE, "golden", "table1_cavity.json")))
    n = 64
    p = orc.cavity_problem(n, gold["Ra"], Pr=gold["Pr"], Ma=gold["Vc"])
    st, steps, res, rc = orc.run_to_steady(p, inputs.conduction_state(p.xf, p.yf), 1e-8, 400000)
    assert rc == 0
    L, chi = float(n), p.chi
    nu_a = orc.nusselt(p, st, orc.NU_A)
    assert nu_a == pytest.approx(gold["Nu_a"], rel=0.01)
    # u along x = L/2 (mean of the two centre columns), v along y = L/2
    u_c = 0.5 * (st[1][:, n // 2 - 1] + st[1][:, n // 2])
    v_c = 0.5 * (st[2][n // 2 - 1, :] + st[2][n // 2, :])
    yc = centres(p.yf) / L
    xc = centres(p.xf) / L
    assert u_c.max() * L / chi == pytest.approx(gold["u_max_centreline_L_over_chi"], rel=0.01)
    assert v_c.max() * L / chi == pytest.approx(gold["v_max_midplane_L_over_chi"], rel=0.01)
    # hot fluid rises: the flow leaves the hot wall along the top
    assert abs(yc[u_c.argmax()] - gold["u_max_y_over_L"]) < 0.02
    assert abs(xc[v_c.argmax()] - gold["v_max_x_over_L"]) < 0.02


def test_non_finite_state_is_divergence(orc):
    """A state that is no longer a number has no residual: the run stops as
    diverged on that step (the convergence test of Section 3.3, Eq. 65,
    needs finite sums)."""
    p = orc.cavity_problem(12, 1e3)
    st = list(inputs.conduction_state(p.xf, p.yf))
    st[1] = st[1].copy()
    st[1][5, 5] = np.nan
    _, steps, res, rc = orc.run_to_steady(p, st, 1e-9, 100)
    assert rc == -4 and steps == 1 and np.isnan(res[0])
    _, _, rc = orc.step(p, st, 3)
    assert rc == -4


def test_small_lattice_spacing_diverges(orc):
    """Section 3.3 (Fig. 4): the terms scaled by the lattice spacing delta t
    are the numerical dissipation; with delta t small they are too weak and
    the heated cavity diverges, with delta t of the cell size it does not
    (20 x 20 unit cells, Ra = 1e6, Pr = 0.71, V_c = 0.1, Delta t = 0.5)."""
    out = {}
    for kappa in (0.1, 0.5, 1.0):
        p = orc.cavity_problem(20, 1e6)
        p.kappa = kappa
        _, steps, _, rc = orc.run_to_steady(p, inputs.conduction_state(p.xf, p.yf), 1e-12, 2000)
        out[kappa] = (rc, steps)
    assert out[0.1][0] == -4 and out[0.1][1] < 2000
    assert out[0.5][0] == -5 and out[1.0][0] == -5
