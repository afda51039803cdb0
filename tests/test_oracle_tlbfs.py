"""Pins of the oracle's second face stage, the original TLBFS of Section 2.2
(Eqs. 29-43), which RTLBFS approximates -- each against something other than
its own formula:

* uniform state: the predicted variables are the state and the fluxes are
  the Euler fluxes (the equilibrium moments of Eqs. 7-8; no dissipation);
* linear fields: the predictor (moment sums, Eqs. 30-32) equals RTLBFS's
  derivative form (Eqs. 46-48), a different formula that is exact there;
* smooth fields: TLBFS and RTLBFS fluxes differ by O(h) at fixed nu, chi:
  RTLBFS keeps the first-order part of the non-equilibrium difference of
  Eqs. 33-34, and the second-order remainder, (tau - 1/2) h^2 (e.grad)^2 f / 2
  with tau - 1/2 = nu / (cs2 h), is nu h / (2 cs2) times a fourth moment;
  a wrong sign or coefficient of the first-order part (the viscous terms)
  would leave O(1);
* whole steps: mass conserved to round-off, the conduction state is a fixed
  point, the x-reflection of the heated cavity is exact;
* steady cavity at Ra = 1e3 within 1 % of the published TLBFS values.
"""
import json
import os

import numpy as np
import pytest

from helpers import CS2, centres
from paper_2202_13449_gb300 import inputs
from test_oracle_pins import lin_problem, sampled_nodes

HERE = os.path.dirname(os.path.abspath(__file__))


def tl(p):
    p.scheme = 1
    return p


@pytest.mark.parametrize("nd", [0, 1])
def test_uniform_state_gives_euler_fluxes(orc, nd):
    r, u, v, T = 1.013, 0.021, -0.017, 0.43
    nodes = np.empty((4, 3, 3))
    nodes[0], nodes[1], nodes[2], nodes[3] = r, u, v, T
    p = tl(orc.Problem(xf=np.arange(3.0), yf=np.arange(3.0), nu=0.02, chi=0.03))
    o = orc.face_from_nodes(p, nd, nodes, 0.7)
    np.testing.assert_allclose(o.pred[:], [r, r * u, r * v, r * T], rtol=0, atol=1e-15)
    un = (u, v)[nd]
    want = [r * un, r * u * un + (r * CS2 if nd == 0 else 0.0),
            r * v * un + (r * CS2 if nd == 1 else 0.0), r * un * T]
    np.testing.assert_allclose(o.flux[:], want, rtol=0, atol=1e-15)


@pytest.mark.parametrize("nd,i,j,kappa", [(0, 5, 4, 1.0), (1, 4, 5, 1.0), (0, 4, 6, 0.55),
                                          (1, 6, 3, 0.3)])
def test_predictor_equals_rtlbfs_on_linear_fields(orc, nd, i, j, kappa):
    p, st = lin_problem(orc, kappa=kappa)
    a = orc.face(p, st, nd, i, j)
    b = orc.face(tl(p), st, nd, i, j)
    np.testing.assert_allclose(b.pred[:], a.pred[:], rtol=0, atol=2e-15)


@pytest.mark.parametrize("nd", [0, 1])
def test_fluxes_first_order_close_to_rtlbfs(orc, nd):
    nu, chi = 0.02, 0.03
    hs = [0.01, 0.005, 0.0025]
    d = []
    for h in hs:
        pr = orc.Problem(xf=np.arange(3.0), yf=np.arange(3.0), nu=nu, chi=chi)
        pt = tl(orc.Problem(xf=np.arange(3.0), yf=np.arange(3.0), nu=nu, chi=chi))
        nodes = sampled_nodes(h)
        a = orc.face_from_nodes(pr, nd, nodes, h)
        b = orc.face_from_nodes(pt, nd, nodes, h)
        d.append(np.abs(np.array(b.flux[:]) - np.array(a.flux[:])))
    d = np.array(d)[:, 1:]  # the mass flux is the predicted momentum: O(h^3) apart
    orders = np.log2(d[:-1] / d[1:])
    assert np.all((orders > 0.85) & (orders < 1.3)), orders
    assert np.all(d[-1] < 1e-4 * nu), d[-1]


def cavity(orc, n=20, Ra=1e5, phi=1.5):
    p = tl(orc.cavity_problem(n, Ra, phi=phi))
    return p, inputs.conduction_state(p.xf, p.yf)


def test_tlbfs_mass_conserved(orc):
    p, _ = cavity(orc)
    st = inputs.perturbed_state(p.nx, p.ny, seed=5)
    dV = np.outer(np.diff(p.yf), np.diff(p.xf))
    m0 = float(np.sum(st[0] * dV))
    st1, _, rc = orc.step(p, st, 200)
    assert rc == 0
    assert abs(float(np.sum(st1[0] * dV)) - m0) / m0 < 1e-13


@pytest.mark.parametrize("phi", [0.0, 2.0])
def test_tlbfs_conduction_is_a_fixed_point(orc, phi):
    """Ra -> 0 (no buoyancy): rest with T linear between the walls."""
    p, st = cavity(orc, n=24, Ra=1e4, phi=phi)
    p.beta_g = 0.0
    st1, _, rc = orc.step(p, st, 20)
    assert rc == 0
    for q in range(4):
        np.testing.assert_allclose(st1[q], st[q], rtol=0, atol=2e-14)


def test_tlbfs_heated_cavity_x_reflection(orc):
    """Gravity acts along y: reflecting x (u -> -u) and swapping the wall
    temperatures maps the cavity onto itself, on an irregular mesh."""
    p = tl(orc.cavity_problem(18, 1e5, phi=0.0))
    p.xf = inputs.random_faces(18, 41, L=18.0)
    q = tl(orc.cavity_problem(18, 1e5, phi=0.0))
    q.xf = p.xf[-1] - p.xf[::-1]
    q.bc_T = (p.bc_T[1], p.bc_T[0], 0.0, 0.0)
    s = inputs.perturbed_state(18, 18, seed=17, T_mean=0.5)
    refl = lambda st: (st[0][:, ::-1], -st[1][:, ::-1], st[2][:, ::-1], st[3][:, ::-1])
    a, _, rc1 = orc.step(p, s, 40)
    b, _, rc2 = orc.step(q, refl(s), 40)
    assert rc1 == rc2 == 0
    for x, y in zip(refl(a), b):
        np.testing.assert_allclose(x, y, rtol=0, atol=2e-14)


@pytest.mark.slow
def test_tlbfs_cavity_ra1e3_against_table1(orc):
    gold = json.load(open(os.path.join(HERE, "golden", "table1_cavity_tlbfs.json")))
    n = 64
    p = tl(orc.cavity_problem(n, gold["Ra"], Pr=gold["Pr"], Ma=gold["Vc"]))
    st, steps, res, rc = orc.run_to_steady(p, inputs.conduction_state(p.xf, p.yf), 1e-8, 400000)
    assert rc == 0
    L, chi = float(n), p.chi
    assert orc.nusselt(p, st, orc.NU_A) == pytest.approx(gold["Nu_a"], rel=0.01)
    u_c = 0.5 * (st[1][:, n // 2 - 1] + st[1][:, n // 2])
    v_c = 0.5 * (st[2][n // 2 - 1, :] + st[2][n // 2, :])
    assert u_c.max() * L / chi == pytest.approx(gold["u_max_centreline_L_over_chi"], rel=0.01)
    assert v_c.max() * L / chi == pytest.approx(gold["v_max_midplane_L_over_chi"], rel=0.01)
    assert abs(centres(p.yf)[u_c.argmax()] / L - gold["u_max_y_over_L"]) < 0.02
    assert abs(centres(p.xf)[v_c.argmax()] / L - gold["v_max_x_over_L"]) < 0.02
