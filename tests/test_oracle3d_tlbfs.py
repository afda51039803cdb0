"""Pins of the 3D oracle's second face stage, the original TLBFS of Section
2.2 with D3Q19 (Eqs. 29-43), each against something other than its own
formula:

* uniform state: the predicted variables are the state and the fluxes are
  the Euler fluxes (the equilibrium moments of Eqs. 7-8);
* linear fields: the moment-sum predictor (Eqs. 30-32) equals RTLBFS's
  derivative form (Eqs. 46-48), exact there for both;
* smooth fields: the TLBFS and RTLBFS fluxes differ by O(h) at fixed nu, chi
  (the second-order remainder of the non-equilibrium difference of Eqs.
  33-34 times tau - 1/2 = nu / (cs2 h)); wrong viscous terms leave O(1);
* a state invariant along a periodic axis evolves as the 2D oracle's TLBFS
  stage does in the other two axes;
* whole steps: mass conserved, the conduction state a fixed point, the
  x-reflection of the heated cavity exact.
"""
import numpy as np
import pytest

from helpers import CS2, E_D3Q19
from paper_2202_13449_gb300 import inputs
from test_oracle3d import FACES, lin_problem, sampled_nodes, _embed


@pytest.fixture(scope="module")
def d3(orc):
    from oracle import d3 as mod
    return mod


def tl(p):
    p.scheme = 1
    return p


def unit_problem(d3, **kw):
    return d3.Problem3(xf=np.arange(3.0), yf=np.arange(3.0), zf=np.arange(3.0), **kw)


@pytest.mark.parametrize("nd", [0, 1, 2])
def test_uniform_state_gives_euler_fluxes(d3, nd):
    r, u, T = 1.013, np.array([0.021, -0.017, 0.012]), 0.43
    nodes = np.empty((5, 19))
    nodes[0], nodes[1], nodes[2], nodes[3], nodes[4] = r, u[0], u[1], u[2], T
    o = d3.face_from_nodes(tl(unit_problem(d3, nu=0.02, chi=0.03)), nd, nodes, 0.7)
    np.testing.assert_allclose(o.pred[:], [r, *(r * u), r * T], rtol=0, atol=1e-15)
    want = [r * u[nd]] + [r * u[a] * u[nd] + (r * CS2 if a == nd else 0.0) for a in range(3)]
    want += [r * u[nd] * T]
    np.testing.assert_allclose(o.flux[:], want, rtol=0, atol=1e-15)


@pytest.mark.parametrize("nd,c,kappa", FACES)
def test_predictor_equals_rtlbfs_on_linear_fields(d3, nd, c, kappa):
    p, st = lin_problem(d3, kappa=kappa)
    a = d3.face(p, st, nd, *c)
    b = d3.face(tl(p), st, nd, *c)
    np.testing.assert_allclose(b.pred[:], a.pred[:], rtol=0, atol=2e-15)


@pytest.mark.parametrize("nd", [0, 1, 2])
def test_fluxes_first_order_close_to_rtlbfs(d3, nd):
    nu, chi = 0.02, 0.03
    d = []
    for h in (0.01, 0.005, 0.0025):
        nodes = sampled_nodes(h)
        a = d3.face_from_nodes(unit_problem(d3, nu=nu, chi=chi), nd, nodes, h)
        b = d3.face_from_nodes(tl(unit_problem(d3, nu=nu, chi=chi)), nd, nodes, h)
        d.append(np.abs(np.array(b.flux[:]) - np.array(a.flux[:])))
    d = np.array(d)[:, 1:]  # the mass flux is the predicted momentum: O(h^3) apart
    orders = np.log2(d[:-1] / d[1:])
    assert np.all((orders > 0.85) & (orders < 1.3)), orders
    # O(nu h): at h = 0.0025 a dropped or wrong viscous term would leave O(nu)
    assert np.all(d[-1] < nu * 0.0025), d[-1]


def test_invariant_direction_reduces_to_the_2d_tlbfs_stage(orc, d3):
    D, A, Pe = orc.DIRICHLET, orc.ADIABATIC, orc.PERIODIC
    nx2, ny2, nP = 9, 7, 3
    f2x, f2y = inputs.random_faces(nx2, 15), inputs.random_faces(ny2, 16)
    p2 = orc.Problem(xf=f2x, yf=f2y, nu=0.03, chi=0.04, beta_g=2e-3, kappa=0.9, dt=0.2,
                     bc_kind=(D, A, A, D), bc_T=(0.9, 0.1, 0.3, 0.6),
                     bc_u=(0.01, 0.0, 0.0, 0.02), scheme=1)
    # 3D: x <- 2D x, z <- 2D y, y periodic and invariant
    bcu = ((0, 0, 0.01), (0, 0, 0), (0, 0, 0), (0, 0, 0), (0, 0, 0), (0.02, 0, 0))
    p3 = d3.Problem3(xf=f2x, yf=np.arange(nP + 1.0), zf=f2y, nu=0.03, chi=0.04, beta_g=2e-3,
                     kappa=0.9, dt=0.2, g_axis=2, bc_kind=(D, A, Pe, Pe, A, D),
                     bc_T=(0.9, 0.1, 0, 0, 0.3, 0.6), bc_u=bcu, scheme=1)
    rho2, u2, v2, T2 = inputs.perturbed_state(nx2, ny2, seed=8)
    emb = lambda a: _embed(a, 0, 2, 1, nP)
    st3 = [emb(rho2), emb(u2), emb(np.zeros_like(u2)), emb(v2), emb(T2)]
    s2, _, rc2 = orc.step(p2, (rho2, u2, v2, T2), 5)
    s3, _, rc3 = d3.step(p3, st3, 5)
    assert rc2 == 0 and rc3 == 0
    want = [s2[0], s2[1], np.zeros_like(s2[1]), s2[2], s2[3]]
    for q in range(5):
        np.testing.assert_allclose(s3[q], emb(want[q]), rtol=0, atol=2e-15)


def test_tlbfs_mass_conserved_and_conduction_fixed(d3):
    p = tl(d3.cubic_cavity(8, 1e5, phi=1.5))
    st = inputs.perturbed_state3(8, 8, 8, seed=6)
    dV = np.einsum("k,j,i->kji", np.diff(p.zf), np.diff(p.yf), np.diff(p.xf))
    m0 = float(np.sum(st[0] * dV))
    s1, _, rc = d3.step(p, st, 60)
    assert rc == 0
    assert abs(float(np.sum(s1[0] * dV)) - m0) / m0 < 1e-13
    p.beta_g = 0.0
    c = inputs.conduction_state3(p.xf, p.yf, p.zf)
    c1, _, rc = d3.step(p, c, 20)
    assert rc == 0
    for q in range(5):
        np.testing.assert_allclose(c1[q], c[q], rtol=0, atol=2e-14)


def test_tlbfs_x_reflection_with_gravity(d3):
    n = (7, 6, 8)
    f = [inputs.random_faces(n[a], 51 + a) for a in range(3)]
    D, A = 0, 1
    p = tl(d3.Problem3(xf=f[0], yf=f[1], zf=f[2], nu=0.03, chi=0.04, beta_g=3e-3, kappa=0.9,
                       dt=0.2, bc_kind=(D, D, A, A, A, A), bc_T=(0.8, 0.2, 0, 0, 0, 0)))
    q = tl(d3.Problem3(xf=(f[0][-1] - f[0])[::-1].copy(), yf=f[1], zf=f[2], nu=0.03, chi=0.04,
                       beta_g=3e-3, kappa=0.9, dt=0.2, bc_kind=(D, D, A, A, A, A),
                       bc_T=(0.2, 0.8, 0, 0, 0, 0)))
    st = inputs.perturbed_state3(*n, seed=3)
    fl = lambda a: np.ascontiguousarray(a[..., ::-1])
    refl = lambda s: (fl(s[0]), -fl(s[1]), fl(s[2]), fl(s[3]), fl(s[4]))
    a, _, rc1 = d3.step(p, st, 4)
    b, _, rc2 = d3.step(q, refl(st), 4)
    assert rc1 == rc2 == 0
    for x, y in zip(refl(a), b):
        np.testing.assert_allclose(x, y, rtol=0, atol=1e-15)
