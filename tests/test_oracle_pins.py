"""Pins of the FP64 oracle's building blocks against what the paper and the
mathematics fix independently of the oracle's own formulas.

* Eq. 74 mesh: end points, symmetry, wall spacing from the derivative.
* Eq. 63: the mapped (nu, chi, beta_g) reproduce Ra, Pr and V_c.
* Eqs. 55-56: Green-Gauss with inverse-distance face values is exact for
  linear fields on any rectilinear mesh and reduces to the central
  difference on a uniform one.
* Eq. 29: every lattice node takes the plane of the cell it lies in.
* Eqs. 46-48 (predictor): for constant rho and linear u, v, T the
  equilibria are quadratic in space, so the second-order Taylor form is
  exact and must equal the D2Q9 moment sums of Eqs. 30-32 -- a different
  formula (distribution functions of Eqs. 3-6) for the same quantity.
* Eqs. 57-59 (flux braces): equal to the distribution-function form of
  Eqs. 39-40 with f_eq(x_S - e dt) replaced by its first-order Taylor
  expansion (the step from Eq. 39 to Eq. 50), again exact for quadratic
  equilibria, again computed from Eqs. 3-6 only.
* On smooth non-polynomial node data the predictor stays O(h^3) and the
  fluxes O(h^2) from those distribution-function forms (the orders the
  Taylor steps of Eqs. 44-51 leave), which catches any wrong second-order
  coefficient that the quadratic case cannot see.
* Boundary readings: zero mass flux through walls, zero energy flux through
  adiabatic walls, wall values at node (0,0).
"""
import numpy as np
import pytest

from helpers import CS2, E_D2Q9, centres, f_eq, g_eq
from paper_2202_13449_gb300 import inputs


# ---------------------------------------------------------------- Eq. 74
def test_tanh_faces_endpoints_symmetry_and_wall_spacing(orc):
    n, L, phi = 512, 512.0, 2.0
    xf = orc.tanh_faces(n, L, phi)
    assert xf[0] == pytest.approx(0.0, abs=1e-12)
    assert xf[-1] == pytest.approx(L, rel=1e-14)
    assert np.all(np.diff(xf) > 0)
    np.testing.assert_allclose(xf + xf[::-1], L, rtol=0, atol=1e-11)
    # first cell ~ dx/di at i = 0: L phi (1 - tanh^2 phi) / (M tanh phi)
    d0 = L * phi * (1 - np.tanh(phi) ** 2) / (n * np.tanh(phi))
    assert (xf[1] - xf[0]) == pytest.approx(d0, rel=0.01)
    # wall cell is the smallest, centre cell the largest
    w = np.diff(xf)
    assert w.argmin() in (0, n - 1) and abs(w.argmax() - n / 2) <= 1
    # phi -> 0 tends to the uniform mesh; phi <= 0 is exactly uniform
    np.testing.assert_allclose(orc.tanh_faces(16, 16.0, 1e-6), np.arange(17.0), atol=1e-9)
    np.testing.assert_array_equal(orc.tanh_faces(16, 16.0, 0.0), np.arange(17.0))


# ---------------------------------------------------------------- Eq. 63
@pytest.mark.parametrize("Ra,Pr,Ma,L", [(1e3, 0.71, 0.1, 64), (1e8, 0.71, 0.1, 512),
                                        (3e5, 7.0, 0.05, 100)])
def test_params_reproduce_ra_pr_vc(orc, Ra, Pr, Ma, L):
    nu, chi, bg = orc.params_from_ra(Ra, Pr, Ma, L, 1.0)
    Vc = Ma  # V_c = Ma c with c = 1
    assert Vc ** 2 * L ** 2 / (chi * nu) == pytest.approx(Ra, rel=1e-13)
    assert nu / chi == pytest.approx(Pr, rel=1e-14)
    assert np.sqrt(bg * 1.0 * L) == pytest.approx(Vc, rel=1e-14)
    # the buoyancy form of Eq. 63: Ra = beta g dT L^3 / (nu chi)
    assert bg * L ** 3 / (nu * chi) == pytest.approx(Ra, rel=1e-13)


# ---------------------------------------------------------------- helpers
def linear_fields(c, x, y):
    """rho, u, v, T as affine functions of position with coefficients c."""
    return tuple(c[q][0] + c[q][1] * x + c[q][2] * y for q in range(4))


LIN = [(1.02, 0.0, 0.0),           # rho constant
       (0.013, 0.0011, -0.0007),   # u
       (-0.008, 0.0004, 0.0009),   # v
       (0.45, -0.006, 0.0031)]     # T


def lin_problem(orc, seed=3, n=10, kappa=1.0, nu=0.04, chi=0.05):
    xf = inputs.random_faces(n, seed)
    yf = inputs.random_faces(n, seed + 1)
    p = orc.Problem(xf=xf, yf=yf, nu=nu, chi=chi, beta_g=0.0, kappa=kappa, dt=0.3)
    X, Y = np.meshgrid(centres(xf), centres(yf))
    return p, linear_fields(LIN, X, Y)


# ---------------------------------------------------------------- Eqs. 55-56
def test_gradients_exact_for_linear_fields_on_irregular_mesh(orc):
    coef = [(1.0, 0.003, -0.002), (0.01, 0.002, 0.001), (-0.02, -0.001, 0.004),
            (0.3, 0.01, 0.02)]
    xf = inputs.random_faces(12, 11)
    yf = inputs.random_faces(9, 12)
    p = orc.Problem(xf=xf, yf=yf, nu=0.1, chi=0.1)
    X, Y = np.meshgrid(centres(xf), centres(yf))
    st = linear_fields(coef, X, Y)
    g = orc.gradients(p, st)
    inner = (slice(1, -1), slice(1, -1))
    for q in range(4):
        np.testing.assert_allclose(g[q, 0][inner], coef[q][1], rtol=0, atol=1e-13)
        np.testing.assert_allclose(g[q, 1][inner], coef[q][2], rtol=0, atol=1e-13)


def test_gradients_uniform_mesh_are_central_differences(orc):
    n = 8
    xf = inputs.uniform_faces(n)
    p = orc.Problem(xf=xf, yf=xf.copy(), nu=0.1, chi=0.1)
    st = inputs.perturbed_state(n, n, seed=5)
    g = orc.gradients(p, st)
    for q in range(4):
        a = st[q]
        cdx = (a[:, 2:] - a[:, :-2]) / 2.0
        cdy = (a[2:, :] - a[:-2, :]) / 2.0
        np.testing.assert_allclose(g[q, 0][:, 1:-1], cdx, rtol=0, atol=1e-14)
        np.testing.assert_allclose(g[q, 1][1:-1, :], cdy, rtol=0, atol=1e-14)


# ---------------------------------------------------------------- Eq. 29
@pytest.mark.parametrize("nd", [0, 1])
def test_nodes_take_the_plane_of_the_cell_they_lie_in(orc, nd):
    """Brute force over the 9 nodes of one face: a node strictly inside the
    left (right) cell equals that cell's reconstruction plane; a node on the
    face line is the mean of the two planes."""
    n = 8
    xf = inputs.random_faces(n, 21)
    yf = inputs.random_faces(n, 22)
    p = orc.Problem(xf=xf, yf=yf, nu=0.05, chi=0.05, kappa=0.8)
    st = inputs.perturbed_state(n, n, seed=23)
    g = orc.gradients(p, st)
    xc, yc = centres(xf), centres(yf)
    i, j = 4, 3
    o = orc.face(p, st, nd, i, j)
    nodes = o.nodes()
    if nd == 0:
        cL, cR = (i - 1, j), (i, j)
        xS = np.array([xf[i], yc[j]])
        h = 0.8 * min(xf[i] - xf[i - 1], xf[i + 1] - xf[i])
    else:
        cL, cR = (i, j - 1), (i, j)
        xS = np.array([xc[i], yf[j]])
        h = 0.8 * min(yf[j] - yf[j - 1], yf[j + 1] - yf[j])
    assert o.h == pytest.approx(h, rel=1e-15)

    def plane(cell, q, pos):
        ci, cj = cell
        ctr = np.array([xc[ci], yc[cj]])
        return st[q][cj, ci] + g[q, 0][cj, ci] * (pos[0] - ctr[0]) + g[q, 1][cj, ci] * (pos[1] - ctr[1])

    face_line = xS[nd]
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            pos = xS + h * np.array([a, b], dtype=float)
            for q in range(4):
                if pos[nd] < face_line - 1e-12:
                    want = plane(cL, q, pos)
                elif pos[nd] > face_line + 1e-12:
                    want = plane(cR, q, pos)
                else:
                    want = 0.5 * (plane(cL, q, pos) + plane(cR, q, pos))
                assert nodes[q, a + 1, b + 1] == pytest.approx(want, rel=0, abs=1e-14)


# ---------------------------------------------------------------- Eqs. 30-32 vs 46-48
def _face_geometry(p, nd, i, j, kappa):
    xc, yc = centres(p.xf), centres(p.yf)
    if nd == 0:
        xS = np.array([p.xf[i], yc[j]])
        h = kappa * min(p.xf[i] - p.xf[i - 1], p.xf[i + 1] - p.xf[i])
    else:
        xS = np.array([xc[i], p.yf[j]])
        h = kappa * min(p.yf[j] - p.yf[j - 1], p.yf[j + 1] - p.yf[j])
    return xS, h


def _fields_at(pos):
    return linear_fields(LIN, pos[0], pos[1])


@pytest.mark.parametrize("nd,i,j,kappa", [(0, 5, 4, 1.0), (1, 4, 5, 1.0), (0, 4, 6, 0.55),
                                          (1, 6, 3, 0.3)])
def test_predictor_equals_d2q9_moment_sums(orc, nd, i, j, kappa):
    p, st = lin_problem(orc, kappa=kappa)
    o = orc.face(p, st, nd, i, j)
    xS, h = _face_geometry(p, nd, i, j, kappa)
    rho_s = m_x = m_y = E_s = 0.0
    for k in range(9):
        e = E_D2Q9[:, k]
        r, u, v, T = _fields_at(xS - e * h)          # x_S - e_i dt (Eq. 29 node)
        fk = f_eq(r, u, v)[k]
        gk = g_eq(r, u, v, T)[k]
        rho_s += fk                                   # Eq. 30
        m_x += e[0] * fk                              # Eq. 31
        m_y += e[1] * fk
        E_s += gk                                     # Eq. 32
    got = np.array(o.pred[:])
    want = np.array([rho_s, m_x, m_y, E_s])
    np.testing.assert_allclose(got, want, rtol=0, atol=2e-15)


@pytest.mark.parametrize("nd,i,j,kappa", [(0, 5, 4, 1.0), (1, 4, 5, 1.0), (0, 4, 6, 0.55),
                                          (1, 6, 3, 0.3)])
def test_flux_equals_distribution_form(orc, nd, i, j, kappa):
    nu, chi = 0.04, 0.05
    p, st = lin_problem(orc, kappa=kappa, nu=nu, chi=chi)
    o = orc.face(p, st, nd, i, j)
    xS, h = _face_geometry(p, nd, i, j, kappa)
    # predicted macroscopic variables from Eqs. 30-32
    rho_s = m = E_s = 0.0
    m = np.zeros(2)
    for k in range(9):
        e = E_D2Q9[:, k]
        r, u, v, T = _fields_at(xS - e * h)
        rho_s += f_eq(r, u, v)[k]
        m += e * f_eq(r, u, v)[k]
        E_s += g_eq(r, u, v, T)[k]
    us, vs, Ts = m[0] / rho_s, m[1] / rho_s, E_s / rho_s
    f_star = f_eq(rho_s, us, vs)
    g_star = g_eq(rho_s, us, vs, Ts)
    r0, u0, v0, T0 = _fields_at(xS)
    f0 = f_eq(r0, u0, v0)
    g0 = g_eq(r0, u0, v0, T0)
    tau_f = nu / (CS2 * h) + 0.5   # Eq. 9
    tau_g = chi / (CS2 * h) + 0.5  # Eq. 10
    # dt e.grad f_i at x_S: exact half-difference for quadratic equilibria
    dfe = np.empty(9)
    dge = np.empty(9)
    for k in range(9):
        e = E_D2Q9[:, k]
        rp, up, vp, Tp = _fields_at(xS + e * h)
        rm, um, vm, Tm = _fields_at(xS - e * h)
        dfe[k] = 0.5 * (f_eq(rp, up, vp)[k] - f_eq(rm, um, vm)[k])
        dge[k] = 0.5 * (g_eq(rp, up, vp, Tp)[k] - g_eq(rm, um, vm, Tm)[k])
    noneq_f = f_star - f0 + dfe   # f* - f_eq(x_S - e dt) to first order
    noneq_g = g_star - g0 + dge
    b = nd  # face normal axis
    P = np.sum(E_D2Q9[b] * f_star)                                    # Eq. 38
    Pi = [np.sum(E_D2Q9[a] * E_D2Q9[b] * (f_star + (0.5 - tau_f) * noneq_f)) for a in (0, 1)]
    Q = np.sum(E_D2Q9[b] * (g_star + (0.5 - tau_g) * noneq_g))          # Eq. 40
    want = np.array([P, Pi[0], Pi[1], Q])
    got = np.array(o.flux[:])
    assert o.tau_f == pytest.approx(tau_f, rel=1e-15)
    np.testing.assert_allclose(got, want, rtol=0, atol=5e-15)


# ---------------------------------------------------------------- boundary readings
def _cavity_like(orc, kinds, seed=31, n=7):
    xf = inputs.random_faces(n, seed)
    yf = inputs.random_faces(n + 2, seed + 1)
    p = orc.Problem(xf=xf, yf=yf, nu=0.03, chi=0.04, beta_g=1e-3, kappa=0.9,
                    bc_kind=kinds, bc_T=(0.9, 0.1, 0.3, 0.6), bc_u=(0.0, 0.0, 0.0, 0.02))
    st = inputs.perturbed_state(p.nx, p.ny, seed=seed + 2)
    return p, st


def test_wall_faces_carry_no_mass_and_adiabatic_walls_no_energy(orc):
    D, A = orc.DIRICHLET, orc.ADIABATIC
    p, st = _cavity_like(orc, (D, D, A, A))
    fx, fy = orc.fluxes(p, st)
    assert np.all(fx[0][:, 0] == 0.0) and np.all(fx[0][:, -1] == 0.0)
    assert np.all(fy[0][0, :] == 0.0) and np.all(fy[0][-1, :] == 0.0)
    assert np.all(fy[3][0, :] == 0.0) and np.all(fy[3][-1, :] == 0.0)
    # the Dirichlet walls do carry heat
    assert np.all(fx[3][:, 0] != 0.0)


def test_wall_node_takes_wall_values(orc):
    D, A = orc.DIRICHLET, orc.ADIABATIC
    p, st = _cavity_like(orc, (D, D, A, D))
    for nd, i, j, side in [(0, 0, 3, orc.W), (0, p.nx, 5, orc.E), (1, 2, p.ny, orc.N)]:
        nodes = orc.face(p, st, nd, i, j).nodes()
        # node column on the wall line (normal offset 0): u_n = 0, u_t = wall velocity
        line = nodes[:, 1, :] if nd == 0 else nodes[:, :, 1]
        un = line[1] if nd == 0 else line[2]
        ut = line[2] if nd == 0 else line[1]
        np.testing.assert_allclose(un, 0.0, atol=1e-16)
        np.testing.assert_allclose(ut, p.bc_u[side], atol=1e-16)
        np.testing.assert_allclose(line[3], p.bc_T[side], atol=1e-15)


def test_periodic_face_is_shared(orc):
    """With x periodic, the face at i = 0 and at i = nx is one face."""
    P, A = orc.PERIODIC, orc.ADIABATIC
    p, st = _cavity_like(orc, (P, P, A, A))
    fx, _ = orc.fluxes(p, st)
    np.testing.assert_array_equal(fx[:, :, 0], fx[:, :, -1])


# ---------------------------------------------------------------- orders in h
def smooth_fields(x, y):
    """Smooth non-polynomial fields (complex-safe for complex-step derivatives)."""
    rho = 1.0 + 0.02 * np.sin(0.9 * x + 0.4 * y + 0.3)
    u = 0.03 * np.cos(0.6 * x - 0.8 * y) + 0.01
    v = -0.02 * np.sin(0.5 * x + 0.7 * y + 1.0)
    T = 0.5 + 0.2 * np.cos(0.8 * x + 0.3 * y - 0.5)
    return rho, u, v, T


XS = np.array([0.37, -0.21])


def sampled_nodes(h):
    nodes = np.empty((4, 3, 3))
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            f = smooth_fields(XS[0] + a * h, XS[1] + b * h)
            for q in range(4):
                nodes[q, a + 1, b + 1] = f[q]
    return nodes


def moment_predictor(h):
    """Eqs. 30-32: rho*, (rho u)*, (rho v)*, (rho T)* as D2Q9 moment sums of
    the equilibria at x_S - e_i h."""
    out = np.zeros(4)
    for k in range(9):
        e = E_D2Q9[:, k]
        r, u, v, T = smooth_fields(*(XS - e * h))
        fk, gk = f_eq(r, u, v)[k], g_eq(r, u, v, T)[k]
        out += np.array([fk, e[0] * fk, e[1] * fk, gk])
    return out


@pytest.mark.parametrize("nd", [0, 1])
def test_predictor_is_third_order_close_to_moment_sums(orc, nd):
    """Eqs. 46-48 are the second-order Taylor form of Eqs. 30-32 (Eqs. 44-45),
    so on smooth data the two differ by O(h^3) in every component; a wrong
    second-order coefficient would leave O(h^2)."""
    p = orc.Problem(xf=np.arange(3.0), yf=np.arange(3.0), nu=0.02, chi=0.03)
    hs = [0.2, 0.1, 0.05]
    d = []
    for h in hs:
        o = orc.face_from_nodes(p, nd, sampled_nodes(h), h)
        d.append(np.abs(np.array(o.pred[:]) - moment_predictor(h)))
    d = np.array(d)
    orders = np.log2(d[:-1] / d[1:])
    assert np.all(orders > 2.7), orders


@pytest.mark.parametrize("nd", [0, 1])
def test_flux_is_second_order_close_to_distribution_form(orc, nd):
    """Eqs. 57-59's braces against Eqs. 38-40 with f_eq(x_S - e h) replaced by
    its first-order Taylor form and the exact gradient (complex step), and the
    prediction taken from Eqs. 30-32: at fixed nu, chi the two differ by
    O(h^2) (derivative truncation, and (tau - 1/2) ~ 1/h times the O(h^3)
    predictor difference).  A dropped viscous term leaves O(1), a wrong
    dissipation coefficient O(h)."""
    nu, chi = 0.02, 0.03
    p = orc.Problem(xf=np.arange(3.0), yf=np.arange(3.0), nu=nu, chi=chi)
    hs = [0.01, 0.005, 0.0025]  # asymptotic range: two O(h^2) terms compete above
    d = []
    for h in hs:
        o = orc.face_from_nodes(p, nd, sampled_nodes(h), h)
        pr = moment_predictor(h)
        rs, us, vs, Ts = pr[0], pr[1] / pr[0], pr[2] / pr[0], pr[3] / pr[0]
        fs, gs = f_eq(rs, us, vs), g_eq(rs, us, vs, Ts)
        f0 = f_eq(*smooth_fields(*XS)[:3])
        g0 = g_eq(*smooth_fields(*XS))
        eps = 1e-20
        dfe = np.empty(9)
        dge = np.empty(9)
        for k in range(9):
            e = E_D2Q9[:, k]
            z = XS + 1j * eps * e
            fz = smooth_fields(z[0], z[1])
            dfe[k] = h * f_eq(*fz[:3])[k].imag / eps
            dge[k] = h * g_eq(*fz)[k].imag / eps
        tf = nu / (CS2 * h) + 0.5
        tg = chi / (CS2 * h) + 0.5
        b = nd
        P = np.sum(E_D2Q9[b] * fs)
        Pi = [np.sum(E_D2Q9[a] * E_D2Q9[b] * (fs + (0.5 - tf) * (fs - f0 + dfe))) for a in (0, 1)]
        Q = np.sum(E_D2Q9[b] * (gs + (0.5 - tg) * (gs - g0 + dge)))
        d.append(np.abs(np.array(o.flux[:]) - np.array([P, Pi[0], Pi[1], Q])))
    d = np.array(d)
    orders = np.log2(d[:-1] / d[1:])
    assert np.all(orders > 1.8), (d, orders)


# ---------------------------------------------------------------- R12 residual
def _r12_from_states(st0, st1):
    """The steady residual of reading R12 (the L2 analogue of Section 3.3's
    Eq. 65), evaluated from its definition on two states: the cell speeds
    |u| = sqrt(u^2 + v^2), a plain sum over cells, the new state's norm as
    the denominator."""
    m0 = np.hypot(st0[1], st0[2])
    m1 = np.hypot(st1[1], st1[2])
    ru = np.sqrt(np.sum((m1 - m0) ** 2)) / np.sqrt(np.sum(m1 ** 2))
    rT = np.sqrt(np.sum((st1[3] - st0[3]) ** 2)) / np.sqrt(np.sum(st1[3] ** 2))
    return float(ru), float(rT)


@pytest.mark.parametrize("kinds", [(0, 0, 1, 1), (2, 2, 0, 1)])
def test_residual_is_relative_l2_change_of_speed_and_temperature(orc, kinds):
    """The residual a step returns equals R12 evaluated here from the state
    before and after that step.  The alternative readings a slip would give
    -- componentwise velocity differences, the old state's norm as the
    denominator, no square root -- are checked to differ on the same states,
    so the comparison can tell them apart."""
    nx, ny = 13, 11
    p = orc.Problem(xf=inputs.random_faces(nx, 21), yf=inputs.random_faces(ny, 22), nu=0.03,
                    chi=0.04, beta_g=2e-4, dt=0.2, bc_kind=kinds)
    st = inputs.perturbed_state(nx, ny, 23)
    for _ in range(3):  # three consecutive steps, each checked
        st1, res, rc = orc.step(p, st, 1)
        assert rc == 0
        ru, rT = _r12_from_states(st, st1)
        assert res[0] == pytest.approx(ru, rel=1e-13, abs=0)
        assert res[1] == pytest.approx(rT, rel=1e-13, abs=0)
        # the readings a slip would produce are far from R12 on this state
        comp = np.sqrt(np.sum((st1[1] - st[1]) ** 2 + (st1[2] - st[2]) ** 2)) / np.sqrt(
            np.sum(np.hypot(st1[1], st1[2]) ** 2))
        old_den = np.sqrt(np.sum((np.hypot(st1[1], st1[2]) - np.hypot(st[1], st[2])) ** 2)) / \
            np.sqrt(np.sum(np.hypot(st[1], st[2]) ** 2))
        for alt in (comp, old_den, ru ** 2):
            assert abs(alt - ru) > 1e-3 * ru
        st = st1
    # after several steps the returned residual is the last step's
    st3, res3, rc = orc.step(p, inputs.perturbed_state(nx, ny, 23), 3)
    assert rc == 0
    np.testing.assert_allclose(res3, res, rtol=1e-13, atol=0)


def test_residual_of_a_resting_state_has_zero_denominator(orc):
    """R12 with |u|^{n+1} = 0 everywhere: the velocity residual's denominator
    is zero, which reads as infinity (no convergence is claimed for a fluid
    at rest); the temperature of the Ra -> 0 conduction profile does not
    change, so R_T is zero to round-off."""
    p = orc.cavity_problem(12, 1e4, phi=1.5)
    p.beta_g = 0.0
    _, res, rc = orc.step(p, inputs.conduction_state(p.xf, p.yf), 1)
    assert rc == 0
    assert res[0] == np.inf
    assert 0.0 <= res[1] < 1e-14
