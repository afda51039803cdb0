"""Pins of the curvilinear FP64 oracle (2D RTLBFS on body-fitted structured
meshes, the local face frames of Section 3.2; Section 4.3), against what the
paper, the mathematics and the separately pinned rectilinear oracle fix:

* a rectilinear mesh given as vertices reproduces the rectilinear oracle,
  with walls, moving walls and a translational periodic seam;
* rotating the mesh, the velocities, gravity, wall velocities and body
  force by an arbitrary angle rotates the result (the local frame, the
  velocity rotation and the rotation of the fluxes back);
* Eqs. 55-56 are exact for linear fields on an affine (sheared, rotated,
  stretched) mesh;
* a uniform free stream stays uniform on an O-mesh between two far fields
  (the face vectors of every cell close);
* mass is conserved on a walled annulus; the conductive heat through a
  concentric annulus converges at second order to 2 pi chi dT / ln(ro/ri).
"""
import numpy as np
import pytest

from paper_2202_13449_gb300 import inputs


@pytest.fixture(scope="module")
def cv(orc):
    from oracle import curv as mod
    return mod


def rect_vertices(xf, yf):
    X, Y = np.meshgrid(xf, yf)
    return X, Y


def o_mesh(ni, nj, ri, ro, stretch=1.0):
    """O-mesh of an annulus: theta decreasing with i (right-handed: i along
    -theta, j along r), radii geometric-like in j."""
    th = -2.0 * np.pi * np.arange(ni + 1) / ni
    th[-1] = -2.0 * np.pi  # the seam: column ni is column 0
    s = np.linspace(0.0, 1.0, nj + 1)
    r = ri * (ro / ri) ** (s ** stretch) if stretch != 1.0 else ri * (ro / ri) ** s
    X = np.outer(r, np.cos(th))
    Y = np.outer(r, np.sin(th))
    X[:, -1], Y[:, -1] = X[:, 0], Y[:, 0]
    return X, Y


def test_rectilinear_mesh_reproduces_the_rectilinear_oracle(orc, cv):
    D, A, P = orc.DIRICHLET, orc.ADIABATIC, orc.PERIODIC
    nx, ny = 11, 9
    xf, yf = inputs.random_faces(nx, 61), inputs.random_faces(ny, 62)
    X, Y = rect_vertices(xf, yf)
    for kinds in ((D, A, A, D), (P, P, D, A)):
        p2 = orc.Problem(xf=xf, yf=yf, nu=0.03, chi=0.04, beta_g=2e-3, kappa=0.9, dt=0.2,
                         fx=1e-4, fy=-2e-4, bc_kind=kinds, bc_T=(0.9, 0.1, 0.3, 0.6),
                         bc_u=(0.01, 0.0, 0.0, 0.02))
        bcu = ((0.0, 0.01), (0.0, 0.0), (0.0, 0.0), (0.02, 0.0))
        pc = cv.ProblemC(X=X, Y=Y, nu=0.03, chi=0.04, beta_g=2e-3, kappa=0.9, dt=0.2,
                         gdir=(0.0, 1.0), force=(1e-4, -2e-4), bc_kind=kinds,
                         bc_T=(0.9, 0.1, 0.3, 0.6), bc_u=bcu)
        st = inputs.perturbed_state(nx, ny, seed=63)
        a, ra, rc1 = orc.step(p2, st, 5)
        b, rb, rc2 = cv.step(pc, st, 5)
        assert rc1 == rc2 == 0
        for q in range(4):
            np.testing.assert_allclose(b[q], a[q], rtol=0, atol=2e-15)
        assert rb == pytest.approx(ra, rel=1e-12)


def rot(a, x, y):
    c, s = np.cos(a), np.sin(a)
    return c * x - s * y, s * x + c * y


def test_rotation_commutes_with_the_step(orc, cv):
    """Rotating the whole problem by an angle rotates the result."""
    D, A = cv.DIRICHLET, cv.ADIABATIC
    nx, ny = 10, 8
    X0, Y0 = rect_vertices(inputs.random_faces(nx, 71), inputs.random_faces(ny, 72))
    # a curved (non-rectilinear) mesh: bend it
    X0 = X0 + 0.15 * np.sin(0.4 * Y0)
    Y0 = Y0 + 0.1 * np.cos(0.3 * X0)
    kinds = (D, A, A, D)
    bcu = ((0.0, 0.01), (0.0, 0.0), (0.0, 0.0), (0.02, -0.005))
    st = inputs.perturbed_state(nx, ny, seed=73)
    g = np.array([0.3, 0.95])
    g /= np.linalg.norm(g)
    f = (1e-4, -2e-4)
    base = dict(nu=0.03, chi=0.04, beta_g=2e-3, kappa=0.9, dt=0.2, bc_kind=kinds,
                bc_T=(0.9, 0.1, 0.3, 0.6))
    p0 = cv.ProblemC(X=X0, Y=Y0, gdir=tuple(g), force=f, bc_u=bcu, **base)
    a = 0.37
    X1, Y1 = rot(a, X0, Y0)
    g1 = rot(a, g[0], g[1])
    f1 = rot(a, *f)
    bcu1 = tuple(tuple(rot(a, *u)) for u in bcu)
    p1 = cv.ProblemC(X=X1, Y=Y1, gdir=g1, force=f1, bc_u=bcu1, **base)
    u1, v1 = rot(a, st[1], st[2])
    s0, _, rc0 = cv.step(p0, st, 4)
    s1, _, rc1 = cv.step(p1, (st[0], u1, v1, st[3]), 4)
    assert rc0 == rc1 == 0
    ur, vr = rot(a, s0[1], s0[2])
    np.testing.assert_allclose(s1[0], s0[0], rtol=0, atol=1e-14)
    np.testing.assert_allclose(s1[3], s0[3], rtol=0, atol=1e-14)
    np.testing.assert_allclose(s1[1], ur, rtol=0, atol=1e-15)
    np.testing.assert_allclose(s1[2], vr, rtol=0, atol=1e-15)


def test_gradients_exact_for_linear_fields_on_an_affine_mesh(cv):
    nx, ny = 8, 7
    I, J = np.meshgrid(np.arange(nx + 1.0), np.arange(ny + 1.0))
    X = 1.3 * I + 0.4 * J + 2.0
    Y = -0.2 * I + 0.9 * J - 1.0
    p = cv.ProblemC(X=X, Y=Y, nu=0.02, chi=0.03,
                    bc_kind=(cv.ADIABATIC, cv.ADIABATIC, cv.ADIABATIC, cv.ADIABATIC))
    # centres of an affine mesh are the images of the index centres
    Ic, Jc = np.meshgrid(np.arange(nx) + 0.5, np.arange(ny) + 0.5)
    xc, yc = 1.3 * Ic + 0.4 * Jc + 2.0, -0.2 * Ic + 0.9 * Jc - 1.0
    coef = [(1.0, 0.002, -0.001), (0.01, 0.003, 0.002), (-0.02, -0.001, 0.004), (0.5, 0.05, -0.03)]
    st = tuple(c0 + cx * xc + cy * yc for c0, cx, cy in coef)
    g, geo = cv.gradients(p, st)
    np.testing.assert_allclose(geo[0], xc, rtol=0, atol=1e-13)
    inner = (slice(1, -1), slice(1, -1))
    for q, (c0, cx, cy) in enumerate(coef):
        np.testing.assert_allclose(g[q, 0][inner], cx, rtol=0, atol=1e-14)
        np.testing.assert_allclose(g[q, 1][inner], cy, rtol=0, atol=1e-14)


def test_uniform_free_stream_is_preserved_on_an_o_mesh(cv):
    X, Y = o_mesh(24, 10, 1.0, 6.0, stretch=1.3)
    inf = (1.0, 0.0577, -0.012, 0.3)
    p = cv.ProblemC(X=X, Y=Y, nu=0.01, chi=0.014, dt=0.02, kappa=0.8,
                    bc_kind=(cv.PERIODIC, cv.PERIODIC, cv.FARFIELD, cv.FARFIELD), inf=inf)
    nj, ni = p.shape
    st = tuple(np.full((nj, ni), v) for v in inf)
    s, _, rc = cv.step(p, st, 20)
    assert rc == 0
    for q in range(4):
        np.testing.assert_allclose(s[q], inf[q], rtol=0, atol=5e-15)


def test_mass_conserved_on_a_walled_annulus(cv):
    X, Y = o_mesh(32, 12, 1.0, 4.0)
    p = cv.ProblemC(X=X, Y=Y, nu=0.02, chi=0.028, beta_g=1e-3, dt=0.02, kappa=0.9,
                    gdir=(0.0, 1.0), bc_kind=(cv.PERIODIC, cv.PERIODIC, cv.DIRICHLET, cv.DIRICHLET),
                    bc_T=(0, 0, 1.0, 0.0))
    nj, ni = p.shape
    st = inputs.perturbed_state(ni, nj, seed=81)
    _, geo = cv.gradients(p, st)
    m0 = float(np.sum(st[0] * geo[2]))
    s, _, rc = cv.step(p, st, 100)
    assert rc == 0
    assert abs(float(np.sum(s[0] * geo[2])) - m0) / m0 < 1e-13


@pytest.mark.slow
def test_annulus_conduction_converges_at_second_order(cv):
    """Ra -> 0 in a concentric annulus: the steady conductive heat through the
    inner wall tends to 2 pi chi dT / ln(ro / ri) (per unit depth)."""
    ri, ro, chi = 1.0, 2.0, 0.05
    errs = []
    for n in (6, 12, 24):
        X, Y = o_mesh(4 * n, n, ri, ro)
        p = cv.ProblemC(X=X, Y=Y, nu=0.05, chi=chi, beta_g=0.0, dt=0.0,
                        kappa=1.0, bc_kind=(cv.PERIODIC, cv.PERIODIC, cv.DIRICHLET, cv.DIRICHLET),
                        bc_T=(0, 0, 1.0, 0.0))
        nj, ni = p.shape
        _, geo = cv.gradients(p, [np.ones((nj, ni))] * 4)
        w = (ro - ri) / n
        p.dt = 0.1 * w * w / chi
        r = np.hypot(geo[0], geo[1])
        T0 = np.log(r / ro) / np.log(ri / ro)
        st = (np.ones((nj, ni)), np.zeros((nj, ni)), np.zeros((nj, ni)), T0)
        # with no buoyancy the velocity stays at round-off, so R_u is noise
        # over noise: run three diffusion times and check R_T instead
        steps = int(3.0 * (ro - ri) ** 2 / chi / p.dt)
        s, res, rc = cv.step(p, st, steps)
        assert rc == 0 and res[1] < 1e-9, res
        q, _ = cv.heat(p, s, 2)
        exact = 2.0 * np.pi * chi / np.log(ro / ri)
        errs.append(abs(q - exact) / exact)
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 2e-3, errs
    assert np.all(orders > 1.7), (errs, orders)


@pytest.mark.parametrize("shear", [0.0, 0.35])
def test_couette_flow_is_a_fixed_point_on_a_sheared_mesh(cv, shear):
    """Plane Couette flow between a wall at rest (j = 0) and a wall moving
    along x at U (j = nj), periodic along x, on a mesh whose i-lines are
    sheared (cells are parallelograms, faces not orthogonal to the centre
    lines): u = U y / H, v = 0, rho = 1 and uniform T solve the steady
    equations, and the scheme keeps them to round-off.  Linear fields are
    reconstructed exactly (Eqs. 29, 55-56), the predictor's central
    differences are exact for the quadratic products (Eqs. 46-48), the
    mirrored wall ghosts lie on the same line, and the viscous flux is the
    same through every x-face: a wrong frame rotation, ghost rule or
    tangential offset breaks the balance."""
    ni, nj, H, U = 12, 9, 9.0, 0.04
    I, J = np.meshgrid(np.arange(ni + 1.0), np.arange(nj + 1.0))
    X = I + shear * J
    Y = J * (H / nj)
    p = cv.ProblemC(X=X, Y=Y, nu=0.05, chi=0.07, dt=0.2, kappa=1.0,
                    bc_kind=(cv.PERIODIC, cv.PERIODIC, cv.ADIABATIC, cv.ADIABATIC),
                    bc_u=((0.0, 0.0), (0.0, 0.0), (0.0, 0.0), (U, 0.0)))
    _, geo = cv.gradients(p, inputs.perturbed_state(ni, nj, seed=3))
    yc = geo[1]
    st = (np.ones((nj, ni)), U * yc / H, np.zeros((nj, ni)), np.full((nj, ni), 0.4))
    s, res, rc = cv.step(p, st, 50)
    assert rc == 0
    np.testing.assert_allclose(s[1], st[1], rtol=0, atol=1e-14)
    np.testing.assert_allclose(s[2], 0.0, rtol=0, atol=1e-14)
    np.testing.assert_allclose(s[0], 1.0, rtol=0, atol=1e-13)
    np.testing.assert_allclose(s[3], 0.4, rtol=0, atol=1e-14)


def _poiseuille(cv, nj, shear, ni=6, nu=0.1, umax=0.01):
    """Steady channel flow driven by a body force f along x between walls at
    rest at y = 0 and y = H (cells of unit height, i-lines sheared by
    `shear` per row): the discrete u at the centres and the closed form
    f / (2 nu) y (H - y)."""
    H = float(nj)
    I, J = np.meshgrid(np.arange(ni + 1.0), np.arange(nj + 1.0))
    p = cv.ProblemC(X=I + shear * J, Y=J.copy(), nu=nu, chi=nu, dt=0.25, kappa=1.0,
                    force=(8.0 * nu * umax / H ** 2, 0.0),
                    bc_kind=(cv.PERIODIC, cv.PERIODIC, cv.ADIABATIC, cv.ADIABATIC))
    _, geo = cv.gradients(p, inputs.perturbed_state(ni, nj, seed=3))
    yc = geo[1]
    st = (np.ones((nj, ni)), np.zeros((nj, ni)), np.zeros((nj, ni)), np.full((nj, ni), 0.4))
    s, _, _, rc = cv.run_to_steady(p, st, 1e-12, 2_000_000)
    assert rc == 0
    exact = p.force[0] / (2.0 * nu) * yc * (H - yc)
    return s, exact


def test_poiseuille_converges_at_second_order_on_a_sheared_mesh(cv):
    """Body-force-driven channel flow, whose shear stress varies across the
    channel (unlike Couette flow, a wrong flux rotation, viscous term or wall
    rule does not cancel between faces).  On a mesh sheared by 0.35 per row
    the steady profile converges to the closed form at second order (error
    3.8 % of u_max with 8 cells across, 0.94 % with 16), the cross-stream
    velocity stays at round-off, and the result equals the unsheared mesh's:
    the face frames and tangential offsets remove the shear exactly for this
    flow."""
    errs = []
    for nj in (8, 16):
        s, exact = _poiseuille(cv, nj, 0.35)
        errs.append(float(np.max(np.abs(s[1] - exact))) / 0.01)
        assert np.max(np.abs(s[2])) < 1e-14
        s0, _ = _poiseuille(cv, nj, 0.0)
        np.testing.assert_allclose(s[1], s0[1], rtol=1e-10, atol=1e-16)
    assert errs[1] < 0.011
    assert 3.6 < errs[0] / errs[1] < 4.4, errs


def test_residual_is_relative_l2_change_of_speed_and_temperature(cv):
    """The residual a curvilinear step returns equals R12 evaluated here from
    the states before and after it (cell speeds, plain sums over cells, the
    new state's norm as the denominator, as on rectilinear meshes); the
    componentwise and old-norm readings differ on these states."""
    X, Y = o_mesh(24, 10, 1.0, 3.0)
    p = cv.ProblemC(X=X, Y=Y, nu=0.02, chi=0.028, beta_g=1e-3, dt=0.02, kappa=0.9,
                    gdir=(0.0, 1.0), bc_kind=(cv.PERIODIC, cv.PERIODIC, cv.DIRICHLET, cv.DIRICHLET),
                    bc_T=(0, 0, 1.0, 0.0))
    nj, ni = p.shape
    st = inputs.perturbed_state(ni, nj, seed=82)
    for _ in range(2):
        st1, res, rc = cv.step(p, st, 1)
        assert rc == 0
        m0, m1 = np.hypot(st[1], st[2]), np.hypot(st1[1], st1[2])
        ru = np.sqrt(np.sum((m1 - m0) ** 2)) / np.sqrt(np.sum(m1 ** 2))
        rT = np.sqrt(np.sum((st1[3] - st[3]) ** 2)) / np.sqrt(np.sum(st1[3] ** 2))
        assert res[0] == pytest.approx(ru, rel=1e-13, abs=0)
        assert res[1] == pytest.approx(rT, rel=1e-13, abs=0)
        comp = np.sqrt(np.sum((st1[1] - st[1]) ** 2 + (st1[2] - st[2]) ** 2)) / np.sqrt(
            np.sum(m1 ** 2))
        old_den = np.sqrt(np.sum((m1 - m0) ** 2)) / np.sqrt(np.sum(m0 ** 2))
        for alt in (comp, old_den, ru ** 2):
            assert abs(alt - ru) > 1e-3 * ru
        st = st1
