"""Curvilinear CUDA path (include/rtlbfs_curv.h) against the curvilinear FP64
oracle, element by element, through the C ABI: FP64 <= 1e-12 after one
step and <= 1e-11 after 20, FP32 <= 1e-5 on u, v, T (1e-6 on rho); wall heat
sums <= 1e-12.  Meshes: a bent (non-orthogonal) cavity with moving walls and
oblique gravity, O-meshes of an annulus (walls, periodic seam) and of a
cylinder in a free stream (wall inside, far field outside), and a 1-cell
wide strip; both tile heights.
"""
import numpy as np
import pytest

from paper_2202_13449_gb300 import capi, inputs
from test_oracle_curv import o_mesh, rect_vertices  # noqa: E402

pytestmark = pytest.mark.gpu
D, A, P, F = capi.WALL_DIRICHLET, capi.WALL_ADIABATIC, capi.PERIODIC, capi.FARFIELD


@pytest.fixture(scope="module")
def cv(orc):
    from oracle import curv as mod
    return mod


def bent(nx, ny, seed):
    X, Y = rect_vertices(inputs.random_faces(nx, seed), inputs.random_faces(ny, seed + 1))
    X = X + 0.15 * np.sin(0.4 * Y)
    Y = Y + 0.1 * np.cos(0.3 * X)
    return X, Y


def case(cv, name):
    # transport coefficients and time step scaled to each mesh's cells (so
    # the explicit step is stable and tau < 1.5): unit cells for the bent
    # cavity and the strip, ~0.1 on the annulus, 0.02 at the cylinder wall
    base = dict(nu=0.03, chi=0.04, beta_g=2e-3, dt=0.05, kappa=0.9, force=(1e-4, -2e-4))
    if name == "annulus":
        base.update(nu=0.003, chi=0.004, dt=0.02)
    if name == "cylinder":
        base.update(nu=0.002, chi=0.003, dt=0.006)
    if name == "bent_cavity":
        X, Y = bent(37, 19, 91)
        g = np.array([0.3, 0.95]) / np.hypot(0.3, 0.95)  # a unit vector, as the library uses
        return cv.ProblemC(X=X, Y=Y, gdir=tuple(g), bc_kind=(D, A, A, D), bc_T=(0.9, 0.1, 0.3, 0.6),
                           bc_u=((0.0, 0.01), (0.0, 0.0), (0.0, 0.0), (0.02, -0.005)), **base), False
    if name == "annulus":
        X, Y = o_mesh(70, 18, 1.0, 3.0)
        return cv.ProblemC(X=X, Y=Y, gdir=(0.0, 1.0), bc_kind=(P, P, D, D), bc_T=(0, 0, 1.0, 0.0),
                           **base), True
    if name == "cylinder":
        X, Y = o_mesh(48, 21, 0.5, 8.0, stretch=1.4)
        return cv.ProblemC(X=X, Y=Y, gdir=(0.0, 1.0), bc_kind=(P, P, D, F), bc_T=(0, 0, 1.0, 0.0),
                           inf=(1.0, 0.0577, 0.0, 0.0), **base), True
    if name == "strip_1xN":
        X, Y = bent(1, 7, 95)
        return cv.ProblemC(X=X, Y=Y, gdir=(0.0, 1.0), bc_kind=(D, A, D, A), bc_T=(1.0, 0, 0.2, 0),
                           **base), False
    raise KeyError(name)


def solver(p, periodic, precision, tile_rows=0):
    s = capi.SolverC(p.X, p.Y, periodic, precision)
    s.set_physics(p.nu, p.chi, p.beta_g, p.dt)
    s.set_lattice(p.kappa)
    s.set_gravity(*p.gdir, p.T_ref)
    s.set_body_force(*p.force)
    s.set_farfield(*p.inf)
    for side in range(4):
        if periodic and side < 2:
            continue
        s.set_bc(side, p.bc_kind[side], p.bc_T[side], *p.bc_u[side])
    s.set_schedule(tile_rows)
    return s


def rel(a, b, floor):
    return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), floor))


def compare(got, ref, tol, precision):
    for q, floor in ((0, 1.0), (1, 1e-2), (2, 1e-2), (3, 1.0)):
        if q == 0 and precision == capi.FP32:
            assert np.max(np.abs(got[0] - ref[0])) < 1e-6
            continue
        e = rel(got[q], ref[q], floor)
        assert e < tol, (q, e)


def state_for(p, name):
    nj, ni = p.shape
    st = list(inputs.perturbed_state(ni, nj, seed=sum(map(ord, name))))
    if name == "cylinder":
        # a free stream of cold fluid against the hot wall: the wall's mirror
        # temperature 2 T_w - T_P is near 2, the edge of a stored FP32 value
        st[1] = st[1] + 0.0577
        st[3] = st[3] - 0.45
    return tuple(st)


NAMES = ["bent_cavity", "annulus", "cylinder", "strip_1xN"]


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("tile_rows", [8, 16])
def test_one_step_fp64(cv, name, tile_rows):
    p, per = case(cv, name)
    st = state_for(p, name)
    ref, rr, rc = cv.step(p, st, 1)
    assert rc == 0
    s = solver(p, per, capi.FP64, tile_rows)
    s.set_state(*st)
    s.step(1)
    compare(s.get_state(), ref, 1e-12, capi.FP64)
    rg, steps = s.residual()
    assert steps == 1
    np.testing.assert_allclose(rg, rr, rtol=1e-9)
    s.close()


@pytest.mark.parametrize("name", NAMES)
def test_twenty_steps_fp64_and_three_fp32(cv, name):
    p, per = case(cv, name)
    st = state_for(p, name)
    ref, _, rc = cv.step(p, st, 20)
    assert rc == 0
    s = solver(p, per, capi.FP64)
    s.set_state(*st)
    s.step(20)
    compare(s.get_state(), ref, 1e-11, capi.FP64)
    s.close()
    ref, _, rc = cv.step(p, st, 3)
    s = solver(p, per, capi.FP32)
    s.set_state(*st)
    s.step(3)
    compare(s.get_state(), ref, 1e-5, capi.FP32)
    s.close()


@pytest.mark.parametrize("name", ["annulus", "cylinder"])
def test_wall_heat_fp64(cv, name):
    p, per = case(cv, name)
    st = state_for(p, name)
    s = solver(p, per, capi.FP64)
    s.set_state(*st)
    for side in (2, 3):
        q, perim = s.wall_heat(side)
        qr, pr = cv.heat(p, st, side)
        assert q == pytest.approx(qr, rel=1e-12, abs=1e-15)
        assert perim == pytest.approx(pr, rel=1e-13)
    s.close()


def test_mass_conserved_on_the_annulus(cv):
    p, per = case(cv, "annulus")
    st = state_for(p, "annulus")
    _, geo = cv.gradients(p, st)
    s = solver(p, per, capi.FP64)
    s.set_state(*st)
    s.step(300)
    got = s.get_state()
    s.close()
    m0, m1 = np.sum(st[0] * geo[2]), np.sum(got[0] * geo[2])
    assert abs(m1 - m0) / m0 < 1e-13


@pytest.mark.parametrize("precision", [capi.FP64, capi.FP32])
def test_full_size_cylinder_450x300_step(cv, precision):
    """The bench's cylinder workload at full size, in its launch
    configuration (automatic tile height): Section 4.3's 450 x 300 O-mesh,
    Re = 20, Gr = 100, Pr = 0.7, buoyancy along the free stream; two steps
    from a perturbed free stream of cold fluid, every cell against the
    oracle, and the FP64 wall heat."""
    import math
    X, Y = inputs.cylinder_o_mesh(450, 300)
    uinf = 0.1 / math.sqrt(3.0)
    nu = uinf / 20.0
    chi = nu / 0.7
    wmin = float(np.min(np.diff(np.hypot(X, Y), axis=0)))
    p = cv.ProblemC(X=X, Y=Y, nu=nu, chi=chi, beta_g=100.0 * nu * nu, dt=0.2 * wmin * wmin / chi,
                    kappa=1.0, gdir=(1.0, 0.0), T_ref=0.0, bc_kind=(P, P, D, F),
                    bc_T=(0.0, 0.0, 1.0, 0.0), inf=(1.0, uinf, 0.0, 0.0))
    rho, u, v, T = inputs.perturbed_state(450, 300, seed=4503)
    st = (rho, u + uinf, v, 0.2 * T)
    ref, rr, rc = cv.step(p, st, 2)
    assert rc == 0
    s = solver(p, True, precision)
    s.set_state(*st)
    s.step(2)
    compare(s.get_state(), ref, 1e-12 if precision == capi.FP64 else 1e-5, precision)
    if precision == capi.FP64:
        np.testing.assert_allclose(s.residual()[0], rr, rtol=1e-9)
        s.set_state(*st)
        q, perim = s.wall_heat(2)
        qr, pr = cv.heat(p, st, 2)
        assert q == pytest.approx(qr, rel=1e-12)
        assert perim == pytest.approx(pr, rel=1e-13)
    s.close()


@pytest.mark.slow
def test_table4_gr100_on_the_paper_mesh():
    """Physics of the curvilinear GPU path at the paper's own setting
    (Section 4.3, Table 4, Gr = 100): the 450 x 300 O-mesh from 0.003 D to
    52.5 D, Re = 20, Pr = 0.7, u_inf = 0.1 c_s with buoyancy along the free
    stream, FP32 from the free stream to a 1e-8 residual (about 2.2e6 steps).
    The oracle cannot run this to a steady state, so the check is against
    the printed values: Eq. 73's mean Nusselt number within 1 % and the
    separation angle within 1.2 degrees (1.5 wall cells of 0.8 degrees)."""
    import json
    import math
    import os
    from paper_2202_13449_gb300 import post
    gold = {c["Gr"]: c for c in json.load(open(os.path.join(
        os.path.dirname(__file__), "golden", "table4_cylinder.json")))["cases"]}[100.0]
    X, Y = inputs.cylinder_o_mesh(450, 300)
    uinf = 0.1 / math.sqrt(3.0)
    nu = uinf / 20.0
    chi = nu / 0.7
    wmin = float(np.min(np.diff(np.hypot(X, Y), axis=0)))
    dt = 0.2 * wmin * wmin / chi
    s = capi.SolverC(X, Y, True, capi.FP32)
    s.set_physics(nu, chi, 100.0 * nu * nu, dt)
    s.set_gravity(1.0, 0.0, 0.0)
    s.set_bc(2, capi.WALL_DIRICHLET, 1.0)
    s.set_bc(3, capi.FARFIELD)
    s.set_farfield(1.0, uinf, 0.0, 0.0)
    nj, ni = 300, 450
    s.set_state(np.ones((nj, ni)), np.full((nj, ni), uinf), np.zeros((nj, ni)),
                np.zeros((nj, ni)))
    rc, steps, res = s.run_to_steady(1e-8, 4000000, timeout_s=400.0)
    assert rc == capi.OK, (rc, steps, res)
    heat, perim = s.wall_heat(2)
    nu_cyl = heat / (chi * perim)
    assert nu_cyl == pytest.approx(gold["Nu"], rel=0.01)
    _, u, v, _ = s.get_state()
    up, lo = post.separation_angle(X, Y, u, v)
    assert up == pytest.approx(lo, abs=1e-3)  # the aiding flow is symmetric
    assert abs(up - gold["theta_s_deg"]) < 1.2
    s.close()
