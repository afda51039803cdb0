"""3D CUDA path (include/rtlbfs3d.h) against the 3D FP64 oracle, element by
element, through the C ABI.

Tolerances (relative to max(max|ref|, floor); floors: rho 1, velocities the
velocity scale of the case, T the temperature difference), as for 2D:
  FP64: <= 1e-12 after one step, <= 1e-11 after tens of steps, <= 1e-10 at
        the steady state;
  FP32 (fixed-point state): <= 1e-5 on u, v, w, T and 1e-6 on rho;
  Nusselt numbers: <= 1e-12 (FP64) on generic states, <= 1e-4 (FP32) at the
  steady state.
Cases span several tiles and z-chunks with ragged tails for each of the
three tile shapes, every boundary kind on every axis, irregular and tanh
meshes, 1-cell axes, and the 80^3 tanh mesh of the cubic cavity of
Section 4.4 at full size.
"""
import numpy as np
import pytest

from paper_2202_13449_gb300 import capi, inputs

pytestmark = pytest.mark.gpu

D, A, P = capi.WALL_DIRICHLET, capi.WALL_ADIABATIC, capi.PERIODIC
VSCALE = 1e-2


def rel(a, b, floor):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(float(np.max(np.abs(b))), floor))


@pytest.fixture(scope="module")
def d3(orc):
    from oracle import d3 as mod
    return mod


BCU = ((0, 0.01, -0.02), (0, 0, 0), (0.015, 0, 0.01), (0, 0, 0), (0, 0, 0), (0.02, -0.01, 0))

CASES = {
    # name: (nx, ny, nz, mesh, kinds, bcT, g_axis, kappa)
    "cavity_irregular": (37, 11, 13, "random", (D, D, A, A, A, A), (0, 1, 0, 0, 0, 0), 2, 1.0),
    "mixed_walls_moving": (20, 9, 19, "random", (D, A, A, D, A, D), (0.9, 0, 0, 0.6, 0, 0.2), 1, 0.8),
    "periodic_x": (33, 7, 10, "random", (P, P, D, A, A, D), (0, 0, 0.7, 0, 0, 0.3), 2, 0.9),
    "periodic_y": (17, 21, 6, "random", (A, D, P, P, D, A), (0, 0.4, 0, 0, 0.8, 0), 0, 1.0),
    "periodic_z": (9, 12, 16, "tanh", (D, D, A, A, P, P), (1, 0, 0, 0, 0, 0), 1, 0.6),
    "all_periodic": (16, 8, 12, "uniform", (P, P, P, P, P, P), (0,) * 6, 2, 1.0),
    "tiny_1x1x1": (1, 1, 1, "uniform", (D, D, A, A, A, A), (0, 1, 0, 0, 0, 0), 2, 1.0),
    "tiny_2x3x1": (2, 3, 1, "random", (A, D, A, D, A, A), (0, 0.3, 0, 0.9, 0, 0), 2, 1.0),
    "tiny_1x5x2": (1, 5, 2, "random", (D, A, D, A, A, D), (1, 0, 0.2, 0, 0, 0.5), 1, 1.0),
}


def case_mesh(d3, name, n, mesh):
    if mesh == "uniform":
        return [inputs.uniform_faces(m) for m in n]
    if mesh == "tanh":
        return [d3.tanh_faces(m, float(m), 1.8) for m in n]
    seed = sum(map(ord, name))
    return [inputs.random_faces(m, seed + a) for a, m in enumerate(n)]


def make_pair(d3, faces, kinds, bcT, g_axis, kappa, precision, nu=0.04, chi=0.05, beta_g=2e-3,
              dt=0.2, force=(1e-4, -5e-5, 2e-5)):
    bcu = tuple(tuple(0.0 if c == s // 2 else BCU[s][c] for c in range(3)) for s in range(6))
    p = d3.Problem3(xf=faces[0], yf=faces[1], zf=faces[2], nu=nu, chi=chi, beta_g=beta_g,
                    T_ref=0.5, dt=dt, kappa=kappa, force=force, g_axis=g_axis, bc_kind=kinds,
                    bc_T=bcT, bc_u=bcu)
    s = capi.Solver3(*faces, precision=precision)
    s.set_params(1e3, 0.71, 0.1, dt)
    s.set_physics(nu, chi, beta_g)
    s.set_lattice(kappa)
    s.set_gravity_axis(g_axis)
    s.set_body_force(*force)
    for side in range(6):
        s.set_bc(side, kinds[side], bcT[side], bcu[side])
    return p, s


def compare(got, ref, tol, precision):
    floors = (1.0, VSCALE, VSCALE, VSCALE, 1.0)
    for q in range(5):
        if q == 0 and precision == capi.FP32:
            assert np.max(np.abs(got[0] - ref[0])) < 1e-6
            continue
        e = rel(got[q], ref[q], floors[q])
        assert e < tol, (q, e)


def run_case(d3, name, precision, nsteps, tile=0, kchunk=0, scheme=0):
    nx, ny, nz, mesh, kinds, bcT, g_axis, kappa = CASES[name]
    faces = case_mesh(d3, name, (nx, ny, nz), mesh)
    p, s = make_pair(d3, faces, kinds, bcT, g_axis, kappa, precision)
    p.scheme = scheme
    s.set_scheme(scheme)
    s.set_schedule(tile, kchunk)
    st = inputs.perturbed_state3(nx, ny, nz, seed=11 + nx * 31 + ny * 7 + nz)
    ref, res_ref, rc = d3.step(p, st, nsteps)
    assert rc == 0
    s.set_state(*st)
    s.step(nsteps)
    got = s.get_state()
    res_gpu, steps = s.residual()
    s.close()
    assert steps == nsteps
    return got, ref, res_gpu, res_ref


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("tile", [0, 1, 2])
def test_one_step_fp64(d3, name, tile):
    got, ref, rg, rr = run_case(d3, name, capi.FP64, 1, tile=tile, kchunk=3)
    compare(got, ref, 1e-12, capi.FP64)
    np.testing.assert_allclose(rg, rr, rtol=1e-9)


@pytest.mark.parametrize("name", ["cavity_irregular", "mixed_walls_moving", "periodic_z",
                                  "all_periodic", "tiny_1x5x2"])
def test_thirty_steps_fp64(d3, name):
    got, ref, _, _ = run_case(d3, name, capi.FP64, 30)
    compare(got, ref, 1e-11, capi.FP64)


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("tile", [0, 2])
def test_steps_fp32(d3, name, tile):
    got, ref, _, _ = run_case(d3, name, capi.FP32, 3, tile=tile, kchunk=4)
    compare(got, ref, 1e-5, capi.FP32)


@pytest.mark.parametrize("name", ["cavity_irregular", "mixed_walls_moving", "periodic_x",
                                  "periodic_z", "tiny_1x5x2"])
@pytest.mark.parametrize("tile", [0, 1, 2])
def test_tlbfs_one_step_fp64(d3, name, tile):
    """The TLBFS face stage (Section 2.2, D3Q19) against the oracle's."""
    got, ref, rg, rr = run_case(d3, name, capi.FP64, 1, tile=tile, kchunk=3, scheme=1)
    compare(got, ref, 1e-12, capi.FP64)
    np.testing.assert_allclose(rg, rr, rtol=1e-9)


@pytest.mark.parametrize("name", ["cavity_irregular", "periodic_y", "all_periodic"])
def test_tlbfs_steps(d3, name):
    got, ref, _, _ = run_case(d3, name, capi.FP64, 20, tile=1, scheme=1)
    compare(got, ref, 1e-11, capi.FP64)
    got, ref, _, _ = run_case(d3, name, capi.FP32, 3, tile=1, scheme=1)
    compare(got, ref, 1e-5, capi.FP32)


def test_tlbfs_nusselt_fp64(d3):
    name = "mixed_walls_moving"
    nx, ny, nz, mesh, kinds, bcT, g_axis, kappa = CASES[name]
    faces = case_mesh(d3, name, (nx, ny, nz), mesh)
    p, s = make_pair(d3, faces, kinds, bcT, g_axis, kappa, capi.FP64)
    p.scheme = 1
    s.set_scheme(1)
    st = inputs.perturbed_state3(nx, ny, nz, seed=15)
    s.set_state(*st)
    for side in range(6):
        for mid in (False, True):
            assert s.nusselt(side, mid) == pytest.approx(d3.nusselt(p, st, side, mid), rel=1e-12,
                                                         abs=1e-13), (side, mid)
    s.close()


@pytest.mark.parametrize("kchunk", [1, 2, 5, 0])
def test_z_chunking_does_not_change_the_result(d3, kchunk):
    got, ref, _, _ = run_case(d3, "mixed_walls_moving", capi.FP64, 4, tile=1, kchunk=kchunk)
    compare(got, ref, 1e-12, capi.FP64)


@pytest.mark.parametrize("name", ["cavity_irregular", "mixed_walls_moving", "periodic_y"])
def test_nusselt_fp64_generic_state(d3, name):
    nx, ny, nz, mesh, kinds, bcT, g_axis, kappa = CASES[name]
    faces = case_mesh(d3, name, (nx, ny, nz), mesh)
    p, s = make_pair(d3, faces, kinds, bcT, g_axis, kappa, capi.FP64)
    st = inputs.perturbed_state3(nx, ny, nz, seed=5)
    s.set_state(*st)
    for side in range(6):
        if kinds[side] == P:
            continue
        for mid in (False, True):
            want = d3.nusselt(p, st, side, mid)
            got = s.nusselt(side, mid)
            assert got == pytest.approx(want, rel=1e-12, abs=1e-13), (side, mid)
    if nx % 2 == 0:
        assert s.nusselt(capi.MID_X) == pytest.approx(d3.nusselt(p, st, d3.MID_PLANE_X), rel=1e-12)
    s.close()


def test_mass_conserved_on_the_gpu():
    n = (24, 18, 20)
    faces = [inputs.random_faces(m, 3 + a) for a, m in enumerate(n)]
    s = capi.Solver3(*faces, precision=capi.FP64)
    s.set_params(1e5, 0.71, 0.1, 0.0)
    st = inputs.perturbed_state3(*n, seed=9)
    s.set_state(*st)
    dV = np.einsum("k,j,i->kji", np.diff(faces[2]), np.diff(faces[1]), np.diff(faces[0]))
    m0 = np.sum(st[0] * dV)
    s.step(200)
    m1 = np.sum(s.get_state()[0] * dV)
    s.close()
    assert abs(m1 - m0) / m0 < 1e-13


def test_cubic_cavity_steady_state_matches_oracle(d3):
    """The Ra = 1e3 cubic cavity of Section 4.4 on 16^3 to a 1e-7 residual:
    FP64 stops on the oracle's step (+-1) with fields within 1e-10; FP32
    fields within 1e-5 and the wall Nusselt numbers within 1e-4."""
    n = 16
    p = d3.cubic_cavity(n, 1e3)
    st0 = inputs.conduction_state3(p.xf, p.yf, p.zf)
    ref, steps_ref, _, rc = d3.run_to_steady(p, st0, 1e-7, 100000)
    assert rc == 0
    nu_ref = [d3.nusselt(p, ref, side) for side in (0, 1)]
    num_ref = d3.nusselt(p, ref, 1, mid=True)
    for precision, tol in ((capi.FP64, 1e-10), (capi.FP32, 1e-5)):
        s = capi.Solver3(p.xf, p.yf, p.zf, precision=precision)
        s.set_params(1e3, 0.71, 0.1, p.dt)
        rc, steps, res = s.run_to_steady(1e-7, 100000)
        assert rc == capi.OK
        got = s.get_state()
        if precision == capi.FP64:
            assert abs(steps - steps_ref) <= 1
            compare(got, ref, tol, precision)
            for side, want in zip((0, 1), nu_ref):
                assert s.nusselt(side) == pytest.approx(want, rel=1e-10)
        else:
            for q in (1, 2, 3, 4):
                assert rel(got[q], ref[q], (1.0, VSCALE, VSCALE, VSCALE, 1.0)[q]) < tol
            for side, want in zip((0, 1), nu_ref):
                assert s.nusselt(side) == pytest.approx(want, rel=1e-4)
            assert s.nusselt(1, mid=True) == pytest.approx(num_ref, rel=1e-4)
        s.close()


def test_full_size_cubic_cavity_80_step(d3):
    """The Table 6 mesh (80^3, tanh phi = 1.8, Ra = 1e6) in the launch
    configuration the benchmark times: two steps from a perturbed state,
    every cell against the oracle, both precisions."""
    n = 80
    p = d3.cubic_cavity(n, 1e6, phi=1.8)
    st = inputs.perturbed_state3(n, n, n, seed=80)
    ref, _, rc = d3.step(p, st, 2)
    assert rc == 0
    for precision, tol in ((capi.FP64, 1e-12), (capi.FP32, 1e-5)):
        s = capi.Solver3(p.xf, p.yf, p.zf, precision=precision)
        s.set_params(1e6, 0.71, 0.1, p.dt)
        s.set_state(*st)
        s.step(2)
        compare(s.get_state(), ref, tol, precision)
        s.close()


def test_autotune_restores_the_state(d3):
    n = (40, 24, 30)
    faces = [inputs.random_faces(m, 21 + a) for a, m in enumerate(n)]
    s = capi.Solver3(*faces, precision=capi.FP32)
    st = inputs.perturbed_state3(*n, seed=4)
    s.set_state(*st)
    s.step(3)
    before = s.get_state()
    tile, ms = s.autotune(4)
    assert tile in (0, 1, 2) and ms > 0
    after = s.get_state()
    for a, b in zip(before, after):
        np.testing.assert_array_equal(a, b)
    (_, _), steps = s.residual()
    assert steps == 3
    s.close()


def test_errors_are_status_codes():
    n = (6, 5, 4)
    faces = [inputs.uniform_faces(m) for m in n]
    st = list(inputs.perturbed_state3(*n, seed=2))
    st[1] = st[1].copy()
    st[1][1, 2, 3] = np.nan
    s = capi.Solver3(*faces, precision=capi.FP64)
    s.set_state(*st)
    assert s.step_rc(2) == capi.ERR_DIVERGED
    s.close()
    s = capi.Solver3(*faces, precision=capi.FP32)
    with pytest.raises(capi.RTLBFSError) as e:
        s.set_state(*st)
    assert e.value.rc == capi.ERR_ARG
    with pytest.raises(capi.RTLBFSError):
        s.set_bc(7, D)
    with pytest.raises(capi.RTLBFSError):
        s.nusselt(capi.MID_X, mid=True)
    s.close()


@pytest.mark.slow
def test_table5_ra1e6_on_the_paper_mesh():
    """Physics of the GPU path at the paper's own 3D setting (Section 4.4,
    Table 5): 80^3 cells, Eq. 74 with phi = 1.8, Ra = 1e6, Pr = 0.71,
    V_c = 0.1, run to a 1e-7 residual in FP32 (about 4.7e5 steps, some 40 s).
    The oracle cannot run this to a steady state, so the check is against
    the printed values: Nu_o and Nu_m within 0.5 %, the velocity maxima
    within 2 % and their positions within a cell.  The lattice spacing is
    half the smaller normal width (kappa = 0.5): with kappa = 1 this mesh
    diverges after about 5e3 steps in both precisions."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                       "table5_cubic_cavity.json")))["Ra1e6"]
    n = 80
    f = capi.tanh_faces(n, float(n), 1.8)
    s = capi.Solver3(f, f, f, capi.FP32)
    s.set_params(1e6, 0.71, 0.1, 0.5 * float(np.min(np.diff(f))))
    s.set_lattice(0.5)
    rc, steps, res = s.run_to_steady(1e-7, 800000, timeout_s=300.0)
    assert rc == capi.OK, (rc, steps, res)
    st = s.get_state()
    nu_hot, nu_cold = -s.nusselt(capi.XP), -s.nusselt(capi.XM)
    assert nu_cold == pytest.approx(nu_hot, rel=1e-4)
    assert nu_hot == pytest.approx(gold["Nu_o"], rel=5e-3)
    assert -s.nusselt(capi.XP, mid=True) == pytest.approx(gold["Nu_m"], rel=5e-3)
    h = n // 2
    u_line = 0.25 * (st[1][:, h - 1, h - 1] + st[1][:, h - 1, h] + st[1][:, h, h - 1]
                     + st[1][:, h, h])
    w_line = 0.25 * (st[3][h - 1, h - 1, :] + st[3][h - 1, h, :] + st[3][h, h - 1, :]
                     + st[3][h, h, :])
    c = 0.5 * (f[1:] + f[:-1]) / n
    assert u_line.max() / 0.1 == pytest.approx(gold["u_max_over_Vc"], rel=0.02)
    assert w_line.max() / 0.1 == pytest.approx(gold["w_max_over_Vc"], rel=0.02)
    w_cells = np.diff(f) / n
    iu, iw = int(u_line.argmax()), int(w_line.argmax())
    assert abs(c[iu] - gold["u_max_z_over_L"]) < w_cells[iu]
    assert abs(c[iw] - gold["w_max_x_over_L"]) < w_cells[iw]
    s.close()


def test_fp32_hot_wall_next_to_cold_fluid(d3):
    """The hot wall (T = 1) next to fluid near T = 0: the mirror temperature
    is beyond a stored FP32 value's range; the kernel forms it relative to a
    temperature inside the unit, so the step still matches the oracle."""
    n = (20, 9, 11)
    faces = [inputs.random_faces(m, 31 + a) for a, m in enumerate(n)]
    p, s = make_pair(d3, faces, (D, D, A, A, A, D), (0.0, 1.0, 0, 0, 0, 1.0), 2, 1.0, capi.FP32)
    rho, u, v, w, T = inputs.perturbed_state3(*n, seed=8)
    st = (rho, u, v, w, T - 0.5)
    ref, _, rc = d3.step(p, st, 3)
    assert rc == 0
    s.set_state(*st)
    s.step(3)
    compare(s.get_state(), ref, 1e-5, capi.FP32)
    s.close()
