"""CUDA path against the FP64 oracle, element by element, through the C ABI.

Tolerances (relative to max(max|ref|, floor); floors: rho 1, u and v the
velocity scale of the case, T the temperature difference):
  FP64: <= 1e-12 after one step, <= 1e-11 after tens of steps, <= 1e-10 at
        the steady state;
  FP32 (rho - 1 stored): <= 1e-5 on u, v, T, and on the density deviation
        |rho_gpu - rho_ref| / max(max|rho_ref - 1|, Ma^2) <= 1e-5 with
        Ma = 0.1 (the weakly compressible density scales with Ma^2).
Cases span several tiles with ragged tails, every boundary kind,
stretched and irregular meshes, degenerate 1-cell meshes, and the full
512 x 512 tanh mesh of the Ra = 1e8 cavity.
"""
import numpy as np
import pytest

from paper_2202_13449_gb300 import capi, inputs

pytestmark = pytest.mark.gpu

D, A, P = capi.WALL_DIRICHLET, capi.WALL_ADIABATIC, capi.PERIODIC
TOL = {capi.FP64: 1e-12, capi.FP32: 1e-5}


def rel(a, b, floor):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(float(np.max(np.abs(b))), floor))


MA2 = 0.1 ** 2


def rho_rel(got, ref, ma2=MA2):
    """FP32 density error on the deviation rho - 1, against max(|rho - 1|, Ma^2)."""
    d = np.abs(np.asarray(got) - np.asarray(ref))
    return float(np.max(d) / max(float(np.max(np.abs(np.asarray(ref) - 1.0))), ma2))


def make_pair(orc, xf, yf, nu, chi, beta_g, dt, kappa, kinds, bcT, bcU, precision,
              fx=0.0, fy=0.0, T_ref=0.5):
    p = orc.Problem(xf=xf, yf=yf, nu=nu, chi=chi, beta_g=beta_g, T_ref=T_ref, dt=dt,
                    kappa=kappa, fx=fx, fy=fy, bc_kind=kinds, bc_T=bcT, bc_u=bcU)
    s = capi.Solver(xf, yf, precision)
    s.set_params_ref(1e3, 0.71, 0.1, dt, 1.0, 1.0, T_ref)
    s.set_physics(nu, chi, beta_g)
    s.set_lattice(kappa)
    s.set_body_force(fx, fy)
    for side in range(4):
        s.set_bc(side, kinds[side], bcT[side], bcU[side])
    return p, s


CASES = {
    # name: (nx, ny, mesh, kinds, bcT, bcU, kappa, beta_g)
    "cavity_irregular_lid": (37, 21, "random", (D, D, A, A), (1, 0, 0, 0), (0, 0, 0, 0.01), 1.0, 2e-3),
    "rb_periodic_x_stretched_y": (45, 17, "tanh_y", (P, P, D, D), (0, 0, 1, 0), (0, 0, 0, 0), 0.7, 1e-3),
    "all_periodic": (33, 9, "uniform", (P, P, P, P), (0, 0, 0, 0), (0, 0, 0, 0), 1.0, 5e-4),
    "periodic_y_walls_x": (19, 26, "random", (D, A, P, P), (0.8, 0, 0, 0), (0.005, 0, 0, 0), 0.55, 1e-3),
    "tiny_1x1": (1, 1, "uniform", (D, D, A, A), (1, 0, 0, 0), (0, 0, 0, 0), 1.0, 1e-3),
    "tiny_1x5": (1, 5, "random", (D, A, D, A), (1, 0, 0.2, 0), (0, 0, 0, 0.01), 1.0, 1e-3),
    "tiny_5x1_periodic": (5, 1, "uniform", (P, P, D, D), (0, 0, 1, 0), (0, 0, 0, 0), 0.8, 1e-3),
    "two_by_three": (2, 3, "random", (A, D, A, D), (0, 0.3, 0, 0.9), (0.02, 0, 0, 0), 1.0, 1e-3),
}


def case_mesh(name, nx, ny, mesh):
    if mesh == "uniform":
        return inputs.uniform_faces(nx), inputs.uniform_faces(ny)
    if mesh == "tanh_y":
        import oracle
        return inputs.uniform_faces(nx), oracle.tanh_faces(ny, float(ny), 2.0)
    seed = sum(map(ord, name))
    return inputs.random_faces(nx, seed), inputs.random_faces(ny, seed + 1)


KERNELS = [0, 1]  # warp-marching strips, shared-memory tiles


def run_case(orc, name, precision, nsteps, kernel=0, chunk_rows=0):
    nx, ny, mesh, kinds, bcT, bcU, kappa, bg = CASES[name]
    xf, yf = case_mesh(name, nx, ny, mesh)
    p, s = make_pair(orc, xf, yf, nu=0.04, chi=0.05, beta_g=bg, dt=0.25, kappa=kappa,
                     kinds=kinds, bcT=bcT, bcU=bcU, precision=precision)
    s.set_schedule(kernel, chunk_rows)
    st = inputs.perturbed_state(nx, ny, seed=7 + nx * 31 + ny)
    ref, _, rc = orc.step(p, st, nsteps)
    assert rc == 0
    s.set_state(*st)
    s.step(nsteps)
    got = s.get_state()
    res_gpu, steps = s.residual()
    s.close()
    assert steps == nsteps
    return ref, got, res_gpu


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("precision", [capi.FP64, capi.FP32])
def test_single_step_matches_oracle(orc, name, precision, kernel):
    ref, got, _ = run_case(orc, name, precision, 1, kernel)
    tol = TOL[precision]
    if precision == capi.FP64:
        assert rel(got[0], ref[0], 1.0) < tol
    else:
        assert rho_rel(got[0], ref[0]) < tol, rho_rel(got[0], ref[0])
    for q in (1, 2):
        assert rel(got[q], ref[q], 1e-2) < tol, (q, rel(got[q], ref[q], 1e-2))
    assert rel(got[3], ref[3], 1.0) < tol


TILE_HEIGHTS = [16, 14, 12, 10, 8, 4, 2]  # compiled tile heights of the FP32 tile kernel
TILE_HEIGHTS_FP64 = [16, 8, 4, 2]


@pytest.mark.parametrize("tile_h", TILE_HEIGHTS)
@pytest.mark.parametrize("name", ["cavity_irregular_lid", "rb_periodic_x_stretched_y",
                                  "periodic_y_walls_x", "all_periodic"])
def test_every_tile_height_matches_oracle_fp32(orc, name, tile_h):
    """Each compiled tile shape (ragged tails in both directions for these
    meshes) against the oracle after three steps."""
    ref, got, _ = run_case(orc, name, capi.FP32, 3, 1, tile_h)
    assert rho_rel(got[0], ref[0]) < 1e-5, rho_rel(got[0], ref[0])
    for q, floor in ((1, 1e-2), (2, 1e-2), (3, 1.0)):
        assert rel(got[q], ref[q], floor) < 1e-5, (q, rel(got[q], ref[q], floor))


@pytest.mark.parametrize("tile_h", TILE_HEIGHTS_FP64)
@pytest.mark.parametrize("name", ["cavity_irregular_lid", "rb_periodic_x_stretched_y",
                                  "periodic_y_walls_x", "tiny_1x5"])
def test_every_fp64_tile_height_matches_oracle(orc, name, tile_h):
    ref, got, _ = run_case(orc, name, capi.FP64, 3, 1, tile_h)
    for q, floor in ((0, 1.0), (1, 1e-2), (2, 1e-2), (3, 1.0)):
        assert rel(got[q], ref[q], floor) < 1e-12, (q, rel(got[q], ref[q], floor))


def test_tile_height_is_validated():
    xf = inputs.uniform_faces(8)
    for prec, bad in ((capi.FP32, 13), (capi.FP32, 32), (capi.FP64, 14)):
        s = capi.Solver(xf, xf, prec)
        with pytest.raises(RuntimeError):
            s.set_schedule(1, bad)
        s.set_schedule(1, 0)
        s.set_schedule(0, 13)  # any chunk height for the marching kernel
        s.close()


@pytest.mark.parametrize("kernel,chunk", [(0, 0), (0, 5), (1, 0)])
@pytest.mark.parametrize("name", ["cavity_irregular_lid", "rb_periodic_x_stretched_y",
                                  "periodic_y_walls_x"])
def test_thirty_steps_match_oracle_fp64(orc, name, kernel, chunk):
    ref, got, res = run_case(orc, name, capi.FP64, 30, kernel, chunk)
    for q, floor in ((0, 1.0), (1, 1e-2), (2, 1e-2), (3, 1.0)):
        assert rel(got[q], ref[q], floor) < 1e-11, (q, rel(got[q], ref[q], floor))


def test_residual_of_last_step_matches_oracle(orc):
    nx, ny, mesh, kinds, bcT, bcU, kappa, bg = CASES["cavity_irregular_lid"]
    xf, yf = case_mesh("cavity_irregular_lid", nx, ny, mesh)
    p, s = make_pair(orc, xf, yf, 0.04, 0.05, bg, 0.25, kappa, kinds, bcT, bcU, capi.FP64)
    st = inputs.perturbed_state(nx, ny, seed=99)
    _, (ru, rT), _ = orc.step(p, st, 3)
    s.set_state(*st)
    s.step(3)
    (gu, gT), steps = s.residual()
    s.close()
    assert gu == pytest.approx(ru, rel=1e-12) and gT == pytest.approx(rT, rel=1e-12)


def config2_pair(orc, precision):
    n = 512
    xf = orc.tanh_faces(n, float(n), 2.0)
    nu, chi, bg = orc.params_from_ra(1e8, 0.71, 0.1, float(n))
    dt = 0.5 * float(np.min(np.diff(xf)))
    return make_pair(orc, xf, xf.copy(), nu, chi, bg, dt, 1.0, (D, D, A, A), (1, 0, 0, 0),
                     (0, 0, 0, 0), precision)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("precision", [capi.FP64, capi.FP32])
def test_full_size_512_tanh_cavity_one_step(orc, precision, kernel):
    """The Ra = 1e8, 512 x 512, tanh (phi = 2) cavity: one step from a
    generic state, every cell compared."""
    p, s = config2_pair(orc, precision)
    s.set_schedule(kernel, 0)
    st = inputs.perturbed_state(512, 512, seed=2024, amp_u=0.05)
    ref, _, rc = orc.step(p, st, 1)
    s.set_state(*st)
    s.step(1)
    got = s.get_state()
    s.close()
    tol = TOL[precision]
    for q, floor in ((1, 0.1), (2, 0.1), (3, 1.0)):
        assert rel(got[q], ref[q], floor) < tol, (q, rel(got[q], ref[q], floor))


@pytest.mark.parametrize("precision", [capi.FP64, capi.FP32])
def test_config2_checkpoints_match_oracle(orc, precision):
    """The config-2 run itself (512 x 512 tanh, Ra = 1e8, conduction start)
    against the oracle at steps 1, 10 and 100, with the schedule the
    autotuner picks: fields and the mean wall Nusselt number."""
    p, s = config2_pair(orc, precision)
    st = inputs.conduction_state(p.xf, p.yf)
    s.set_state(*st)
    s.autotune(16)
    ref, done = st, 0
    for cp in (1, 10, 100):
        ref, _, rc = orc.step(p, ref, cp - done)
        assert rc == 0
        s.step(cp - done)
        done = cp
        got = s.get_state()
        tol = 1e-11 if precision == capi.FP64 else 1e-5
        for q, floor in ((1, 0.1), (2, 0.1), (3, 1.0)):
            assert rel(got[q], ref[q], floor) < tol, (cp, q, rel(got[q], ref[q], floor))
        nu_ref = 0.5 * (orc.nusselt(p, ref, 0) + orc.nusselt(p, ref, 1))
        nu_gpu = 0.5 * (s.nusselt(capi.NU_WEST) + s.nusselt(capi.NU_EAST))
        assert abs(nu_gpu - nu_ref) / abs(nu_ref) < (1e-10 if precision == capi.FP64 else 1e-4)
    s.close()


@pytest.mark.parametrize("kernel", KERNELS)
def test_mass_conserved_to_round_off_on_gpu(orc, kernel):
    nx, ny = 40, 24
    xf, yf = inputs.random_faces(nx, 5), inputs.random_faces(ny, 6)
    _, s = make_pair(orc, xf, yf, 0.03, 0.04, 2e-3, 0.3, 1.0, (D, D, A, A), (1, 0, 0, 0),
                     (0, 0, 0, 0), capi.FP64)
    s.set_schedule(kernel, 7 if kernel == 0 else 0)
    st = inputs.perturbed_state(nx, ny, seed=11)
    dV = np.outer(np.diff(yf), np.diff(xf))
    m0 = float(np.sum(st[0] * dV))
    s.set_state(*st)
    s.step(500)
    m1 = float(np.sum(s.get_state()[0] * dV))
    s.close()
    assert abs(m1 - m0) / m0 < 1e-13


def cavity_solver(orc, n, Ra, precision):
    p = orc.cavity_problem(n, Ra)
    s = capi.Solver(p.xf, p.yf, precision)
    s.set_params(Ra, 0.71, 0.1, p.dt)
    return p, s


def test_config1_run_to_steady_fp64(orc):
    """64 x 64, Ra = 1e3, to max(R_u, R_T) < 1e-8: the GPU stops on the same
    step as the oracle and the steady fields agree to 1e-10."""
    p, s = cavity_solver(orc, 64, 1e3, capi.FP64)
    st0 = inputs.conduction_state(p.xf, p.yf)
    ref, n_ref, res_ref, rc = orc.run_to_steady(p, st0, 1e-8, 400000)
    assert rc == 0
    rc, n_gpu, res_gpu = s.run_to_steady(1e-8, 400000)
    assert rc == capi.OK
    assert abs(n_gpu - n_ref) <= 1, (n_gpu, n_ref)
    if n_gpu != n_ref:  # compare at the oracle's step count
        s.set_state(*st0)
        s.step(n_ref)
    got = s.get_state()
    for q, floor in ((0, 1.0), (1, 0.1), (2, 0.1), (3, 1.0)):
        assert rel(got[q], ref[q], floor) < 1e-10, (q, rel(got[q], ref[q], floor))
    for which in (capi.NU_WEST, capi.NU_EAST, capi.NU_AVG, capi.NU_HALF):
        assert s.nusselt(which) == pytest.approx(orc.nusselt(p, ref, which), rel=1e-10)
    s.close()


@pytest.mark.parametrize("kernel", KERNELS)
def test_config1_fp32_against_fp64_oracle(orc, kernel):
    """FP32 bulk with FP64 reductions on the same case: fields within 1e-5 and
    the mean wall Nusselt number within 1e-4 of the FP64 oracle."""
    p, s = cavity_solver(orc, 64, 1e3, capi.FP32)
    s.set_schedule(kernel, 0)
    st0 = inputs.conduction_state(p.xf, p.yf)
    ref, n_ref, _, rc = orc.run_to_steady(p, st0, 1e-8, 400000)
    assert rc == 0
    s.step(n_ref)
    got = s.get_state()
    for q, floor in ((1, 0.1), (2, 0.1), (3, 1.0)):
        assert rel(got[q], ref[q], floor) < 1e-5, (q, rel(got[q], ref[q], floor))
    nu_ref = 0.5 * (orc.nusselt(p, ref, 0) + orc.nusselt(p, ref, 1))
    nu_gpu = 0.5 * (s.nusselt(capi.NU_WEST) + s.nusselt(capi.NU_EAST))
    assert abs(nu_gpu - nu_ref) / nu_ref < 1e-4
    s.close()


@pytest.mark.parametrize("precision", [capi.FP64, capi.FP32])
def test_nusselt_of_generic_state(orc, precision):
    nx, ny = 38, 22
    xf, yf = inputs.random_faces(nx, 71), inputs.random_faces(ny, 72)
    p, s = make_pair(orc, xf, yf, 0.03, 0.05, 1e-3, 0.3, 0.9, (D, D, D, D), (1, 0, 0.7, 0.2),
                     (0, 0, 0, 0), precision)
    st = inputs.perturbed_state(nx, ny, seed=73)
    s.set_state(*st)
    tol = 1e-12 if precision == capi.FP64 else 1e-4
    for which in range(6):
        want = orc.nusselt(p, st, which)
        got = s.nusselt(which)
        assert abs(got - want) <= tol * max(abs(want), 1.0), (which, got, want)
    s.close()


def test_nan_state_fp64_reports_divergence(orc):
    """Host-side fault injection: a NaN in the uploaded FP64 state makes the
    step return RTLBFS_ERR_DIVERGED; the handle stays usable."""
    p, s = cavity_solver(orc, 16, 1e4, capi.FP64)
    st = list(inputs.conduction_state(p.xf, p.yf))
    st[3] = st[3].copy()
    st[3][5, 5] = np.nan
    s.set_state(*st)
    with pytest.raises(capi.RTLBFSError) as e:
        s.step(10)
    assert e.value.rc == capi.ERR_DIVERGED
    s.set_state(*inputs.conduction_state(p.xf, p.yf))
    s.step(10)
    assert np.all(np.isfinite(s.get_state()[3]))
    s.close()


def test_nan_state_fp32_is_rejected_at_upload(orc):
    """The fixed-point FP32 state cannot hold NaN or out-of-range values: the
    upload says so instead of storing a wrapped integer."""
    p, s = cavity_solver(orc, 16, 1e4, capi.FP32)
    st = list(inputs.conduction_state(p.xf, p.yf))
    st[3] = st[3].copy()
    st[3][5, 5] = np.nan
    with pytest.raises(capi.RTLBFSError) as e:
        s.set_state(*st)
    assert e.value.rc == capi.ERR_ARG
    st[3][5, 5] = 0.5
    st[1] = st[1].copy()
    st[1][2, 2] = 1.5  # |u| >= 0.99 is outside the representable range
    with pytest.raises(capi.RTLBFSError):
        s.set_state(*st)
    s.close()


@pytest.mark.parametrize("precision", [capi.FP64, capi.FP32])
def test_blow_up_is_reported_as_divergence(orc, precision):
    """An unstable time step: the run stops with RTLBFS_ERR_DIVERGED (NaN in
    FP64, a field leaving its range in the fixed-point FP32 state)."""
    p, s = cavity_solver(orc, 16, 1e6, precision)
    s.set_params(1e6, 0.71, 0.1, 40.0)
    rc, n, _ = s.run_to_steady(1e-8, 5000)
    assert rc == capi.ERR_DIVERGED
    assert n < 5000
    s.close()


def test_run_controls(orc):
    p, s = cavity_solver(orc, 16, 1e4, capi.FP64)
    rc, n, _ = s.run_to_steady(1e-8, 0)
    assert rc == capi.ERR_NOT_CONVERGED and n == 0
    rc, n, _ = s.run_to_steady(1e-30, 300)
    assert rc == capi.ERR_NOT_CONVERGED and n == 300
    (r, _), steps = s.residual()
    assert steps == 300
    s.step(0)
    assert s.residual()[1] == 300
    s.close()


def test_autotune_keeps_the_state(orc):
    """The autotuner times schedules on a snapshot: afterwards the state,
    step counter and results are those of an untuned run."""
    p, s = cavity_solver(orc, 96, 1e5, capi.FP64)
    s.step(7)
    before = s.get_state()
    (_, _), steps = s.residual()
    kernel, rows, ms = s.autotune(16)
    assert kernel in (0, 1, 2) and ms > 0
    after = s.get_state()
    assert s.residual()[1] == steps
    for a, b in zip(before, after):
        np.testing.assert_array_equal(a, b)
    s.step(5)
    ref, _, _ = orc.step(p, before, 5)
    got = s.get_state()
    for q, floor in ((1, 0.1), (2, 0.1), (3, 1.0)):
        assert rel(got[q], ref[q], floor) < 1e-12
    s.close()


@pytest.mark.parametrize("kernel", KERNELS)
def test_fp32_hot_wall_next_to_cold_fluid(orc, kernel):
    """A Dirichlet wall far from the fluid beside it (T_w = 1 next to T near
    0): the ghost's mirror temperature 2 T_w - T_P is about 2, beyond the
    range of a stored FP32 temperature; the kernels form it relative to a
    temperature inside the tile, so the step still matches the oracle."""
    nx, ny = 40, 24
    xf, yf = inputs.random_faces(nx, 5), inputs.random_faces(ny, 6)
    p, s = make_pair(orc, xf, yf, nu=0.04, chi=0.05, beta_g=2e-3, dt=0.25, kappa=1.0,
                     kinds=(D, D, A, D), bcT=(1.0, 0.0, 0.0, 1.0), bcU=(0.0, 0.0, 0.0, 0.0),
                     precision=capi.FP32)
    s.set_schedule(kernel, 0)
    rho, u, v, T = inputs.perturbed_state(nx, ny, seed=3)
    st = (rho, u, v, T - 0.5)
    ref, _, rc = orc.step(p, st, 3)
    assert rc == 0
    s.set_state(*st)
    s.step(3)
    got = s.get_state()
    s.close()
    assert rho_rel(got[0], ref[0]) < 1e-5, rho_rel(got[0], ref[0])
    for q, floor in ((1, 1e-2), (2, 1e-2), (3, 1.0)):
        assert rel(got[q], ref[q], floor) < 1e-5, q


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("precision", [capi.FP64, capi.FP32])
def test_temperatures_outside_the_unit_interval(orc, precision, kernel):
    """Walls at T = 5 and -5 (dT = 10, T_ref = 0 through set_params_ref) and a
    state with |T| up to 4: beyond the FP32 state's +-1.98 at T_unit = 1, so
    the FP32 handle stores T / 4.  Fields after 1 and 5 steps and the wall
    Nusselt numbers against the oracle (T floor dT = 10)."""
    nx, ny = 37, 21
    xf, yf = inputs.random_faces(nx, 501), inputs.random_faces(ny, 502)
    bcT = (5.0, -5.0, 0.0, 0.0)
    nu, chi, bg, dt = 0.04, 0.05, 2e-5, 0.25
    p = orc.Problem(xf=xf, yf=yf, nu=nu, chi=chi, beta_g=bg, T_ref=0.0, dT=10.0, dt=dt,
                    bc_kind=(D, D, A, A), bc_T=bcT)
    s = capi.Solver(xf, yf, precision)
    s.set_params_ref(1e3, 0.71, 0.1, dt, 1.0, 10.0, 0.0)
    s.set_physics(nu, chi, bg)
    for side in range(4):
        s.set_bc(side, (D, D, A, A)[side], bcT[side], 0.0)
    s.set_schedule(kernel, 0)
    st = inputs.perturbed_state(nx, ny, seed=503, amp_T=4.0, T_mean=0.0)
    s.set_state(*st)
    ref, done = st, 0
    tol = TOL[precision]
    for n in (1, 5):
        ref, _, rc = orc.step(p, ref, n - done)
        assert rc == 0
        s.step(n - done)
        done = n
        got = s.get_state()
        if precision == capi.FP32:
            assert rho_rel(got[0], ref[0]) < tol, rho_rel(got[0], ref[0])
        for q, floor in ((1, 1e-2), (2, 1e-2), (3, 10.0)):
            assert rel(got[q], ref[q], floor) < tol, (n, q, rel(got[q], ref[q], floor))
    for which, side in ((capi.NU_WEST, orc.NU_W), (capi.NU_EAST, orc.NU_E)):
        want = orc.nusselt(p, ref, side)
        ntol = 1e-10 if precision == capi.FP64 else 1e-4
        assert abs(s.nusselt(which) - want) <= ntol * max(1.0, abs(want))
    s.close()


def test_fp32_temperature_unit_follows_the_configuration(orc):
    """The FP32 state's temperature unit grows when a wall is set hotter than
    the stored range allows: stepping then matches a handle set up with that
    wall from the start.  A NaN state is still rejected."""
    nx, ny = 24, 18
    xf, yf = inputs.uniform_faces(nx), inputs.uniform_faces(ny)
    st = inputs.perturbed_state(nx, ny, seed=601, amp_T=0.5, T_mean=0.5)
    a = capi.Solver(xf, yf, capi.FP32)
    a.set_state(*st)      # unit 1: walls 1 / 0
    a.set_bc(capi.WEST, D, 6.0, 0.0)  # now needs unit 4: the state is rescaled
    a.step(3)
    b = capi.Solver(xf, yf, capi.FP32)
    b.set_bc(capi.WEST, D, 6.0, 0.0)
    b.set_state(*st)
    b.step(3)
    ga, gb = a.get_state(), b.get_state()
    for q, floor in ((1, 1e-2), (2, 1e-2), (3, 6.0)):
        assert rel(ga[q], gb[q], floor) < 1e-6, q
    bad = list(st)
    bad[3] = bad[3].copy()
    bad[3][3, 4] = np.nan
    with pytest.raises(RuntimeError):
        b.set_state(*bad)
    a.close()
    b.close()
