"""The persistent tile kernel (schedule kernel 2) through the C ABI.

It runs the launch-per-step tile kernel's arithmetic (the same tile_step) in
one cooperative launch per chunk of steps, each tile waiting only for the
eight tiles around it.  Checked here:
  - bit-identical fields and step counts to the tile kernel at
    the same tile height (FP64 and FP32, walls, periodic sides, ragged
    tiles, the full 512 x 512 bench mesh), residuals equal to rounding (their
    FP64 block sums are added in arrival order in both kernels);
  - the FP64 oracle within the parity tolerances;
  - the same stop step as the oracle and the tile kernel under
    run_to_steady, and exact step counts for any number of steps;
  - meshes it cannot take are refused with ERR_ARG;
  - its bounded waits: a tile that never reports progress makes the step
    fail with ERR_CUDA within seconds, and the context stays usable.
"""
import time

import numpy as np
import pytest

from paper_2202_13449_gb300 import capi, inputs
from test_gpu_parity import CASES, TOL, case_mesh, cavity_solver, make_pair, rel

pytestmark = pytest.mark.gpu

HEIGHTS = {capi.FP32: [16, 14, 12, 10, 8, 4, 2], capi.FP64: [16, 8, 4, 2]}
ELIGIBLE = ["cavity_irregular_lid", "rb_periodic_x_stretched_y", "periodic_y_walls_x",
            "two_by_three"]


def heights_for(nx, ny, precision):
    """Tile heights the persistent kernel takes for an nx x ny mesh."""
    if nx % 32 == 1:
        return []
    return [h for h in HEIGHTS[precision] if ny % h != 1]


def solver_for(orc, name, precision, kernel, h):
    nx, ny, mesh, kinds, bcT, bcU, kappa, bg = CASES[name]
    xf, yf = case_mesh(name, nx, ny, mesh)
    p, s = make_pair(orc, xf, yf, nu=0.04, chi=0.05, beta_g=bg, dt=0.25, kappa=kappa,
                     kinds=kinds, bcT=bcT, bcU=bcU, precision=precision)
    s.set_schedule(kernel, h)
    st = inputs.perturbed_state(nx, ny, seed=7 + nx * 31 + ny)
    s.set_state(*st)
    return p, s, st


def run(orc, name, precision, kernel, h, nsteps):
    p, s, st = solver_for(orc, name, precision, kernel, h)
    s.step(nsteps)
    got = s.get_state()
    res, steps = s.residual()
    s.close()
    return got, res, steps, p, st


@pytest.mark.parametrize("name", ELIGIBLE)
@pytest.mark.parametrize("precision", [capi.FP64, capi.FP32])
def test_bit_identical_to_the_tile_kernel(orc, name, precision):
    nx, ny = CASES[name][:2]
    hs = heights_for(nx, ny, precision)
    if not hs:
        pytest.skip("no tile height the persistent kernel takes for this mesh")
    for h in (hs[0], hs[-1]):
        a = run(orc, name, precision, 1, h, 25)
        b = run(orc, name, precision, 2, h, 25)
        for x, y in zip(a[0], b[0]):
            np.testing.assert_array_equal(x, y)
        # the residual's FP64 sums are added in arrival order: equal to rounding
        np.testing.assert_allclose(a[1], b[1], rtol=1e-12)
        assert a[2] == b[2] == 25


@pytest.mark.parametrize("name", ELIGIBLE)
def test_matches_the_oracle(orc, name):
    nx, ny = CASES[name][:2]
    for precision, nsteps in ((capi.FP64, 30), (capi.FP32, 3)):
        hs = heights_for(nx, ny, precision)
        if not hs:
            continue
        got, res, steps, p, st = run(orc, name, precision, 2, hs[0], nsteps)
        ref, rr, rc = orc.step(p, st, nsteps)
        assert rc == 0 and steps == nsteps
        tol = 1e-11 if precision == capi.FP64 else TOL[capi.FP32]
        for q, floor in ((1, 1e-2), (2, 1e-2), (3, 1.0)):
            assert rel(got[q], ref[q], floor) < tol, (precision, q, rel(got[q], ref[q], floor))
        if precision == capi.FP64:
            assert rel(got[0], ref[0], 1.0) < tol
            np.testing.assert_allclose(res, rr, rtol=1e-9)


@pytest.mark.parametrize("nsteps", [1, 2, 3, 7, 300])
def test_exact_step_counts(orc, nsteps):
    a = run(orc, "cavity_irregular_lid", capi.FP32, 1, 8, nsteps)
    b = run(orc, "cavity_irregular_lid", capi.FP32, 2, 8, nsteps)
    for x, y in zip(a[0], b[0]):
        np.testing.assert_array_equal(x, y)
    assert a[2] == b[2] == nsteps


def test_full_size_512_tanh_cavity(orc):
    """The bench mesh (512 x 512 tanh, Ra = 1e8, FP32) at its tile height, 20
    steps: the same bits as the tile kernel.  (In FP64 its 512 or more tiles
    do not fit on the GPU at once; that is refused, below.)"""
    out = []
    precision = capi.FP32
    for kernel in (1, 2):
        p = orc.cavity_problem(512, 1e8, phi=2.0)
        s = capi.Solver(p.xf, p.yf, precision)
        s.set_params(1e8, 0.71, 0.1, p.dt)
        s.set_schedule(kernel, 14)
        s.set_state(*inputs.conduction_state(p.xf, p.yf))
        s.step(20)
        out.append((s.get_state(), s.residual()))
        s.close()
    for x, y in zip(out[0][0], out[1][0]):
        np.testing.assert_array_equal(x, y)
    np.testing.assert_allclose(out[0][1][0], out[1][1][0], rtol=1e-12)
    assert out[0][1][1] == out[1][1][1] == 20


def test_run_to_steady_stops_on_the_same_step(orc):
    """64 x 64, Ra = 1e3, FP64, to max(R_u, R_T) < 1e-8: the persistent kernel
    stops where the tile kernel does (the oracle's step, within one), with
    the same fields; a step it takes past the stop is discarded."""
    p, s1 = cavity_solver(orc, 64, 1e3, capi.FP64)
    st0 = inputs.conduction_state(p.xf, p.yf)
    s1.set_schedule(1, 8)
    s1.set_state(*st0)
    rc1, n1, r1 = s1.run_to_steady(1e-8, 400000)
    _, s2 = cavity_solver(orc, 64, 1e3, capi.FP64)
    s2.set_schedule(2, 8)
    s2.set_state(*st0)
    rc2, n2, r2 = s2.run_to_steady(1e-8, 400000)
    assert rc1 == rc2 == capi.OK
    assert n1 == n2
    np.testing.assert_allclose(r1, r2, rtol=1e-12)
    for x, y in zip(s1.get_state(), s2.get_state()):
        np.testing.assert_array_equal(x, y)
    ref, n_ref, _, rc = orc.run_to_steady(p, st0, 1e-8, 400000)
    assert rc == 0 and abs(n2 - n_ref) <= 1
    s1.close()
    s2.close()


def test_meshes_it_cannot_take_are_refused(orc):
    # a last tile column one cell wide: its neighbours' halo reaches past it
    p, s, _ = solver_for(orc, "all_periodic", capi.FP32, 2, 8)  # 33 x 9
    with pytest.raises(capi.RTLBFSError) as e:
        s.step(1)
    assert e.value.rc == capi.ERR_ARG
    s.close()
    # FP64 on a 17-row mesh: every FP64 tile height leaves a 1-row tile
    p, s, _ = solver_for(orc, "rb_periodic_x_stretched_y", capi.FP64, 2, 0)
    with pytest.raises(capi.RTLBFSError) as e:
        s.step(1)
    assert e.value.rc == capi.ERR_ARG
    s.close()
    # FP64 512 x 512: more tiles than fit on the GPU at once
    p = orc.cavity_problem(512, 1e8, phi=2.0)
    s = capi.Solver(p.xf, p.yf, capi.FP64)
    s.set_params(1e8, 0.71, 0.1, p.dt)
    s.set_schedule(2, 16)
    with pytest.raises(capi.RTLBFSError) as e:
        s.step(1)
    assert e.value.rc == capi.ERR_ARG
    s.close()


def test_a_withheld_tile_stalls_the_step_with_a_status(orc):
    """Tile 3 never reports its progress: its neighbours' waits run out
    (about a second), the step returns ERR_CUDA, and the context still runs
    the next steps correctly."""
    p, s, st = solver_for(orc, "periodic_y_walls_x", capi.FP32, 2, 4)
    s.debug_withhold_tile(3)
    t0 = time.perf_counter()
    with pytest.raises(capi.RTLBFSError) as e:
        s.step(50)
    assert e.value.rc == capi.ERR_CUDA
    assert time.perf_counter() - t0 < 30.0
    s.debug_withhold_tile(-1)
    s.set_state(*st)
    s.step(10)
    got = s.get_state()
    s.close()
    ref = run(orc, "periodic_y_walls_x", capi.FP32, 1, 4, 10)[0]
    for x, y in zip(got, ref):
        np.testing.assert_array_equal(x, y)
