"""Checkpoint/resume and wall-clock limits of the handle API, on the GPU.

* A state taken with rtlbfs_get_state_raw after some steps and restored
  into a fresh handle with rtlbfs_set_state_raw continues bit for bit like
  the uninterrupted run, in both precisions (the cell records are copied,
  not converted); in FP32 the FP64 planes of rtlbfs_get_state /
  rtlbfs_set_state are exact too (fixed-point values convert to doubles and
  back without rounding).
* rtlbfs_run_to_steady with a wall-clock limit shorter than one chunk of
  steps returns RTLBFS_ERR_TIMEOUT after that chunk, and the handle keeps
  working.
"""
import numpy as np
import pytest

from paper_2202_13449_gb300 import capi, inputs

pytestmark = pytest.mark.gpu


def cavity(precision, n=48, phi=1.5):
    xf = capi.tanh_faces(n, float(n), phi)
    s = capi.Solver(xf, xf, precision)
    s.set_params(1e5, 0.71, 0.1, 0.0)
    return s


@pytest.mark.parametrize("precision", [capi.FP64, capi.FP32])
def test_raw_checkpoint_resumes_bit_for_bit(precision):
    a = cavity(precision)
    a.step(40)
    rec, tu = a.get_state_raw()
    assert rec.size == a.raw_bytes() == a.nx * a.ny * (32 if precision == capi.FP64 else 16)
    a.step(25)
    want = a.get_state()
    b = cavity(precision)
    b.set_state_raw(rec, tu)
    b.step(25)
    got = b.get_state()
    for q in range(4):
        np.testing.assert_array_equal(got[q], want[q])
    # and the records themselves after the same steps
    np.testing.assert_array_equal(a.get_state_raw()[0], b.get_state_raw()[0])
    a.close()
    b.close()


def test_fp32_plane_checkpoint_is_exact_too():
    a = cavity(capi.FP32)
    a.step(40)
    st = a.get_state()
    a.step(25)
    want = a.get_state()
    b = cavity(capi.FP32)
    b.set_state(*st)
    b.step(25)
    got = b.get_state()
    for q in range(4):
        np.testing.assert_array_equal(got[q], want[q])
    a.close()
    b.close()


def test_raw_records_keep_their_temperature_unit():
    """FP32 records stored with T_unit = 4 (walls at +-5) restored into a
    handle configured the same way: the same fields; a bad unit is refused."""
    xf = inputs.uniform_faces(24)
    a = capi.Solver(xf, xf, capi.FP32)
    a.set_bc(capi.WEST, capi.WALL_DIRICHLET, 5.0, 0.0)
    a.set_bc(capi.EAST, capi.WALL_DIRICHLET, -5.0, 0.0)
    a.set_state(*inputs.perturbed_state(24, 24, seed=9, amp_T=3.0, T_mean=0.0))
    a.step(10)
    rec, tu = a.get_state_raw()
    assert tu == 4.0
    b = capi.Solver(xf, xf, capi.FP32)
    b.set_bc(capi.WEST, capi.WALL_DIRICHLET, 5.0, 0.0)
    b.set_bc(capi.EAST, capi.WALL_DIRICHLET, -5.0, 0.0)
    b.set_state_raw(rec, tu)
    ga, gb = a.get_state(), b.get_state()
    for q in range(4):
        np.testing.assert_array_equal(ga[q], gb[q])
    with pytest.raises(RuntimeError):
        b.set_state_raw(rec, 3.0)  # not a power of two
    a.close()
    b.close()


def test_run_to_steady_stops_at_its_wall_clock_limit():
    s = cavity(capi.FP64, n=96)
    rc, steps, res = s.run_to_steady(1e-12, 10_000_000, timeout_s=1e-6)
    assert rc == capi.ERR_TIMEOUT
    assert 0 < steps < 10_000_000  # stopped after the first chunk of steps
    assert np.isfinite(res[0]) and np.isfinite(res[1])
    # the handle keeps working after the timeout
    s.step(3)
    (_, _), total = s.residual()
    assert total == steps + 3
    s.close()
