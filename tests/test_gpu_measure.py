"""The FMA-rate probe that the ALU rooflines are stated against, on the GPU.

rtlbfs_fma_rate times independent FMA chains on every SM.  Checked here:
the three kinds return finite positive rates below the unit-count bound
(SMs x FP32 lanes x the SM clock, FP64 far below FP32), the packed FP32x2
kind retires at least as many FMAs per second as the scalar one (two per
instruction at the same pipe rate), the rate does not depend on the loop
length once launch overhead is amortised, and bad arguments are refused.
"""
import pytest

from paper_2202_13449_gb300 import capi

pytestmark = pytest.mark.gpu


def _bound():
    import torch
    p = torch.cuda.get_device_properties(0)
    # 128 FP32 lanes per SM on this architecture; a generous 2.5 GHz clock
    return p.multi_processor_count * 128 * 2.5e9


def test_rates_are_positive_and_below_the_unit_bound():
    bound = _bound()
    f32, ms32 = capi.fma_rate(capi.RATE_FP32, 20000)
    f2, ms2 = capi.fma_rate(capi.RATE_FP32X2, 20000)
    f64, ms64 = capi.fma_rate(capi.RATE_FP64, 500)
    for r, ms in ((f32, ms32), (f2, ms2), (f64, ms64)):
        assert r > 0.0 and ms > 0.0
    assert f32 < bound and f2 < 2.0 * bound
    assert f64 < 0.25 * f32  # the narrow FP64 units
    assert f2 >= 0.9 * f32  # two FMAs per packed instruction


def test_rate_is_independent_of_the_loop_length():
    a, _ = capi.fma_rate(capi.RATE_FP32, 40000)
    b, _ = capi.fma_rate(capi.RATE_FP32, 80000)
    assert abs(a - b) <= 0.1 * max(a, b)


@pytest.mark.parametrize("kind,reps", [(3, 100), (-1, 100), (capi.RATE_FP32, 0)])
def test_bad_arguments_are_refused(kind, reps):
    with pytest.raises(capi.RTLBFSError):
        capi.fma_rate(kind, reps)
