"""The stability test of Section 3.3 (Figs. 4-5) as one batched launch,
through the C ABI (rtlbfs_stability_map), against the FP64 oracle run case
by case: the same outcome (converged / diverged / step cap) for every case,
and a diverging case stops within a few steps of the oracle's (FP64) or
no later (FP32, whose fixed-point range is left before values overflow)."""
import numpy as np
import pytest

from paper_2202_13449_gb300 import capi

pytestmark = pytest.mark.gpu

CASES = [(n, Ra, kappa) for n in (20, 33) for Ra in (1e6, 1e8) for kappa in (0.1, 0.5, 1.0)]


def oracle_outcomes(orc, cases, tol, cap):
    out = []
    for n, Ra, kappa in cases:
        p = orc.cavity_problem(n, Ra, dt=0.5)
        p.kappa = kappa
        from paper_2202_13449_gb300 import inputs
        _, steps, _, rc = orc.run_to_steady(p, inputs.conduction_state(p.xf, p.yf), tol, cap)
        status = {0: capi.SLOT_CONVERGED, -4: capi.SLOT_DIVERGED, -5: capi.SLOT_MAX_STEPS}[rc]
        out.append((status, steps))
    return out


@pytest.mark.parametrize("precision", [capi.FP64, capi.FP32])
def test_stability_map_matches_oracle(orc, precision):
    tol, cap = 1e-9, 3000
    n, Ra, kappa = (np.array(c) for c in zip(*CASES))
    status, steps, _ = capi.stability_map(n, Ra, kappa, np.full(len(CASES), 0.5), tol=tol,
                                          max_steps=cap, precision=precision, chunk_steps=128)
    ref = oracle_outcomes(orc, CASES, tol, cap)
    for k, (case, (st_ref, steps_ref)) in enumerate(zip(CASES, ref)):
        assert status[k] == st_ref, (case, status[k], st_ref)
        if st_ref == capi.SLOT_DIVERGED and precision == capi.FP64:
            assert abs(steps[k] - steps_ref) <= max(3, 0.03 * steps_ref), (case, steps[k], steps_ref)
        elif st_ref == capi.SLOT_DIVERGED:
            # the FP32 state stops when a value leaves the fixed-point range
            # (|u| >= 0.99 ...), before the FP64 values turn into NaN
            assert steps[k] <= steps_ref + 3, (case, steps[k], steps_ref)
        else:
            assert steps[k] == steps_ref
    # the trend of Fig. 4: at each (n, Ra) the smallest lattice spacing diverges
    assert all(status[k] == capi.SLOT_DIVERGED for k, c in enumerate(CASES) if c[2] == 0.1)


def test_stability_map_cases_are_independent():
    """A case gives the same outcome and step count alone and in the map."""
    n, Ra, kappa = (np.array(c) for c in zip(*CASES))
    dt = np.full(len(CASES), 0.5)
    status, steps, _ = capi.stability_map(n, Ra, kappa, dt, max_steps=1500, precision=capi.FP64)
    for k in (0, 4, len(CASES) - 1):
        s1, n1, _ = capi.stability_map(n[k:k + 1], Ra[k:k + 1], kappa[k:k + 1], dt[k:k + 1],
                                       max_steps=1500, precision=capi.FP64)
        assert s1[0] == status[k] and n1[0] == steps[k]


def test_stability_map_arguments():
    with pytest.raises(capi.RTLBFSError):
        capi.stability_map([10], [1e3], [0.0])
    s, n, el = capi.stability_map([], [], [])
    assert len(s) == 0 and el == 0.0
