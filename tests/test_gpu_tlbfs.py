"""The TLBFS face stage (Section 2.2) on the GPU against the oracle's TLBFS
stage, element by element through the C ABI, and its schedule rules."""
import numpy as np
import pytest

from paper_2202_13449_gb300 import capi, inputs
from test_gpu_parity import CASES, case_mesh, make_pair, rel, config2_pair

pytestmark = pytest.mark.gpu

TOL = {capi.FP64: 1e-12, capi.FP32: 1e-5}


def run_tlbfs(orc, name, precision, nsteps):
    nx, ny, mesh, kinds, bcT, bcU, kappa, bg = CASES[name]
    xf, yf = case_mesh(name, nx, ny, mesh)
    p, s = make_pair(orc, xf, yf, nu=0.04, chi=0.05, beta_g=bg, dt=0.25, kappa=kappa,
                     kinds=kinds, bcT=bcT, bcU=bcU, precision=precision)
    p.scheme = orc.TLBFS
    s.set_scheme(capi.TLBFS)
    st = inputs.perturbed_state(nx, ny, seed=3 + nx * 7 + ny)
    ref, _, rc = orc.step(p, st, nsteps)
    assert rc == 0
    s.set_state(*st)
    s.step(nsteps)
    got = s.get_state()
    nu = {w: s.nusselt(w) for w in (capi.NU_WEST, capi.NU_SOUTH)}
    s.close()
    return p, ref, got, nu


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("precision", [capi.FP64, capi.FP32])
def test_tlbfs_steps_match_oracle(orc, name, precision):
    p, ref, got, nu = run_tlbfs(orc, name, precision, 3)
    tol = 10 * TOL[precision] if precision == capi.FP64 else TOL[precision]
    if precision == capi.FP64:
        assert rel(got[0], ref[0], 1.0) < tol
    else:
        drho = np.max(np.abs(got[0] - ref[0])) / max(np.max(np.abs(ref[0] - 1.0)), 0.01)
        assert drho < tol, drho  # density deviation against max(|rho - 1|, Ma^2)
    for q, floor in ((1, 1e-2), (2, 1e-2), (3, 1.0)):
        assert rel(got[q], ref[q], floor) < tol, (q, rel(got[q], ref[q], floor))
    if precision == capi.FP64 and p.bc_kind[0] != orc.PERIODIC:
        want = orc.nusselt(p, ref, orc.NU_W)
        assert abs(nu[capi.NU_WEST] - want) <= 1e-10 * max(1.0, abs(want))


@pytest.mark.parametrize("precision", [capi.FP64, capi.FP32])
def test_tlbfs_full_size_512_tanh_cavity_one_step(orc, precision):
    p, s = config2_pair(orc, precision)
    p.scheme = orc.TLBFS
    s.set_scheme(capi.TLBFS)
    st = inputs.perturbed_state(512, 512, seed=2025, amp_u=0.05)
    ref, _, rc = orc.step(p, st, 1)
    s.set_state(*st)
    s.step(1)
    got = s.get_state()
    s.close()
    for q, floor in ((1, 0.1), (2, 0.1), (3, 1.0)):
        assert rel(got[q], ref[q], floor) < TOL[precision], (q, rel(got[q], ref[q], floor))


def test_tlbfs_schedule_rules():
    xf = inputs.uniform_faces(16)
    s = capi.Solver(xf, xf, capi.FP32)
    s.set_scheme(capi.TLBFS)
    for bad in ((0, 0), (1, 8)):
        with pytest.raises(capi.RTLBFSError):
            s.set_schedule(*bad)
    s.set_schedule(1, 0)
    k, r, _ = s.autotune(8)
    assert (k, r) == (1, 16)
    with pytest.raises(capi.RTLBFSError):
        s.set_scheme(5)
    s.set_scheme(capi.RTLBFS)
    s.set_schedule(0, 8)  # the marching kernel again
    s.close()
