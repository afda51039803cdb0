"""Row strips of one mesh on the GPU (rtlbfs_create_strip) against the FP64
oracle of the whole mesh, through the C ABI.

Strips exchange their two boundary rows before every step (host planes
through rtlbfs_strip_get_rows / rtlbfs_strip_set_halo, or device records
through rtlbfs_strip_pack / rtlbfs_strip_unpack); assembled, they must give
the whole mesh's step: FP64 <= 1e-12 per step, FP32 <= 1e-5 (the parity
norms of test_gpu_parity).  The whole mesh's residual is the R12 of the
summed residual sums; its wall and Eq. 69 Nusselt numbers are the sums of
the strips' shares.
"""
import math

import numpy as np
import pytest

from paper_2202_13449_gb300 import capi, inputs, strips

pytestmark = pytest.mark.gpu

D, A, P = capi.WALL_DIRICHLET, capi.WALL_ADIABATIC, capi.PERIODIC
S, N, W, E = capi.SOUTH, capi.NORTH, capi.WEST, capi.EAST


def rel(a, b, floor):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(float(np.max(np.abs(b))), floor))


def make(orc, nx, ny, kinds, bcT, bcU, precision, parts, seed, kappa=0.8, bg=1e-3):
    xf, yf = inputs.random_faces(nx, seed), inputs.random_faces(ny, seed + 1)
    nu, chi, dt = 0.04, 0.05, 0.25
    p = orc.Problem(xf=xf, yf=yf, nu=nu, chi=chi, beta_g=bg, dt=dt, kappa=kappa,
                    bc_kind=kinds, bc_T=bcT, bc_u=bcU)
    out = []
    for j0, j1 in strips.split_rows(ny, parts):
        s = capi.Solver(xf, yf, precision, rows=(j0, j1))
        s.set_params_ref(1e3, 0.71, 0.1, dt, 1.0, 1.0, 0.5)
        s.set_physics(nu, chi, bg)
        s.set_lattice(kappa)
        for side in (W, E):
            s.set_bc(side, kinds[side], bcT[side], bcU[side])
        if j0 == 0:
            s.set_bc(S, kinds[S], bcT[S], bcU[S])
        if j1 == ny:
            s.set_bc(N, kinds[N], bcT[N], bcU[N])
        out.append(s)
    return p, out


def upload(ss, st):
    for s in ss:
        j0, j1 = s.rows
        s.set_state(*[a[j0:j1] for a in st])


def exchange_host(ss):
    for lo, hi in zip(ss, ss[1:]):
        up, down = lo.strip_get_rows(N), hi.strip_get_rows(S)
        hi.strip_set_halo(S, up)
        lo.strip_set_halo(N, down)


def assemble(ss):
    parts = [s.get_state() for s in ss]
    return tuple(np.concatenate([p[q] for p in parts], axis=0) for q in range(4))


def check_fields(got, ref, precision):
    tol = 1e-12 if precision == capi.FP64 else 1e-5
    if precision == capi.FP64:
        assert rel(got[0], ref[0], 1.0) < tol
    else:
        d = np.max(np.abs(got[0] - ref[0])) / max(np.max(np.abs(ref[0] - 1.0)), 0.01)
        assert d < tol, d
    for q, floor in ((1, 1e-2), (2, 1e-2), (3, 1.0)):
        assert rel(got[q], ref[q], floor) < tol, (q, rel(got[q], ref[q], floor))


CASES = {
    # name: (nx, ny, kinds, bcT, bcU, parts)
    "cavity_two_strips": (37, 26, (D, D, A, A), (1, 0, 0, 0), (0, 0, 0, 0.01), 2),
    "cavity_three_strips": (45, 40, (D, A, D, A), (0.9, 0, 0.2, 0), (0, 0.01, 0, 0), 3),
    "periodic_x_two_strips": (33, 21, (P, P, D, D), (0, 0, 1, 0), (0, 0, 0, 0), 2),
}


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("precision", [capi.FP64, capi.FP32])
@pytest.mark.parametrize("name", sorted(CASES))
def test_strips_match_the_whole_mesh(orc, name, precision, kernel):
    nx, ny, kinds, bcT, bcU, parts = CASES[name]
    p, ss = make(orc, nx, ny, kinds, bcT, bcU, precision, parts, seed=sum(map(ord, name)))
    for s in ss:
        s.set_schedule(kernel, 0)
    st = inputs.perturbed_state(nx, ny, seed=17 + nx)
    upload(ss, st)
    ref, done = st, 0
    for n in (1, 3, 5):
        for _ in range(n - done):
            exchange_host(ss)
            for s in ss:
                s.step(1)
        ref, (ru, rT), rc = orc.step(p, ref, n - done)
        assert rc == 0
        done = n
        check_fields(assemble(ss), ref, precision)
        # the whole mesh's residual of the last step from the strips' sums
        tot = sum(s.residual_sums()[0] for s in ss)
        gu = math.sqrt(tot[0]) / math.sqrt(tot[1])
        gT = math.sqrt(tot[2]) / math.sqrt(tot[3])
        rtol = 1e-12 if precision == capi.FP64 else 1e-4
        assert gu == pytest.approx(ru, rel=rtol) and gT == pytest.approx(rT, rel=rtol)
    if precision == capi.FP64:
        exchange_host(ss)  # the gradients next to a halo side read the halo rows
        whiches = [(capi.NU_AVG, orc.NU_A)]
        if kinds[W] != P:
            whiches += [(capi.NU_WEST, orc.NU_W), (capi.NU_EAST, orc.NU_E)]
        for mine, theirs in whiches:
            want = orc.nusselt(p, ref, theirs)
            got = sum(s.nusselt(mine) for s in ss)
            assert abs(got - want) <= 1e-11 * max(1.0, abs(want)), (mine, got, want)
    for s in ss:
        s.close()


@pytest.mark.parametrize("precision", [capi.FP64, capi.FP32])
def test_device_exchange_equals_host_exchange(orc, precision):
    """Halos through device byte buffers (pack / unpack of the records,
    buffer = steps % 2) give the fields of halos through host planes: the
    same bits in FP32 (the fixed-point records convert to doubles and back
    exactly); in FP64 within one rounding, since a host plane carries rho =
    1 + (rho - 1) and the record rho - 1."""
    import torch
    torch.cuda.init()
    nx, ny, kinds, bcT, bcU, parts = CASES["cavity_three_strips"]
    seed = sum(map(ord, "device"))
    _, a = make(orc, nx, ny, kinds, bcT, bcU, precision, parts, seed)
    _, b = make(orc, nx, ny, kinds, bcT, bcU, precision, parts, seed)
    st = inputs.perturbed_state(nx, ny, seed=71)
    upload(a, st)
    upload(b, st)
    nbytes = a[0].strip_rows(N, False, 0)[1]
    bufs = [torch.empty(nbytes, dtype=torch.uint8, device="cuda") for _ in range(2)]
    for k in range(4):
        exchange_host(a)
        for s in a:
            s.step(1)
        for lo, hi in zip(b, b[1:]):
            assert lo.current_buffer() == k % 2 == hi.current_buffer()
            lo.strip_pack(N, k % 2, bufs[0].data_ptr())
            hi.strip_pack(S, k % 2, bufs[1].data_ptr())
            lo.sync()
            hi.sync()
            hi.strip_unpack(S, k % 2, bufs[0].data_ptr())
            lo.strip_unpack(N, k % 2, bufs[1].data_ptr())
            lo.sync()
            hi.sync()
        for s in b:
            s.step(1)
    ga, gb = assemble(a), assemble(b)
    for q in range(4):
        if precision == capi.FP32:
            np.testing.assert_array_equal(ga[q], gb[q])
        else:
            np.testing.assert_allclose(ga[q], gb[q], rtol=0, atol=4e-16 * max(1.0, np.max(np.abs(gb[q]))))
    for s in a + b:
        s.close()


def test_strip_arguments_are_checked(orc):
    xf, yf = inputs.uniform_faces(8), inputs.uniform_faces(10)
    with pytest.raises(RuntimeError):
        capi.Solver(xf, yf, capi.FP64, rows=(4, 5))  # one row: no room for a halo
    with pytest.raises(RuntimeError):
        capi.Solver(xf, yf, capi.FP64, rows=(6, 11))  # beyond the mesh
    s = capi.Solver(xf, yf, capi.FP64, rows=(0, 5))
    with pytest.raises(RuntimeError):
        s.set_bc(N, D, 0.0, 0.0)  # the north side is the strip's halo side
    with pytest.raises(RuntimeError):
        s.nusselt(capi.NU_NORTH)  # no wall there
    with pytest.raises(RuntimeError):
        s.strip_get_rows(S)  # the south side is the mesh's wall, not a halo
    s.close()
