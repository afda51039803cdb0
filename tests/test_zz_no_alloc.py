"""The allocation-free Nusselt entry point against the handle API.

rtlbfs_nusselt_noalloc serves callers that cannot allocate device memory
when they call in (a real-time loop, where cudaMalloc may block or fail at an
unpredictable moment; a host that lends the library only a fixed memory
pool): it takes caller-owned FP64 device fields and keeps its working memory
in a file-scope device array.  Here torch owns the fields; two consecutive calls
(which reuse that array) must each agree with rtlbfs_nusselt of a handle
holding the same state, to the FP64 tolerance of the other GPU tests.
"""
import numpy as np
import pytest

from paper_2202_13449_gb300 import capi, inputs

pytestmark = pytest.mark.gpu


def test_noalloc_nusselt_matches_handle_twice():
    import torch
    torch.cuda.init()
    D, A, P = capi.WALL_DIRICHLET, capi.WALL_ADIABATIC, capi.PERIODIC
    cases = [
        # (nx, ny, kinds, bc_T, bc_u, which list, seed)
        (38, 22, (D, D, A, A), (1.0, 0.0, 0.0, 0.0), (0.0, 0.0, 0.0, 0.0),
         [capi.NU_WEST, capi.NU_EAST, capi.NU_AVG, capi.NU_HALF], 5),
        (29, 41, (A, D, D, D), (0.0, 0.2, 0.9, 0.3), (0.01, 0.0, 0.0, 0.02),
         [capi.NU_SOUTH, capi.NU_NORTH, capi.NU_EAST, capi.NU_AVG], 6),
        # periodic in x: the wrapped widths of the mesh-line builder
        (33, 18, (P, P, D, D), (0.0, 0.0, 1.0, 0.0), (0.0, 0.0, 0.0, 0.03),
         [capi.NU_SOUTH, capi.NU_NORTH, capi.NU_AVG], 7),
        # periodic in y
        (24, 27, (D, A, P, P), (0.8, 0.0, 0.0, 0.0), (0.0, 0.02, 0.0, 0.0),
         [capi.NU_WEST, capi.NU_EAST, capi.NU_AVG, capi.NU_HALF], 8),
    ]
    stream = torch.cuda.current_stream()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for nx, ny, kinds, bT, bU, whiches, seed in cases:  # two calls in a row per selector
        xf, yf = inputs.random_faces(nx, seed), inputs.random_faces(ny, seed + 1)
        nu, chi, kappa = 0.03, 0.05, 0.9
        st = inputs.perturbed_state(nx, ny, seed=seed + 2)
        s = capi.Solver(xf, yf, capi.FP64)
        s.set_params(1e4, 0.71, 0.1, 0.3)
        s.set_physics(nu, chi, 1e-3)
        s.set_lattice(kappa)
        for side in range(4):
            s.set_bc(side, kinds[side], bT[side], bU[side])
        s.set_state(*st)
        dev = [torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
               for a in st]
        for which in whiches:
            want = s.nusselt(which)
            got = []
            for _ in range(2):
                out.fill_(np.nan)
                rc = capi.nusselt_noalloc(xf, yf, *[t.data_ptr() for t in dev], nu, chi, kappa,
                                          1.0, kinds, bT, bU, which, out.data_ptr(), stream)
                assert rc == capi.OK
                torch.cuda.synchronize()
                got.append(float(out.item()))
            for g in got:
                assert abs(g - want) <= 1e-12 * max(abs(want), 1.0), (which, g, want)
        s.close()


def test_noalloc_rejects_sizes_beyond_its_array():
    import torch
    torch.cuda.init()
    n = 8193
    xf = np.arange(n + 1, dtype=np.float64)
    yf = np.arange(4, dtype=np.float64)
    buf = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    rc = capi.nusselt_noalloc(xf, yf, p, p, p, p, 0.1, 0.1, 1.0, 1.0, (0, 0, 1, 1),
                              (1, 0, 0, 0), (0, 0, 0, 0), capi.NU_WEST, out.data_ptr())
    assert rc == capi.ERR_ARG
