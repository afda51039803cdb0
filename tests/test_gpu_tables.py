"""Table 1 of the paper (Section 4.2) on the GPU at the paper's own meshes.

The square cavity at Ra = 1e3 (100^2) and 1e4 (150^2), uniform, Pr = 0.71,
V_c = 0.1, FP32, run from the conduction state to max(R_u, R_T) < 1e-7 on
the device; the centreline velocity maxima, their positions and Eq. 69's
Nu_a against the paper's RTLBFS row (tests/golden/tables123_cavity.json).
The higher Rayleigh numbers and Tables 2-3 run as the cavity_tables bench
workload (minutes of device time).
"""
import json
import os

import numpy as np
import pytest

from paper_2202_13449_gb300 import capi, inputs, post

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = {c["Ra"]: c for c in json.load(open(os.path.join(HERE, "golden", "tables123_cavity.json")))["cases"]}


@pytest.mark.parametrize("Ra", [1e3, 1e4])
def test_table1_on_the_paper_mesh(Ra):
    g = GOLD[Ra]
    n, L = g["n"], float(g["n"])
    xf = inputs.uniform_faces(n, L)
    s = capi.Solver(xf, xf, capi.FP32)
    s.set_params(Ra, 0.71, 0.1, 0.0)
    rc, steps, res = s.run_to_steady(1e-7, 400_000)
    assert rc == capi.OK, (rc, steps, res)
    chi = 0.1 * L * np.sqrt(0.71 / Ra) / 0.71  # nu / Pr (Eq. 63, V_c = Ma)
    rho, u, v, T = s.get_state()
    umax, uy, vmax, vx = post.cavity_centrelines(xf, xf, u, v)
    assert umax * L / chi == pytest.approx(g["u_max"], rel=5e-3)
    assert vmax * L / chi == pytest.approx(g["v_max"], rel=5e-3)
    assert abs(uy - g["u_max_y"]) < 5e-3 and abs(vx - g["v_max_x"]) < 5e-3
    assert s.nusselt(capi.NU_AVG) == pytest.approx(g["Nu_a"], rel=5e-3)
    s.close()
