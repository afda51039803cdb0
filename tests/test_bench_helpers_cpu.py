"""Host helpers of bench.py that set up the paper's workloads, on the CPU.

stretch_to_first_cell fits Eq. 74's tanh faces to the first-cell distances
the paper gives for its Ra = 1e7 and 1e8 cavity meshes (Section 4.2): the
fitted mesh must have that first cell, be symmetric about the centre and
grow monotonically towards it.
"""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2202_13449_gb300 import capi  # noqa: E402


@pytest.mark.parametrize("n,wall", [(300, 0.0004), (400, 0.0002), (64, 0.005)])
def test_stretch_to_first_cell(n, wall):
    L = float(n)
    phi = bench.stretch_to_first_cell(n, L, wall * L)
    xf = capi.tanh_faces(n, L, phi)
    w = np.diff(xf)
    assert w[0] == pytest.approx(wall * L, rel=1e-9)
    np.testing.assert_allclose(w, w[::-1], rtol=1e-9)  # symmetric
    half = w[: n // 2]
    assert np.all(np.diff(half) > 0)  # growing towards the centre
    assert xf[0] == pytest.approx(0.0, abs=1e-12) and xf[-1] == pytest.approx(L, rel=1e-12)


def test_tables_golden_cases_cover_the_paper_meshes():
    import json
    with open(os.path.join(ROOT, "tests", "golden", "tables123_cavity.json")) as f:
        gold = json.load(f)
    cases = {c["Ra"]: (c["n"], c["wall"]) for c in gold["cases"]}
    assert cases == {1e3: (100, 0.0), 1e4: (150, 0.0), 1e5: (200, 0.0), 1e6: (250, 0.0),
                     1e7: (300, 0.0004), 1e8: (400, 0.0002)}
