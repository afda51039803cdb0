"""Host helpers of bench.py that set up the paper's workloads, on the CPU.

stretch_to_first_cell fits Eq. 74's tanh faces to the first-cell distances
the paper gives for its Ra = 1e7 and 1e8 cavity meshes (Section 4.2): the
fitted mesh must have that first cell, be symmetric about the centre and
grow monotonically towards it.  The clock sampler's parsing of the
nvidia-smi query lines and the roofline arithmetic (operations or
algorithmic bytes per launch over the launch time, against the peak) are
checked on made-up inputs.
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


class _DoneProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_sampler_parses_the_query_lines(tmp_path):
    """Median SM clock under load, the maximum clock and the throttle
    reasons that were active in any sample; malformed lines are skipped."""
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    rows = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "garbage line",
        "0, [N/A], 2070, 10.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1200.5, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    with open(s.path, "w") as f:
        f.write("\n".join(rows) + "\n")
    s.f = open(s.path, "a")
    s.proc = _DoneProc()
    c = s.stop()
    assert c == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                 "samples": 3}


def test_clock_sampler_without_samples(tmp_path):
    s = bench.ClockSampler(0)
    assert s.stop() is None  # never started
    s.path = str(tmp_path / "empty.csv")
    open(s.path, "w").close()
    s.f = open(s.path, "a")
    s.proc = _DoneProc()
    assert s.stop() is None


def test_rooflines_arithmetic(monkeypatch):
    """achieved = operations (or algorithmic bytes) per launch / launch time,
    frac = achieved / peak, with the library's operation count and 8 words of
    state per cell-update (4 read, 4 written)."""
    import types
    import torch
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    monkeypatch.setattr(torch.cuda, "get_device_properties",
                        lambda i: types.SimpleNamespace(multi_processor_count=152))
    monkeypatch.setitem(bench._ALU_PEAKS, 4, (38.0, "test peak"))
    cells, t = 262144, 11.25e-6
    alu, hbm = bench.rooflines("k", cells, t, 4, 4319488.0, {"sm_max_mhz": 2070.0})
    _, ops, _ = capi.op_counts(0)
    assert alu["alg_ops_per_launch"] == ops * cells
    assert alu["achieved"] == pytest.approx(ops * cells / t / 1e12, abs=1e-3)
    assert alu["frac"] == pytest.approx(ops * cells / t / 1e12 / 38.0, abs=1e-4)
    assert alu["peak_derived"]["value"] == pytest.approx(152 * 128 * 2070e6 / 1e12, abs=1e-3)
    assert hbm["alg_bytes_per_launch"] == 32 * cells
    peak, _ = bench.peaks()
    assert hbm["achieved"] == pytest.approx(32 * cells / t / 1e9, abs=0.1)
    assert hbm["frac"] == pytest.approx(32 * cells / t / 1e9 / peak, abs=1e-4)
    assert alu["traffic"] == hbm["traffic"] == 4319488.0
    # FP64: 64 B per cell-update, no derived FP32 lane peak
    monkeypatch.setitem(bench._ALU_PEAKS, 8, (0.5, "test peak"))
    alu8, hbm8 = bench.rooflines("k", cells, t, 8, None, None)
    assert hbm8["alg_bytes_per_launch"] == 64 * cells and "peak_derived" not in alu8
