"""Row-strip decomposition on CPU ranks (gloo, world size 2): the host side
of splitting one mesh by rows (paper_2202_13449_gb300.strips).

The strips here are a stand-in with the same interface as a library strip
(strip_get_rows / strip_set_halo) and the same reach as the RTLBFS step:
each new row depends on the rows up to two away (a five-row average per
field, walls mirrored at the mesh's own south and north sides).  A run
split into two strips that exchange halos before every step must equal the
run of the whole mesh exactly; the whole mesh's residual must come out of
the all-reduced strip sums; and a halo that a rank fails to send must stop
its neighbour with HaloLost instead of letting it step on stale rows.
"""
import math
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SOUTH, NORTH = 2, 3


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def smooth(ext):
    """Five-row average of ext (4, n + 4, nx): the n rows in the middle."""
    return (ext[:, :-4] + ext[:, 1:-3] + ext[:, 2:-2] + ext[:, 3:-1] + ext[:, 4:]) / 5.0


def whole_mesh_steps(f, nsteps):
    """The stand-in step on the whole mesh: rows beyond the south and north
    sides mirror the rows inside (walls)."""
    for _ in range(nsteps):
        ext = np.concatenate([f[:, 1::-1], f, f[:, :-3:-1]], axis=1)
        f = smooth(ext)
    return f


class FakeStrip:
    """Rows j0 <= j < j1 of the mesh f0 with the library strip's halo calls."""

    def __init__(self, f0, j0, j1):
        self.ny_mesh = f0.shape[1]
        self.j0, self.j1 = j0, j1
        self.f = f0[:, j0:j1].copy()
        self.halo = {SOUTH: None, NORTH: None}

    def strip_get_rows(self, side):
        return self.f[:, :2].copy() if side == SOUTH else self.f[:, -2:].copy()

    def strip_set_halo(self, side, rows):
        self.halo[side] = np.asarray(rows).reshape(4, 2, -1).copy()

    def step(self):
        lo = self.halo[SOUTH] if self.j0 > 0 else self.f[:, 1::-1]
        hi = self.halo[NORTH] if self.j1 < self.ny_mesh else self.f[:, :-3:-1]
        self.halo = {SOUTH: None, NORTH: None}  # a halo serves one step
        self.f = smooth(np.concatenate([lo, self.f, hi], axis=1))

    def residual_sums(self, f_old):
        d = self.f - f_old
        return np.array([np.sum(d[1] ** 2), np.sum(self.f[1] ** 2), np.sum(d[3] ** 2),
                         np.sum(self.f[3] ** 2)])


def mesh0(nx=7, ny=13):
    g = np.random.Generator(np.random.Philox(5))
    return g.uniform(-1.0, 1.0, size=(4, ny, nx))


def worker(rank, world, port, out, nsteps, drop):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import datetime

    import torch.distributed as dist

    from paper_2202_13449_gb300 import strips
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=60))
    try:
        f0 = mesh0()
        j0, j1 = strips.split_rows(f0.shape[1], world)[rank]
        s = FakeStrip(f0, j0, j1)
        ex = strips.StripExchange(rank, world, f0.shape[2], mode="host", timeout_s=3.0)
        ex.drop = drop if rank == 1 else None
        try:
            res = None
            for k in range(nsteps):
                ex.exchange(s, k)
                old = s.f.copy()
                s.step()
                res = strips.global_residual(s.residual_sums(old))
            out[rank] = ("ok", (j0, j1), s.f, res)
        except strips.HaloLost as e:
            out[rank] = ("lost", (j0, j1), str(e), None)
        except RuntimeError as e:  # the other rank has left the job
            out[rank] = ("error", (j0, j1), str(e), None)
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def run(nsteps, drop=None):
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(worker, args=(world, free_port(), out, nsteps, drop), nprocs=world,
                       join=True, start_method="spawn")
    return {r: out[r] for r in range(world)}


def test_split_rows_and_neighbours():
    sys.path.insert(0, ROOT)
    from paper_2202_13449_gb300 import strips
    assert strips.split_rows(13, 2) == [(0, 7), (7, 13)]
    parts = strips.split_rows(8192, 7)
    assert parts[0][0] == 0 and parts[-1][1] == 8192
    assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
    assert max(j1 - j0 for j0, j1 in parts) - min(j1 - j0 for j0, j1 in parts) <= 1
    with pytest.raises(ValueError):
        strips.split_rows(5, 3)  # a strip needs two rows for its halo
    assert strips.neighbours(0, 3) == (None, 1)
    assert strips.neighbours(1, 3) == (0, 2)
    assert strips.neighbours(2, 3) == (1, None)


def test_two_ranks_equal_the_whole_mesh():
    nsteps = 4
    res = run(nsteps)
    f0 = mesh0()
    want = whole_mesh_steps(f0, nsteps)
    got = np.zeros_like(want)
    for r in range(2):
        status, (j0, j1), f, _ = res[r]
        assert status == "ok"
        got[:, j0:j1] = f
    np.testing.assert_array_equal(got, want)
    # the whole mesh's residual of the last step from the all-reduced sums
    before = whole_mesh_steps(f0, nsteps - 1)
    d = want - before
    ru = math.sqrt(np.sum(d[1] ** 2)) / math.sqrt(np.sum(want[1] ** 2))
    rT = math.sqrt(np.sum(d[3] ** 2)) / math.sqrt(np.sum(want[3] ** 2))
    for r in range(2):
        assert res[r][3] == pytest.approx((ru, rT), rel=1e-12)


def test_lost_halo_stops_the_neighbour():
    """Rank 1 withholds its south rows of step 2: rank 0 must not take step
    2 on stale rows -- its exchange raises HaloLost naming the step."""
    res = run(4, drop=(2, SOUTH))
    status, _, msg, _ = res[0]
    assert status == "lost" and "step 2" in msg
