"""The seeded input recipes (paper_2202_13449_gb300/inputs.py) against the
workloads they stand for: the trace and batch statistics of the serving and
batched configurations, and the O-mesh of the heated cylinder (Section 4.3:
far field 52.5 D from the centre, first spacing 0.003 D)."""
import numpy as np
import pytest

from paper_2202_13449_gb300 import inputs


@pytest.mark.parametrize("ni,nj", [(450, 300), (40, 12), (3600, 2400)])
def test_cylinder_o_mesh_geometry(ni, nj):
    X, Y = inputs.cylinder_o_mesh(ni, nj)
    assert X.shape == Y.shape == (nj + 1, ni + 1)
    r = np.hypot(X, Y)
    # rings of constant radius: the wall at D / 2, the far field at 52.5 D
    np.testing.assert_allclose(r[0], 0.5, rtol=0, atol=1e-14)
    np.testing.assert_allclose(r[-1], 52.5, rtol=0, atol=1e-12)
    np.testing.assert_allclose(r - r[:, :1], 0.0, rtol=0, atol=1e-12)
    dr = np.diff(r[:, 0])
    assert dr[0] == pytest.approx(0.003, rel=1e-9)
    # geometric growth: a constant ratio between consecutive spacings
    q = dr[1:-1] / dr[:-2]
    np.testing.assert_allclose(q, q[0], rtol=1e-9)
    # the seam closes (column ni repeats column 0) and the cells are
    # right-handed in (i, j): every shoelace area is positive
    np.testing.assert_array_equal(X[:, -1], X[:, 0])
    np.testing.assert_array_equal(Y[:, -1], Y[:, 0])
    x0, y0 = X[:-1, :-1], Y[:-1, :-1]
    x1, y1 = X[:-1, 1:], Y[:-1, 1:]
    x2, y2 = X[1:, 1:], Y[1:, 1:]
    x3, y3 = X[1:, :-1], Y[1:, :-1]
    area = 0.5 * ((x0 * y1 - x1 * y0) + (x1 * y2 - x2 * y1) + (x2 * y3 - x3 * y2)
                  + (x3 * y0 - x0 * y3))
    assert np.all(area > 0.0)
    # the cells tile the annulus between the regular ni-gons inscribed in
    # the circles of radius D / 2 and 52.5 D
    polygon = 0.5 * ni * np.sin(2.0 * np.pi / ni) * (52.5 ** 2 - 0.25)
    assert float(area.sum()) == pytest.approx(polygon, rel=1e-12)


def test_batch_specs_follow_the_recipe():
    specs = inputs.batch_specs()
    assert len(specs) == 1024
    sides = np.array([s.n for s in specs])
    assert set(sides.tolist()) <= set(inputs.BATCH_SIDES)
    phis = np.array([s.phi for s in specs])
    assert phis.min() >= 1.0 and phis.max() <= 2.5
    ras = np.array([s.Ra for s in specs])
    assert ras.min() >= 1e3 * (1 - 1e-12) and ras.max() <= 1e6 * (1 + 1e-12)
    # mean cells per cavity of the side set drawn uniformly: ~19.3 k
    assert 17000 < float(np.mean(sides.astype(float) ** 2)) < 21700
    # the same seed gives the same batch
    again = inputs.batch_specs()
    assert [(s.n, s.phi, s.Ra) for s in specs] == [(s.n, s.phi, s.Ra) for s in again]


def test_serving_trace_follows_the_recipe():
    tr = inputs.serving_trace()
    assert len(tr) == 10000
    t = np.array([r.t_arrive for r in tr])
    assert np.all(np.diff(t) >= 0.0)
    # Poisson arrivals at 200 per second: mean gap 5 ms, within 5 %
    assert np.mean(np.diff(t)) == pytest.approx(1.0 / 200.0, rel=0.05)
    n = np.array([r.n for r in tr])
    assert n.min() >= 64 and n.max() <= 1024
    ra = np.array([r.Ra for r in tr])
    assert ra.min() >= 1e3 * (1 - 1e-12) and ra.max() <= 1e8 * (1 + 1e-12)
    pr = {r.Pr for r in tr}
    assert pr <= {0.71, 7.0}
