"""Host post-processing: the separation angle on a cylinder (Section 4.3),
and the square cavity's centreline maxima and streamfunction maximum
(Section 4.2, Tables 1-3), pinned on fields with known extrema."""
import math

import numpy as np
import pytest

from paper_2202_13449_gb300 import inputs, post


def _field(X, Y, phi_s_up, phi_s_lo):
    """First-row velocities whose tangential component crosses zero at
    phi_s_up on the upper half and -phi_s_lo on the lower half, reversed
    (counter-clockwise on top) behind the crossing."""
    xc = 0.25 * (X[:-1, :-1] + X[:-1, 1:] + X[1:, :-1] + X[1:, 1:])
    yc = 0.25 * (Y[:-1, :-1] + Y[:-1, 1:] + Y[1:, :-1] + Y[1:, 1:])
    phi = np.arctan2(yc, xc)
    a = np.where(phi >= 0, phi, -phi)
    s = np.where(phi >= 0, 1.0, -1.0)
    cut = np.where(phi >= 0, math.radians(phi_s_up), math.radians(phi_s_lo))
    ut = s * (cut - a)  # > 0 (reversed) behind the separation point
    return -ut * np.sin(phi), ut * np.cos(phi)


@pytest.mark.parametrize("up,lo", [(43.65, 43.65), (29.9, 35.2), (5.0, 60.0)])
def test_separation_angle_of_a_linear_profile(up, lo):
    X, Y = inputs.cylinder_o_mesh(360, 6)
    u, v = _field(X, Y, up, lo)
    got = post.separation_angle(X, Y, u, v)
    # linear in the angle between cell centres: exact up to rounding
    assert got[0] == pytest.approx(up, abs=1e-9)
    assert got[1] == pytest.approx(lo, abs=1e-9)


def test_attached_flow_has_no_separation():
    """A uniform stream along +x: u_phi <= 0 on the whole upper half."""
    X, Y = inputs.cylinder_o_mesh(90, 4)
    u = np.ones((4, 90))
    v = np.zeros((4, 90))
    assert post.separation_angle(X, Y, u, v) == (0.0, 0.0)


def test_parabola_peak_is_exact_on_quadratics():
    x = np.array([0.1, 0.25, 0.7])  # uneven spacing
    for a, x0, c in ((2.0, 0.3, 5.0), (0.5, 0.62, -1.0), (7.0, 0.12, 0.0)):
        xs, fs = post.parabola_peak(x, c - a * (x - x0) ** 2)
        assert xs == pytest.approx(x0, abs=1e-12) and fs == pytest.approx(c, abs=1e-12)
    # collinear points, and a vertex outside the bracket: the middle sample
    assert post.parabola_peak(x, 2.0 * x) == (0.25, 0.5)
    assert post.parabola_peak(x, -(x - 2.0) ** 2) == (0.25, -(0.25 - 2.0) ** 2)


def test_line_max_at_an_end_is_the_end_sample():
    pos = np.linspace(0.0, 1.0, 11)
    assert post.line_max(pos, pos) == (1.0, 1.0)
    assert post.line_max(pos, -pos) == (0.0, 0.0)


@pytest.mark.parametrize("n,phi", [(40, 0.0), (41, 0.0), (60, 2.0)])
def test_cavity_centrelines_of_quadratic_profiles(n, phi):
    """u depends on y only and v on x only, each a downward parabola with a
    known peak: the centreline maxima and their positions come out exact
    on uniform and stretched meshes, for even and odd cell counts."""
    L = 3.0
    if phi == 0.0:
        xf = inputs.uniform_faces(n, L)
    else:
        from paper_2202_13449_gb300 import capi
        xf = capi.tanh_faces(n, L, phi)
    yf = xf.copy()
    xc, yc = 0.5 * (xf[1:] + xf[:-1]), 0.5 * (yf[1:] + yf[:-1])
    u = np.repeat((2.0 - 4.0 * (yc - 0.7 * L) ** 2)[:, None], n, axis=1)
    v = np.repeat((1.0 - 3.0 * (xc - 0.2 * L) ** 2)[None, :], n, axis=0)
    umax, uy, vmax, vx = post.cavity_centrelines(xf, yf, u, v)
    assert umax == pytest.approx(2.0, abs=1e-12) and uy == pytest.approx(0.7, abs=1e-12)
    assert vmax == pytest.approx(1.0, abs=1e-12) and vx == pytest.approx(0.2, abs=1e-12)


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_streamfunction_max_of_a_single_cell_vortex(sign):
    """psi = A sin(pi x/L) sin(pi y/L) on [0, L]^2: u = d psi / dy sampled at
    cell centres, integrated up each column by the midpoint rule (second
    order): |psi|_max = A at the centre."""
    n, L, A = 200, 2.0, 3.5 * sign
    xf = inputs.uniform_faces(n, L)
    xc = 0.5 * (xf[1:] + xf[:-1])
    X, Y = np.meshgrid(xc, xc)
    u = A * np.pi / L * np.sin(np.pi * X / L) * np.cos(np.pi * Y / L)
    pmax, px, py = post.streamfunction_max(xf, xf, u)
    assert pmax == pytest.approx(abs(A), rel=1e-4)
    assert px == pytest.approx(0.5, abs=2e-3) and py == pytest.approx(0.5, abs=2e-3)
