"""Host post-processing: the separation angle on a cylinder (Section 4.3)."""
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
