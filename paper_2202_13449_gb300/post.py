"""Post-processing of downloaded states (host side, NumPy).

Quantities the paper reports from a converged field rather than computes on
the hot path: the separation angle on a circular cylinder (Section 4.3,
Table 4)."""
import math

import numpy as np


def separation_angle(X, Y, u, v):
    """Separation angles (degrees, measured from the rear stagnation point
    on the +x axis) of the upper and lower halves of a cylinder wall at
    vertex row j = 0 of the O-mesh (X, Y); (u, v) are nj x ni cell fields.

    The wall shear changes sign where the tangential velocity of the first
    cell row does: counter-clockwise velocity u_phi > 0 near phi = 0+ is the
    reversed flow of the recirculation.  The angle is where u_phi, followed
    from the rear towards the front, first turns negative (linear
    interpolation between cell centres); 0 when the flow never reverses."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    xc = 0.25 * (X[0, :-1] + X[0, 1:] + X[1, :-1] + X[1, 1:])
    yc = 0.25 * (Y[0, :-1] + Y[0, 1:] + Y[1, :-1] + Y[1, 1:])
    phi = np.arctan2(yc, xc)
    ut = -np.asarray(u)[0] * np.sin(phi) + np.asarray(v)[0] * np.cos(phi)
    out = []
    for sgn in (1.0, -1.0):  # upper half, then the lower half mirrored
        a, w = sgn * phi, sgn * ut
        m = a > 0.0
        order = np.argsort(a[m])
        aa, ww = a[m][order], w[m][order]
        if len(ww) < 2 or ww[0] <= 0.0:
            out.append(0.0)
            continue
        k = 0
        while k + 1 < len(ww) and ww[k + 1] > 0.0:
            k += 1
        if k + 1 == len(ww):
            out.append(180.0)
            continue
        a0, a1, w0, w1 = aa[k], aa[k + 1], ww[k], ww[k + 1]
        out.append(math.degrees(a0 + (a1 - a0) * w0 / (w0 - w1)))
    return out[0], out[1]
