"""Post-processing of downloaded states (host side, NumPy).

Quantities the paper reports from a converged field rather than computes on
the hot path: the separation angle on a circular cylinder (Section 4.3,
Table 4), and the square cavity's centreline velocity maxima and
streamfunction maximum (Section 4.2, Tables 1-3)."""
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


def parabola_peak(x, f):
    """Vertex (x*, f*) of the quadratic through three points (x[k], f[k]),
    k = 0, 1, 2, with ascending, possibly unevenly spaced x; the middle
    point itself when the three are collinear or the vertex falls outside
    [x[0], x[2]]."""
    x0, x1, x2 = (float(t) for t in x)
    f0, f1, f2 = (float(t) for t in f)
    d01 = (f1 - f0) / (x1 - x0)
    d12 = (f2 - f1) / (x2 - x1)
    c = (d12 - d01) / (x2 - x0)  # leading coefficient
    if c == 0.0:
        return x1, f1
    b = d01 - c * (x0 + x1)  # f = c x^2 + b x + const
    xs = -b / (2.0 * c)
    if not (x0 <= xs <= x2):
        return x1, f1
    # Newton form of the same quadratic
    return xs, f0 + d01 * (xs - x0) + c * (xs - x0) * (xs - x1)


def line_max(pos, vals):
    """Maximum of a sampled line and its position: the largest sample,
    refined by parabola_peak through it and its two neighbours (the sample
    itself at an end of the line)."""
    pos = np.asarray(pos, dtype=np.float64)
    vals = np.asarray(vals, dtype=np.float64)
    k = int(np.argmax(vals))
    if k == 0 or k == len(vals) - 1:
        return float(pos[k]), float(vals[k])
    return parabola_peak(pos[k - 1:k + 2], vals[k - 1:k + 2])


def cavity_centrelines(xf, yf, u, v):
    """The square-cavity quantities of Section 4.2 from cell fields u, v
    (ny x nx, face coordinates xf, yf): the largest u along the vertical
    centreline x = L/2 and its height, and the largest v along the
    horizontal centreline y = L/2 and its abscissa, both lines taken
    between the two middle cell columns (rows) for an even cell count, or
    through the middle cells for an odd one.  Positions as fractions of
    the box sides, measured from the south-west corner."""
    xf = np.asarray(xf, dtype=np.float64)
    yf = np.asarray(yf, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    ny, nx = u.shape
    xc, yc = 0.5 * (xf[1:] + xf[:-1]), 0.5 * (yf[1:] + yf[:-1])
    Lx, Ly = xf[-1] - xf[0], yf[-1] - yf[0]

    def mid(a, n, axis):
        if n % 2:
            return np.take(a, n // 2, axis=axis)
        return 0.5 * (np.take(a, n // 2 - 1, axis=axis) + np.take(a, n // 2, axis=axis))

    yu, umax = line_max(yc, mid(u, nx, 1))
    xv, vmax = line_max(xc, mid(v, ny, 0))
    return umax, (yu - yf[0]) / Ly, vmax, (xv - xf[0]) / Lx


def streamfunction_max(xf, yf, u):
    """Largest |psi| of the streamfunction (u = d psi / dy, psi = 0 on the
    south wall) and its position as fractions of the box sides: psi at the
    cell columns' centres x_i and the horizontal faces y_j is the
    midpoint-rule integral of u up the column; the grid maximum is refined
    by parabola_peak along the column and across the columns."""
    xf = np.asarray(xf, dtype=np.float64)
    yf = np.asarray(yf, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    dy = np.diff(yf)
    psi = np.zeros((u.shape[0] + 1, u.shape[1]))
    psi[1:] = np.cumsum(u * dy[:, None], axis=0)
    a = np.abs(psi)
    j, i = np.unravel_index(int(np.argmax(a)), a.shape)
    xc = 0.5 * (xf[1:] + xf[:-1])
    ys, vy = (yf[j], a[j, i]) if j in (0, a.shape[0] - 1) else parabola_peak(yf[j - 1:j + 2], a[j - 1:j + 2, i])
    xs, vx = (xc[i], a[j, i]) if i in (0, a.shape[1] - 1) else parabola_peak(xc[i - 1:i + 2], a[j, i - 1:i + 2])
    Lx, Ly = xf[-1] - xf[0], yf[-1] - yf[0]
    return max(vy, vx), (xs - xf[0]) / Lx, (ys - yf[0]) / Ly
