"""Small helpers shared by the test modules (no solver arithmetic here)."""
import numpy as np

CS2 = 1.0 / 3.0
# D2Q9 lattice of Eqs. 5-6, written out for the distribution-function pins.
E_D2Q9 = np.array([[0, 1, 0, -1, 0, 1, -1, -1, 1],
                   [0, 0, 1, 0, -1, 1, 1, -1, -1]], dtype=np.float64)
W_D2Q9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, dtype=np.float64)


def f_eq(rho, u, v):
    """Eq. 3 for all nine directions."""
    eu = E_D2Q9[0] * u + E_D2Q9[1] * v
    return W_D2Q9 * rho * (1.0 + eu / CS2 + eu ** 2 / (2 * CS2 ** 2) - (u * u + v * v) / (2 * CS2))


def g_eq(rho, u, v, T):
    """Eq. 4 with c_p = 1 for all nine directions."""
    eu = E_D2Q9[0] * u + E_D2Q9[1] * v
    return W_D2Q9 * rho * T * (1.0 + eu / CS2)


def centres(f):
    f = np.asarray(f)
    return 0.5 * (f[1:] + f[:-1])


def rel_err(a, b, scale):
    """max|a-b| / max(max|b|, scale) -- the parity norm of the tests."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), scale))


# D3Q19 of Eqs. 5-6, in the printed column order, with the printed column 14
# (a repeat of column 12, (-1, 0, 1)) read as (-1, 0, -1): the only
# completion that gives 19 distinct velocities.
E_D3Q19 = np.array([[0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0],
                    [0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1],
                    [0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1]],
                   dtype=np.float64)
W_D3Q19 = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12, dtype=np.float64)


def f_eq3(rho, u, v, w):
    """Eq. 3 for the nineteen D3Q19 directions."""
    eu = E_D3Q19[0] * u + E_D3Q19[1] * v + E_D3Q19[2] * w
    usq = u * u + v * v + w * w
    return W_D3Q19 * rho * (1.0 + eu / CS2 + eu ** 2 / (2 * CS2 ** 2) - usq / (2 * CS2))


def g_eq3(rho, u, v, w, T):
    """Eq. 4 with c_p = 1 for the nineteen D3Q19 directions."""
    eu = E_D3Q19[0] * u + E_D3Q19[1] * v + E_D3Q19[2] * w
    return W_D3Q19 * rho * T * (1.0 + eu / CS2)
