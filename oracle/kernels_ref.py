"""Closed-form deformation kernels for piecewise-constant pressure (test infrastructure).

Sec. 3.3.1 approximates the pressure by a constant on each cell
``[x_k - h/2, x_k + h/2]`` (x ``[y_l - h/2, y_l + h/2]`` for point contact)
and integrates the elastic kernel over the cell analytically.

Line contact (Sec. 3.3.1 Case 1, Eqs. eqn101, eqn16-eqn19): with ``t = x - x'``
the cell integral of ``log|t|`` is ``[t (log|t| - 1)]`` between
``t_- = (d - 1/2) h`` and ``t_+ = (d + 1/2) h`` (signed ``t``; the printed
``|x_pm|`` form is only right for ``t > 0``).  The film thickness uses
``K[i, k] = G_{|i-k|} / pi`` with a minus sign:
``H_i = H0 + X_i^2/2 - sum_k K[i, k] P_k``.

Point contact (Sec. 3.3.1 Case 2): the cell integral of ``1/r`` is the
four-corner difference of ``F(x, y) = x asinh(y/|x|) + y asinh(x/|y|)``
(equal to the printed ``|x| asinh(y/x) + |y| asinh(x/y)``), and
``H_ij = H0 + X^2/2 + Y^2/2 + (2/pi^2) sum G P`` with the factor 2/pi^2
applied once.

Pins (tests/test_oracle_kernels.py): each coefficient against adaptive
numerical quadrature of the cell integral, and the discrete deformation of the
Hertzian pressure against its closed form.
"""
import numpy as np


def g_line(d, h):
    """Cell integral of ``log|x_i - x'|`` over cell k, ``d = i - k`` (any sign)."""
    d = np.abs(np.asarray(d, dtype=np.float64))
    tp = (d + 0.5) * h
    tm = (d - 0.5) * h

    def f(t):
        at = np.abs(t)
        return t * (np.log(at) - 1.0)

    return f(tp) - f(tm)


def k_line(N, h):
    """Dense line-contact deformation matrix ``K[i, k] = G_{|i-k|} / pi`` ([N, N])."""
    idx = np.arange(N)
    return g_line(idx[:, None] - idx[None, :], h) / np.pi


def _f_point(x, y):
    return x * np.arcsinh(y / np.abs(x)) + y * np.arcsinh(x / np.abs(y))


def g_point(dx, dy, h):
    """Cell integral of ``1/r`` over cell (k, l), offsets ``dx = i - k``, ``dy = j - l``."""
    dx = np.asarray(dx, dtype=np.float64)
    dy = np.asarray(dy, dtype=np.float64)
    xp, xm = (dx + 0.5) * h, (dx - 0.5) * h
    yp, ym = (dy + 0.5) * h, (dy - 0.5) * h
    return _f_point(xp, yp) - _f_point(xm, yp) - _f_point(xp, ym) + _f_point(xm, ym)


def g_point_table(nx, ny, h):
    """Table ``T[a, b] = (2/pi^2) G(a, b)`` for offsets ``0 <= a < nx``, ``0 <= b < ny``."""
    a = np.arange(nx)[:, None]
    b = np.arange(ny)[None, :]
    return (2.0 / np.pi**2) * g_point(a, b, h)


def deform_point(P, h, table=None):
    """Point-contact deformation ``D_ij = (2/pi^2) sum_{k,l} G(i-k, j-l) P_kl``.

    Direct summation over all source cells, organised as one sum per
    x-offset ``a = |i - k|``: for each ``a`` the rows of ``P`` at that offset
    are multiplied by the Toeplitz matrix ``T_a[j, l] = (2/pi^2) G(a, j-l)``.
    ``P`` is ``[nx, ny]`` (x index first).
    """
    P = np.asarray(P, dtype=np.float64)
    nx, ny = P.shape
    if table is None:
        table = g_point_table(nx, ny, h)
    jj = np.arange(ny)
    D = np.zeros_like(P)
    for a in range(nx):
        Ta = table[a][np.abs(jj[:, None] - jj[None, :])]  # [ny, ny], symmetric
        # sources k = i - a and k = i + a contribute T_a @ P[k]
        Q = P @ Ta  # Q[k, j] = sum_l P[k, l] T_a[l, j]
        if a == 0:
            D += Q
        else:
            D[a:] += Q[:-a]
            D[:-a] += Q[a:]
    return D


def hertz_deform_line(x):
    """Closed form of ``(1/pi) int_{-1}^{1} sqrt(1-s^2) log|x-s| ds``."""
    x = np.abs(np.asarray(x, dtype=np.float64))
    inside = 0.5 * (x**2 - 0.5 - np.log(2.0))
    xo = np.maximum(x, 1.0)
    q = np.sqrt(xo**2 - 1.0)
    outside = 0.5 * (xo**2 - xo * q - 0.5 + np.log(xo + q) - np.log(2.0))
    return np.where(x <= 1.0, inside, outside)


def hertz_deform_point(r):
    """Closed form of ``(2/pi^2) int int_{disk} sqrt(1-rho^2) / |r - r'| dA'``."""
    r = np.asarray(r, dtype=np.float64)
    inside = 1.0 - 0.5 * r**2
    ro = np.maximum(r, 1.0)
    outside = ((2.0 - ro**2) * np.arcsin(1.0 / ro) + np.sqrt(ro**2 - 1.0)) / np.pi
    return np.where(r <= 1.0, inside, outside)
