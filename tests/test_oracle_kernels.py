"""Pins of the deformation-kernel oracle.

* every cell coefficient against adaptive numerical quadrature of its
  defining integral (scipy.integrate, independent of the closed forms);
* the self-cell coefficient of the point kernel against the textbook value
  ``int int_{square of side h} 1/r = 4 h ln(1 + sqrt 2)``;
* the discrete deformation of the Hertzian pressure against the closed-form
  potential of the half-ellipse (line) and hemisphere (point) pressure:
  the film thickness inside the contact must come out flat, the error must
  shrink under refinement.
"""
import numpy as np
import pytest
from scipy import integrate

from oracle import kernels_ref as kr


@pytest.mark.parametrize("h", [0.05, 0.3, 1.7])
@pytest.mark.parametrize("d", [0, 1, 2, 5, 40])
def test_line_kernel_vs_quadrature(d, h):
    # int_{x_k - h/2}^{x_k + h/2} log|x_i - x'| dx' with x_i - x_k = d h
    f = lambda xp: np.log(abs(d * h - xp))
    pts = [0.0] if d == 0 else None
    val, err = integrate.quad(f, -h / 2, h / 2, points=pts, epsabs=1e-14, epsrel=1e-13, limit=200)
    assert abs(kr.g_line(d, h) - val) <= 1e-12 * max(1.0, abs(val))
    assert kr.g_line(-d, h) == kr.g_line(d, h)


@pytest.mark.parametrize("dx,dy", [(1, 0), (0, 3), (2, 1), (5, 7), (30, 2)])
def test_point_kernel_vs_quadrature(dx, dy):
    h = 0.1
    f = lambda y, x: 1.0 / np.hypot(dx * h - x, dy * h - y)
    val, err = integrate.dblquad(f, -h / 2, h / 2, -h / 2, h / 2, epsabs=1e-13, epsrel=1e-12)
    assert abs(kr.g_point(dx, dy, h) - val) <= 1e-10 * abs(val)
    assert kr.g_point(-dx, dy, h) == pytest.approx(kr.g_point(dx, dy, h), rel=1e-15)
    assert kr.g_point(dy, dx, h) == pytest.approx(kr.g_point(dx, dy, h), rel=1e-14)


def test_point_self_cell_textbook():
    for h in (0.01, 0.5, 2.0):
        assert kr.g_point(0, 0, h) == pytest.approx(4.0 * h * np.log(1.0 + np.sqrt(2.0)), rel=1e-14)


def test_line_hertz_deformation_converges():
    errs = []
    for N in (129, 513, 2049):
        xa, xb = -4.5, 1.5
        h = (xb - xa) / (N - 1)
        X = xa + h * np.arange(N)
        P = np.sqrt(np.maximum(0.0, 1.0 - X**2))
        D = kr.k_line(N, h) @ P
        mask = np.abs(X) <= 0.9
        errs.append(np.max(np.abs(D[mask] - kr.hertz_deform_line(X[mask]))))
        # film X^2/2 - D is flat inside the contact: H - H0 = 1/4 + ln(2)/2
        flat = 0.5 * X[mask] ** 2 - D[mask]
        assert np.max(np.abs(flat - (0.25 + 0.5 * np.log(2.0)))) < 5 * errs[-1] + 1e-12
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 2e-4


def test_point_hertz_deformation_converges():
    errs = []
    for n in (33, 65):
        h = 6.0 / (n - 1)
        x = -3.0 + h * np.arange(n)
        X, Y = np.meshgrid(x, x, indexing="ij")
        r = np.hypot(X, Y)
        P = np.sqrt(np.maximum(0.0, 1.0 - r**2))
        D = kr.deform_point(P, h)
        mask = r <= 0.8
        errs.append(np.max(np.abs(D[mask] - kr.hertz_deform_point(r[mask]))))
    assert errs[1] < errs[0] < 0.05


def test_point_deformation_direct_sum_small():
    """The per-offset organisation equals the literal quadruple sum."""
    rng = np.random.default_rng(3)
    P = rng.uniform(0, 1, (5, 4))
    h = 0.2
    D = kr.deform_point(P, h)
    ref = np.zeros_like(P)
    for i in range(5):
        for j in range(4):
            for k in range(5):
                for l in range(4):
                    ref[i, j] += (2 / np.pi**2) * kr.g_point(i - k, j - l, h) * P[k, l]
    assert np.max(np.abs(D - ref)) < 1e-14
