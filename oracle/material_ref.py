"""Lubricant model and Moes parameter conversion (test infrastructure).

Sec. 3.3 (Examples 5 and 6) and Appendix A:

* ``eps = rho H^3 / (eta lambda)``;
* Roelands viscosity ``eta(P) = exp{(alpha p0 / z)(-1 + (1 + P p_H / p0)^z)}``
  with ``p0 = 1.98e8`` and ``z = 0.68``;
* Dowson-Higginson density
  ``rho(P) = (0.59e9 + 1.34 P p_H) / (0.59e9 + P p_H)``;
* incompressible / isoviscous option ``rho = eta = 1``.

The paper gives the Moes parameters ``M, L`` but not their conversion to the
dimensionless speed parameter ``lambda`` and ``alpha_bar = alpha p_H``.  The
conversions below follow from the definitions in Appendix A with Hertzian
scaling (line: half-width b, point: radius a):

* line   ``lambda = 3 pi^2 / (8 M^2)``,       ``alpha_bar = L sqrt(M / (2 pi))``;
* point  ``lambda = (128 pi^3 / (3 M^4))^{1/3}``, ``alpha_bar = (L/pi)(3M/2)^{1/3}``;

and ``p_H = alpha_bar / alpha``.
"""
import numpy as np

P0_ROELANDS = 1.98e8
Z_ROELANDS = 0.68


def moes_line(M, L):
    """``(lambda, alpha_bar)`` for line contact."""
    return 3.0 * np.pi**2 / (8.0 * M**2), L * np.sqrt(M / (2.0 * np.pi))


def moes_point(M, L):
    """``(lambda, alpha_bar)`` for point (circular) contact."""
    return (128.0 * np.pi**3 / (3.0 * M**4)) ** (1.0 / 3.0), (L / np.pi) * (1.5 * M) ** (1.0 / 3.0)


def viscosity(P, alpha_bar, alpha, p0=P0_ROELANDS, z=Z_ROELANDS):
    """Roelands ``eta(P)`` and ``d eta / dP``."""
    pH = alpha_bar / alpha
    base = 1.0 + np.asarray(P, dtype=np.float64) * pH / p0
    eta = np.exp((alpha * p0 / z) * (-1.0 + base**z))
    deta = eta * alpha * pH * base ** (z - 1.0)
    return eta, deta


def density(P, alpha_bar, alpha):
    """Dowson-Higginson ``rho(P)`` and ``d rho / dP``."""
    pH = alpha_bar / alpha
    P = np.asarray(P, dtype=np.float64)
    a = 0.59e9
    num = a + 1.34 * P * pH
    den = a + P * pH
    rho = num / den
    drho = a * (1.34 * pH - pH) / den**2
    return rho, drho


def material(P, alpha_bar, alpha, compressible=True, p0=P0_ROELANDS, z=Z_ROELANDS):
    """``(rho, drho/dP, eta, deta/dP)``; ``rho = eta = 1`` when not compressible."""
    P = np.asarray(P, dtype=np.float64)
    if not compressible:
        one = np.ones_like(P)
        zero = np.zeros_like(P)
        return one, zero, one, zero
    rho, drho = density(P, alpha_bar, alpha)
    eta, deta = viscosity(P, alpha_bar, alpha, p0, z)
    return rho, drho, eta, deta
