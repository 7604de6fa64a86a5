"""Pins of the lubricant model's pressure dependence (Sec. 3.3, Examples 5 and 6;
Appendix A: Roelands viscosity with p0 = 1.98e8, z = 0.68, Dowson-Higginson
density, p_H = alpha_bar / alpha).

Each pin is a value the mathematics fixes, worked out by hand from the
dimensional formulas, not a re-evaluation of the oracle's expression:

* Barus slope: d ln(eta) / dP at P = 0 equals alpha p_H = alpha_bar, for any
  p0 and z;
* curvature: d^2 ln(eta) / dP^2 at P = 0 equals alpha (z - 1) p_H^2 / p0;
* at the dimensional pressure p = p0 (2^{1/z} - 1) the Roelands exponent is
  alpha p0 / z = 4.95 for alpha = 1.7e-8; at p = p0 (3^{1/z} - 1) it is 9.9;
* Dowson-Higginson: rho = 1.17 at p = 0.59 GPa, 3.68 / 3 at p = 1.18 GPa, the
  slope 0.34 p_H / 0.59e9 at P = 0 and the limit 1.34;

all at two values of alpha_bar (so p_H takes two values and a slip between
alpha_bar and p_H moves the dimensionless pressure at which a hand value
holds).  The planted-mistake test shows that each plausible slip in the
oracle's formulas fails at least one pin.
"""
import math

import numpy as np
import pytest

from oracle import material_ref as mr

ALPHA = 1.7e-8
P0 = 1.98e8
Z = 0.68
ABARS = (17.84, 31.0)  # C1's alpha_bar and a second, larger one


def _pin_failures(viscosity, density):
    """Names of the pins that the pair (viscosity, density) fails."""
    bad = []
    for abar in ABARS:
        pH = abar / ALPHA
        # Barus slope and curvature at P = 0, from eta'/eta and a central
        # difference of eta'/eta (the analytic derivative the oracle returns)
        eta0, deta0 = viscosity(np.array([0.0]), abar, ALPHA)
        if abs(deta0[0] / eta0[0] - abar) > 1e-12 * abar:
            bad.append("barus_slope")
        e = 1e-5
        etap, detap = viscosity(np.array([e]), abar, ALPHA)
        etam, detam = viscosity(np.array([-e]), abar, ALPHA)
        curv = (detap[0] / etap[0] - detam[0] / etam[0]) / (2 * e)
        curv_hand = ALPHA * (Z - 1.0) * pH**2 / P0
        if abs(curv - curv_hand) > 1e-6 * abs(curv_hand):
            bad.append("curvature")
        # hand values of the exponent: (1 + p/p0)^z = 2 and 3
        for k, lneta_hand in ((2.0, 4.95), (3.0, 9.9)):
            p = P0 * (k ** (1.0 / Z) - 1.0)
            eta, _ = viscosity(np.array([p / pH]), abar, ALPHA)
            if abs(math.log(eta[0]) - lneta_hand) > 1e-12 * lneta_hand:
                bad.append(f"eta_at_{k:g}")
        # Dowson-Higginson hand values
        for p, rho_hand in ((0.59e9, 1.17), (1.18e9, 3.68 / 3.0)):
            rho, _ = density(np.array([p / pH]), abar, ALPHA)
            if abs(rho[0] - rho_hand) > 1e-14:
                bad.append(f"rho_at_{p:g}")
        _, drho0 = density(np.array([0.0]), abar, ALPHA)
        if abs(drho0[0] - 0.34 * pH / 0.59e9) > 1e-13 * (0.34 * pH / 0.59e9):
            bad.append("rho_slope")
        rho_big, drho_big = density(np.array([1e6]), abar, ALPHA)
        if abs(rho_big[0] - 1.34) > 1e-6:
            bad.append("rho_limit")
        # the returned derivatives against central differences (the slopes of
        # the functions the pins above fix)
        P = np.linspace(0.05, 3.0, 9)
        h = 1e-6
        _, dr = density(P, abar, ALPHA)
        rp, _ = density(P + h, abar, ALPHA)
        rm, _ = density(P - h, abar, ALPHA)
        if not np.allclose(dr, (rp - rm) / (2 * h), rtol=1e-6, atol=0):
            bad.append("drho_fd")
        _, de = viscosity(P, abar, ALPHA)
        ep, _ = viscosity(P + h, abar, ALPHA)
        em, _ = viscosity(P - h, abar, ALPHA)
        if not np.allclose(de, (ep - em) / (2 * h), rtol=1e-6, atol=0):
            bad.append("deta_fd")
    return sorted(set(bad))


def test_oracle_material_meets_every_pin():
    assert _pin_failures(mr.viscosity, mr.density) == []


def test_material_combines_the_pinned_functions():
    P = np.linspace(0.0, 2.0, 5)
    rho, drho, eta, deta = mr.material(P, ABARS[0], ALPHA)
    r, dr = mr.density(P, ABARS[0], ALPHA)
    e, de = mr.viscosity(P, ABARS[0], ALPHA)
    assert np.array_equal(rho, r) and np.array_equal(drho, dr)
    assert np.array_equal(eta, e) and np.array_equal(deta, de)
    assert (mr.P0_ROELANDS, mr.Z_ROELANDS) == (P0, Z)


# --- planted mistakes: each is a plausible slip in the oracle's formulas ----------------------

def _visc(slip):
    def viscosity(P, abar, alpha):
        pH = abar / alpha
        P = np.asarray(P, dtype=np.float64)
        p0, z, scale = P0, Z, pH
        if slip == "abar_for_pH":
            scale = abar
        elif slip == "z":
            z = 0.6
        elif slip == "p0":
            p0 = 1.96e8
        base = 1.0 + P * scale / p0
        c = alpha * p0 / z
        if slip == "exponent_no_z":
            c = alpha * p0
        eta = np.exp(c * (-1.0 + base**z))
        deta = eta * c * z * (scale / p0) * base ** (z - 1.0)
        if slip == "deta_power":
            deta = eta * c * z * (scale / p0) * base**z
        return eta, deta

    return viscosity


def _dens(slip):
    def density(P, abar, alpha):
        pH = abar / alpha
        P = np.asarray(P, dtype=np.float64)
        a = 0.59e8 if slip == "a_1e8" else 0.59e9
        k = 1.34 if slip != "k" else 1.43
        scale = abar if slip == "abar_for_pH" else pH
        num = a + k * P * scale
        den = a + P * scale
        rho = num / den
        drho = a * (k - 1.0) * scale / den**2
        if slip == "drho_sign":
            drho = -drho
        return rho, drho

    return density


def test_slip_free_restatement_meets_the_pins():
    # the helpers below are only useful if their unslipped form passes
    assert _pin_failures(_visc(None), _dens(None)) == []


@pytest.mark.parametrize("slip", ["abar_for_pH", "z", "p0", "exponent_no_z", "deta_power"])
def test_viscosity_slips_fail_a_pin(slip):
    assert _pin_failures(_visc(slip), mr.density) != []


@pytest.mark.parametrize("slip", ["abar_for_pH", "a_1e8", "k", "drho_sign"])
def test_density_slips_fail_a_pin(slip):
    assert _pin_failures(mr.viscosity, _dens(slip)) != []
