"""Pins of the adjoint oracle (sensitivities of the converged line-contact solution).

Independent checks:
* the forward-mode partial derivatives of R against central differences of
  the residual itself (roughness at single nodes, M and L through the Moes
  conversion) and against the exact P-Jacobian of the line oracle;
* the adjoint gradients of H_c, H_min and h sum P^2 against central
  differences of re-converged solutions (the forward solver alone).
"""
import numpy as np
import pytest

from oracle import adjoint_ref as ar
from oracle import line_ref as lr
from oracle import material_ref as mr
from paper_2008_03276_gb300 import inputs

N0, M0, L0 = 129, 20.0, 10.0


def rough_profile(N, seed=2):
    X = np.linspace(-4.5, 1.5, N)
    return inputs.sin_grf_roughness(X, seed=seed, amp=0.01, wavelength=0.5, sigma=0.005, corr=0.2)


def problem(M=M0, L=L0, rough=None, N=N0, limiter="minmod"):
    return lr.LineProblem(N, M, L, limiter=limiter, rough=rough)


@pytest.fixture(scope="module")
def converged():
    rgh = rough_profile(N0)
    pb = problem(rough=rgh)
    P, H0, info = lr.solve(pb, tol=1e-13)
    assert info["converged"]
    return pb, rgh, P, H0


def test_moes_log_derivatives_vs_central_differences():
    for M, L in [(20.0, 10.0), (200.0, 5.0)]:
        dlam, dpH = ar.moes_line_log_derivatives(M, L)
        for k, (dM, dL) in enumerate([(1e-6 * M, 0.0), (0.0, 1e-6 * L)]):
            lp, ap = mr.moes_line(M + dM, L + dL)
            lm, am = mr.moes_line(M - dM, L - dL)
            step = 2.0 * (dM + dL)
            assert abs((np.log(lp) - np.log(lm)) / step - dlam[k]) <= 1e-8 * max(1.0, abs(dlam[k]))
            assert abs((np.log(ap) - np.log(am)) / step - dpH[k]) <= 1e-8 * abs(dpH[k])


@pytest.mark.parametrize("limiter", ["minmod", "vanleer"])
def test_tangent_vs_residual_differences(converged, limiter):
    pb0, rgh, P, H0 = converged
    pb = problem(rough=rgh, limiter=limiter)
    # a state off the solution, so that every term is active
    rng = np.random.default_rng(3)
    Pt = np.clip(P * (1.0 + 0.02 * rng.standard_normal(pb.n)), 0.0, None)
    T = ar.tangent(pb, Pt, H0)
    J, JH = lr.jacobian_exact(pb, Pt, H0)
    assert np.allclose(T["P"], J, rtol=0, atol=1e-12 * np.max(np.abs(J)))
    assert np.allclose(T["H0"], JH, rtol=0, atol=1e-12 * np.max(np.abs(JH)))
    R0 = lr.residual(pb, Pt, H0)
    scale = np.max(np.abs(R0)) + 1.0
    for k in (5, 60, 96, 110):           # roughness at single nodes
        d = 1e-6
        rp, rm = rgh.copy(), rgh.copy()
        rp[k] += d
        rm[k] -= d
        fd = (lr.residual(problem(rough=rp, limiter=limiter), Pt, H0)
              - lr.residual(problem(rough=rm, limiter=limiter), Pt, H0)) / (2 * d)
        assert np.max(np.abs(fd - T["rough"][:, k])) <= 1e-6 * max(scale, np.max(np.abs(fd)))
    for name, (dM, dL) in (("M", (1e-6 * M0, 0.0)), ("L", (0.0, 1e-6 * L0))):
        fd = (lr.residual(problem(M0 + dM, L0 + dL, rgh, limiter=limiter), Pt, H0)
              - lr.residual(problem(M0 - dM, L0 - dL, rgh, limiter=limiter), Pt, H0)) / (2 * (dM + dL))
        assert np.max(np.abs(fd - T[name])) <= 1e-6 * max(1.0, np.max(np.abs(fd)))


def _value(which, M=M0, L=L0, rough=None, P0=None, H00=None):
    pb = problem(M, L, rough)
    P, H0, info = lr.solve(pb, P_init=P0, H0_init=H00, tol=1e-13)
    assert info["converged"]
    return ar.objective_seeds(pb, P, H0, which)[0]


@pytest.mark.slow
@pytest.mark.parametrize("which", ["H_c", "H_min", "P2"])
def test_adjoint_vs_resolved_differences(converged, which):
    pb, rgh, P, H0 = converged
    val, gP, gH, gH0 = ar.objective_seeds(pb, P, H0, which)
    g = ar.adjoint(pb, P, H0, gP, gH, gH0)
    # roughness at nodes in the inlet, the Hertzian zone and the outlet; the step is
    # small because the minmod branches and the cavitation boundary make the
    # solution only piecewise smooth in the data
    d = 1e-6
    for k in (40, 90, 100):
        rp, rm = rgh.copy(), rgh.copy()
        rp[k] += d
        rm[k] -= d
        fd = (_value(which, rough=rp, P0=P, H00=H0) - _value(which, rough=rm, P0=P, H00=H0)) / (2 * d)
        assert abs(fd - g["rough"][k]) <= 1e-5 * abs(fd) + 1e-7 * np.max(np.abs(g["rough"])), (k, fd, g["rough"][k])
    for name, (dM, dL) in (("M", (1e-6 * M0, 0.0)), ("L", (0.0, 1e-6 * L0))):
        fd = (_value(which, M0 + dM, L0 + dL, rgh, P, H0) - _value(which, M0 - dM, L0 - dL, rgh, P, H0)) / (2 * (dM + dL))
        assert abs(fd - g[name]) <= 1e-5 * abs(fd), (name, fd, g[name])


def test_adjoint_multipliers_solve_the_transposed_system(converged):
    pb, rgh, P, H0 = converged
    _, gP, gH, gH0 = ar.objective_seeds(pb, P, H0, "H_c")
    g = ar.adjoint(pb, P, H0, gP, gH, gH0)
    rows = g["rows"]
    # cavitated rows carry no multiplier; the equation rows cover the pressure zone
    assert np.all(g["lam"][:-1][~rows] == 0.0)
    assert np.all(P[rows] > 0.0)
    assert rows.sum() > pb.n // 4
