"""Pins of the point-contact oracle (residual, exact Jacobian, dense solve).

Independent checks:
* reduction to line contact: with rigid surfaces, a roughness that cancels
  the Y^2/2 term and a pressure that does not depend on Y, the 2-D residual
  on rows away from the y-boundaries equals the line oracle's residual
  (limited x-flux and x-Poiseuille term), i.e. the y-Poiseuille term vanishes;
* the y-Poiseuille term against a hand-evaluated 5-point sum at one node;
* the exact Jacobian against central differences of the residual;
* the converged solution: complementarity, the force balance 2 pi / 3, the
  mirror symmetry Y -> -Y of the problem, and agreement of the nested
  iteration with the direct solve.
"""
import numpy as np
import pytest

from oracle import line_ref as lr
from oracle import point_ref as pr


def test_point_residual_reduces_to_line_contact():
    nx, ny, M, L = 65, 17, 20.0, 10.0
    pb = pr.PointProblem(nx, ny, M, L, elastic=False, limiter="vanleer")
    X, Y = np.meshgrid(pb.X, pb.Y, indexing="ij")
    pb.rough = -0.5 * Y**2
    rng = np.random.default_rng(0)
    p = np.clip(np.sqrt(np.clip(1 - pb.X**2, 0, None)) * (1 + 0.1 * rng.standard_normal(nx)), 0, None)
    p[0] = p[-1] = 0.0
    P = np.tile(p[:, None], (1, ny))
    P[:, 0] = P[:, -1] = 0.0
    H0 = 0.3
    R2 = pr.residual(pb, P[1:-1, 1:-1].ravel(), H0).reshape(nx - 2, ny - 2)
    pl = lr.LineProblem(nx, M, L, elastic=False, limiter="vanleer")
    pl.lam, pl.abar = pb.lam, pb.abar           # the point-contact lubricant constants
    R1 = lr.residual(pl, p[1:-1], H0)
    for j in range(2, ny - 2):                   # node rows whose y-neighbours are interior
        assert np.max(np.abs(R2[:, j - 1] - R1)) <= 1e-12 * np.max(np.abs(R1))


def test_point_y_poiseuille_term_by_hand():
    pb = pr.PointProblem(17, 17, 20.0, 10.0, elastic=False)
    rng = np.random.default_rng(1)
    P_int = rng.uniform(0.1, 1.0, pb.n)
    H0 = 0.4
    s = pr.state(pb, P_int, H0)
    i, j = 7, 9
    e, P, h = s["eps"], s["P"], pb.h
    eyp, eym = 0.5 * (e[i, j] + e[i, j + 1]), 0.5 * (e[i, j] + e[i, j - 1])
    exp_, exm = 0.5 * (e[i, j] + e[i + 1, j]), 0.5 * (e[i, j] + e[i - 1, j])
    Qy = (eyp * (P[i, j + 1] - P[i, j]) - eym * (P[i, j] - P[i, j - 1])) / h**2
    Qx = (exp_ * (P[i + 1, j] - P[i, j]) - exm * (P[i, j] - P[i - 1, j])) / h**2
    C = (s["F"][i, j] - s["F"][i - 1, j]) / h
    assert s["R"][i - 1, j - 1] == pytest.approx(C - Qx - Qy, rel=1e-13, abs=1e-13 * abs(Qy))


@pytest.mark.parametrize("limiter", ["minmod", "vanleer"])
def test_point_jacobian_vs_central_differences(limiter):
    pb = pr.PointProblem(17, 17, 20.0, 10.0, limiter=limiter)
    rng = np.random.default_rng(2)
    P_int = pb.hertz() * (1 + 0.05 * rng.standard_normal(pb.n)).clip(0)
    H0 = pb.h0_for_min_film(P_int, 0.1)
    J, JH = pr.jacobian_exact(pb, P_int, H0, block=37)
    scale = np.max(np.abs(J))
    for col in (0, 37, 100, 112, pb.n - 1):
        d = 1e-6 * max(1.0, abs(P_int[col]))
        Pp, Pm = P_int.copy(), P_int.copy()
        Pp[col] += d
        Pm[col] -= d
        fd = (pr.residual(pb, Pp, H0) - pr.residual(pb, Pm, H0)) / (2 * d)
        assert np.max(np.abs(fd - J[:, col])) <= 1e-6 * scale
    fd = (pr.residual(pb, P_int, H0 + 1e-6) - pr.residual(pb, P_int, H0 - 1e-6)) / 2e-6
    assert np.max(np.abs(fd - JH)) <= 1e-6 * np.max(np.abs(JH))


def test_point_hertz_start_gives_flat_film():
    # the Hertzian pressure deforms the surface by 1 - r^2/2 inside the contact,
    # so H = H0 + 1 there up to the discretisation error
    pb = pr.PointProblem(65, 65, 100.0, 10.0, xa=-2.0, xb=2.0, ya=-2.0)
    P = pb.hertz()
    H = pb.film(P, 0.0)
    X, Y = np.meshgrid(pb.X, pb.Y, indexing="ij")
    inside = X**2 + Y**2 < 0.6
    assert np.max(np.abs(H[inside] - 1.0)) < 0.03


@pytest.fixture(scope="module")
def solved_33():
    pb = pr.PointProblem(33, 33, 20.0, 10.0)
    P, H0, info = pr.solve(pb, tol=1e-11)
    return pb, P, H0, info


def test_point_solution_complementarity_force_symmetry(solved_33):
    pb, P, H0, info = solved_33
    assert info["converged"]
    R = pr.residual(pb, P, H0)
    assert np.min(P) >= 0.0
    assert np.max(np.abs(np.minimum(P, R))) <= max(1e-11, pr.rounding_floor(pb, P, H0))
    assert abs(pb.h**2 * P.sum() - 2 * np.pi / 3) <= 1e-12
    Pg = pb.full(P)
    assert np.max(np.abs(Pg - Pg[:, ::-1])) <= 1e-8 * np.max(Pg)   # Y -> -Y
    assert np.argmax(Pg.max(axis=1)) > np.argmin(np.abs(pb.X))       # pressure peak downstream of X = 0


def test_point_nested_matches_direct(solved_33):
    pb, P, H0, info = solved_33
    fac = lambda gx, gy: pr.PointProblem(gx, gy, 20.0, 10.0)
    pbn, Pn, H0n, inf = pr.solve_nested(fac, 33, 33, n_min=17, tol=1e-11)
    assert inf["converged"] and [l[0] for l in inf["levels"]] == [(17, 17), (33, 33)]
    assert np.max(np.abs(Pn - P)) <= 1e-8 * np.max(P)
    assert abs(H0n - H0) <= 1e-8 * abs(H0)


def test_point_parameter_tangents_vs_residual_differences(solved_33):
    pb, P, H0, info = solved_33
    s = pr.state(pb, P, H0)
    dlam, dpH = pr.moes_point_log_derivatives(pb.M, pb.L)
    T = pr._tangent(pb, s, np.zeros((pb.nx, pb.ny, 2)), np.zeros((pb.nx, pb.ny, 2)), dlnpH=dpH, dlnlam=dlam)
    for k, (dM, dL) in enumerate([(1e-6 * pb.M, 0.0), (0.0, 1e-6 * pb.L)]):
        Rp = pr.residual(pr.PointProblem(pb.nx, pb.ny, pb.M + dM, pb.L + dL), P, H0)
        Rm = pr.residual(pr.PointProblem(pb.nx, pb.ny, pb.M - dM, pb.L - dL), P, H0)
        fd = (Rp - Rm) / (2 * (dM + dL))
        assert np.max(np.abs(fd - T[:, k])) <= 1e-6 * max(1.0, np.max(np.abs(fd)))


@pytest.mark.slow
def test_point_adjoint_vs_resolved_differences(solved_33):
    pb, P, H0, info = solved_33
    c = (int(np.argmin(np.abs(pb.X))), int(np.argmin(np.abs(pb.Y))))
    gH = np.zeros((pb.nx, pb.ny))
    gH[c] = 1.0                                   # H_c = H at (0, 0)
    g = pr.adjoint(pb, P, H0, np.zeros_like(gH), gH, 0.0)

    def hc(M=pb.M, L=pb.L, rough=None):
        q = pr.PointProblem(pb.nx, pb.ny, M, L, rough=rough)
        Pq, H0q, inf = pr.solve(q, P_init=P, H0_init=H0, tol=1e-12)
        assert inf["converged"]
        return q.film(Pq, H0q)[c]

    d = 1e-6
    for node in ((c[0], c[1]), (c[0] - 3, c[1] + 2)):
        rp, rm = np.zeros((pb.nx, pb.ny)), np.zeros((pb.nx, pb.ny))
        rp[node] += d
        rm[node] -= d
        fd = (hc(rough=rp) - hc(rough=rm)) / (2 * d)
        assert abs(fd - g["rough"][node]) <= 1e-5 * abs(fd) + 1e-7 * np.max(np.abs(g["rough"]))
    fd = (hc(M=pb.M * (1 + d)) - hc(M=pb.M * (1 - d))) / (2 * d * pb.M)
    assert abs(fd - g["M"]) <= 1e-5 * abs(fd)
    fd = (hc(L=pb.L * (1 + d)) - hc(L=pb.L * (1 - d))) / (2 * d * pb.L)
    assert abs(fd - g["L"]) <= 1e-5 * abs(fd)


@pytest.mark.parametrize("n,beta,limiter", [(17, 2, "minmod"), (21, 3, "vanleer")])
def test_xline_band_is_the_band_of_the_dense_exact_jacobian(n, beta, limiter):
    pb = pr.PointProblem(n, n, 20.0, 10.0, limiter=limiter)
    rng = np.random.default_rng(n)
    P = pb.hertz() * (1 + 0.05 * rng.standard_normal(pb.n)).clip(0)
    H0 = pb.h0_for_min_film(P, 0.1)
    J, _ = pr.jacobian_exact(pb, P, H0)
    band = pr.xline_band_exact(pb, P, H0, beta)
    m = n - 2
    for j in range(m):
        for i in range(m):
            for d in range(-beta, beta + 1):
                k = i + d
                want = J[i * m + j, k * m + j] if 0 <= k < m else 0.0
                assert band[j, i, beta + d] == want


@pytest.mark.parametrize("n,beta,limiter", [(17, 2, "minmod"), (21, 3, "vanleer")])
def test_yline_band_is_the_band_of_the_dense_exact_jacobian(n, beta, limiter):
    pb = pr.PointProblem(n, n, 20.0, 10.0, limiter=limiter)
    rng = np.random.default_rng(n + 1)
    P = pb.hertz() * (1 + 0.05 * rng.standard_normal(pb.n)).clip(0)
    H0 = pb.h0_for_min_film(P, 0.1)
    J, _ = pr.jacobian_exact(pb, P, H0)
    band = pr.yline_band_exact(pb, P, H0, beta)
    m = n - 2
    for i in range(m):
        for j in range(m):
            for d in range(-beta, beta + 1):
                l = j + d
                want = J[i * m + j, i * m + l] if 0 <= l < m else 0.0
                assert band[i, j, beta + d] == want
