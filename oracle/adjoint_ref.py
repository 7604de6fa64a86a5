"""Sensitivities of the converged line-contact solution (test infrastructure).

The paper stops at the solution.  The derivatives here follow from the
discrete problem it states (Sec. 3.3 Example 6, Eqs. eqn19 and eqn62-eqn65,
with the line-contact force balance) by the implicit-function theorem:

at a converged ``(P, H0)`` let ``A`` be the rows whose equation is
``R_i = 0`` (``P_i > R_i / |dR_i/dP_i|``; elsewhere ``P_i = 0`` stays
fixed).  With unknowns ``x = (P_A, H0)`` and equations
``F(x; theta) = (R_A, h sum P - pi/2) = 0``, an objective ``J(P, H, H0)``
has ``dJ/dtheta = dJ/dtheta|_explicit - lam^T dF/dtheta`` where
``F_x^T lam = dJ/dx``.  ``theta`` is the roughness profile at every node,
the Moes load ``M`` and the lubricant parameter ``L``.

Dense matrices and ``numpy.linalg.solve`` throughout (plain, not fast).
"""
import numpy as np

from . import line_ref


def moes_line_log_derivatives(M, L):
    """``d ln(lambda)/d(M, L)`` and ``d ln(p_H)/d(M, L)`` for ``lambda = 3 pi^2/(8 M^2)``,
    ``p_H = alpha_bar / alpha``, ``alpha_bar = L sqrt(M / (2 pi))``."""
    return np.array([-2.0 / M, 0.0]), np.array([0.5 / M, 1.0 / L])


def tangent(pb, P_int, H0):
    """Exact partial derivatives of the interior residual ``R_1..R_{N-2}``.

    Returns a dict with ``P`` ([n, n], equal to ``line_ref.jacobian_exact``),
    ``H0`` ([n]), ``rough`` ([n, N]), ``M`` ([n]) and ``L`` ([n]), each on the
    limiter branch of the current state.  Forward mode over the columns
    ``(P_int, H0, rough, M, L)``: the film carries ``-K`` (P), ``1`` (H0) and
    the identity (rough); ``rho`` and ``eta`` depend on ``P p_H`` so that
    ``d/d ln p_H = P d/dP``; ``eps = rho H^3/(eta lambda)``.
    """
    s = line_ref.state(pb, P_int, H0)
    N, n, h = pb.N, pb.n, pb.h
    H, rho, eps, P = s["H"], s["rho"], s["eps"], s["P"]
    c = n + 1 + N + 2
    iP, iH0, iR, iM, iL = 0, n, n + 1, n + 1 + N, n + 2 + N
    dH = np.zeros((N, c))
    dH[:, iP:iP + n] = -pb.K[:, 1:-1]
    dH[:, iH0] = 1.0
    dH[:, iR:iR + N] = np.eye(N)
    dP = np.zeros((N, c))
    dP[1:-1, iP:iP + n] = np.eye(n)
    dlnlam = np.zeros(c)
    dlnpH = np.zeros(c)
    dlam_ML, dpH_ML = moes_line_log_derivatives(pb.M, pb.L)
    dlnlam[[iM, iL]] = dlam_ML
    dlnpH[[iM, iL]] = dpH_ML
    drho_dP, deta_dP, eta = s["drho"], s["deta"], s["eta"]
    drho = drho_dP[:, None] * dP + (drho_dP * P)[:, None] * dlnpH[None, :]
    dlneta = (deta_dP / eta)[:, None] * dP + (deta_dP / eta * P)[:, None] * dlnpH[None, :]
    deps = eps[:, None] * (drho / rho[:, None] + 3.0 * dH / H[:, None] - dlneta - dlnlam[None, :])
    du = drho * H[:, None] + rho[:, None] * dH
    # limited face values F_{j+1/2}, j = 0..N-2 (first-order at j = 0)
    dF = du[:-1].copy()
    j = np.arange(1, N - 1)
    pa, pbb = s["psi_a"], s["psi_b"]
    dF[1:] += 0.5 * (pa[1:, None] * (du[j] - du[j - 1]) + pbb[1:, None] * (du[j + 1] - du[j]))
    dC = (dF[1:] - dF[:-1]) / h
    depsf = 0.5 * (deps[:-1] + deps[1:])
    epsf = s["epsf"]
    dQ = (depsf[1:] * (P[2:] - P[1:-1])[:, None] + epsf[1:, None] * (dP[2:] - dP[1:-1])
          - depsf[:-1] * (P[1:-1] - P[:-2])[:, None] - epsf[:-1, None] * (dP[1:-1] - dP[:-2])) / h**2
    D = dC - dQ
    return dict(P=D[:, iP:iP + n], H0=D[:, iH0], rough=D[:, iR:iR + N], M=D[:, iM], L=D[:, iL])


def equation_rows(pb, P_int, H0, J=None):
    """Rows where ``R_i = 0`` is imposed: ``P_i > R_i / |dR_i/dP_i|``."""
    R = line_ref.residual(pb, P_int, H0)
    if J is None:
        J, _ = line_ref.jacobian_exact(pb, P_int, H0)
    d = np.abs(np.diag(J))
    d = np.where(d > 0.0, d, 1.0)
    return P_int > R / d


def adjoint(pb, P_int, H0, gP, gH, gH0):
    """Gradient of ``J(P, H, H0)`` with respect to roughness, ``M`` and ``L``.

    ``gP`` and ``gH`` ([N], nodal) and ``gH0`` (scalar) are the partial
    derivatives of ``J`` with ``P``, ``H`` and ``H0`` taken as independent;
    ``H = H0 + X^2/2 - K P + rough`` is chained here.  Returns a dict with
    ``rough`` ([N]), ``M``, ``L``, the multipliers ``lam`` ([n + 1], zero on
    rows that are not equations) and the equation-row mask ``rows``.
    """
    T = tangent(pb, P_int, H0)
    rows = equation_rows(pb, P_int, H0, T["P"])
    A = np.nonzero(rows)[0]
    na = len(A)
    Fx = np.zeros((na + 1, na + 1))
    Fx[:na, :na] = T["P"][np.ix_(A, A)]
    Fx[:na, na] = T["H0"][A]
    Fx[na, :na] = pb.h
    gP = np.asarray(gP, dtype=np.float64)
    gH = np.asarray(gH, dtype=np.float64)
    gPt = gP[1:-1] - pb.K[:, 1:-1].T @ gH          # dJ/dP_int through H as well
    gH0t = float(gH0) + float(np.sum(gH))           # dJ/dH0 through H as well
    rhs = np.concatenate([gPt[A], [gH0t]])
    lam_a = np.linalg.solve(Fx.T, rhs)
    lam = np.zeros(pb.n + 1)
    lam[A] = lam_a[:na]
    lam[pb.n] = lam_a[na]
    grad_rough = gH - lam_a[:na] @ T["rough"][A]
    grad_M = -float(lam_a[:na] @ T["M"][A])
    grad_L = -float(lam_a[:na] @ T["L"][A])
    return dict(rough=grad_rough, M=grad_M, L=grad_L, lam=lam, rows=rows)


def objective_seeds(pb, P_int, H0, which):
    """``(value, gP, gH, gH0)`` of ``H_c`` (H at X = 0), ``H_min`` (min_i H_i,
    the gradient of the minimising node) or ``P2`` (``h sum P_i^2``)."""
    N = pb.N
    H = pb.film(P_int, H0)
    gP, gH = np.zeros(N), np.zeros(N)
    if which == "H_c":
        c = int(np.argmin(np.abs(pb.X)))
        if abs(pb.X[c]) > 1e-12 * pb.h:
            raise ValueError("X = 0 is not a grid node")
        gH[c] = 1.0
        return float(H[c]), gP, gH, 0.0
    if which == "H_min":
        m = int(np.argmin(H))
        gH[m] = 1.0
        return float(H[m]), gP, gH, 0.0
    if which == "P2":
        P = pb.full(P_int)
        gP[:] = 2.0 * pb.h * P
        return float(pb.h * np.sum(P**2)), gP, gH, 0.0
    raise ValueError(which)
