"""Linear convection-diffusion workload of the AQIF line splittings (test infrastructure).

Sec. 3.1, Examples 1 and 2:  L u = (a u)_x + (b u)_y - eps (u_xx + u_yy) = f on
Omega = [-1, 1]^2, u = g on the boundary; Sec. 6 (numerical results): the exact
solution u = x^4 + y^4, eps = 1e-6, kappa in {0, 1/3, -1}, splittings Ls0 and
Ls1.  Constant a > 0, b >= 0 (the paper's printed splittings carry no y-convection
term, which makes b = 0 the reading of its experiments).

Discretisation (Sec. 3.1, Eqs. eqn41, eqn42, eqn46, eqn47): van Leer's kappa-scheme
for the convective term through the face value
    F_{i+1/2} = u_i + (1 - kappa)/4 (u_i - u_{i-1}) + (1 + kappa)/4 (u_{i+1} - u_i),
    (a u)_x ~ a (F_{i+1/2} - F_{i-1/2}) / h,
which expands to the printed stencil (kappa = 0: a/h [0.25, -1.25, 0.75, 0.25, 0]);
at the inflow face, whose stencil leaves the grid, the missing node is the linear
extrapolation u_{-1} = 2 u_0 - u_1 (the boundary value alone, F_{1/2} = u_0, would make
the scheme inconsistent at the first interior node).  The same in y with b.  Diffusion: the
5-point Laplacian.  Arrays are [nx, ny] with x first.

Line relaxation (Sec. 3.1): the operator is split as L = L^+ + L^0 + L^- with
  L^0  the x-line operator of the splitting (tridiagonal): the first-order upwind
       difference c (u_i - u_{i-1}) a / h with c = (2 - kappa)/2 (Ls1, Eq. eqn49) or
       (2 - kappa)/2 + (1 - kappa)/4 (Ls0, Eq. eqn48), plus the x part and the
       diagonal of the diffusion (-eps/h^2, 4 eps/h^2, -eps/h^2);
  L^+  the couplings to the lines below (j - 1, j - 2: diffusion and the upwind
       y-convection), taken at the new iterate;
  L^-  everything else, L - L^0 - L^+ (the identity the paper states; its printed
       L^- coefficients do not add up to the kappa-scheme, see the readings).
One sweep solves, line by line in increasing y (the paper's lexicographic order),
  L^0 sigma = f - L^- u^n - L^0 u^n - L^+ u^{n+1},   u^{n+1} = u^n + omega sigma,
which with the iterate held in place is the current residual of the line; the
"jacobi" order solves every line from the same iterate.  Each line system is
solved by dense LU (a library primitive) in place of AQIF.
"""
import numpy as np


class CDProblem:
    """Grid, coefficients and data of one instance (nx = ny = N nodes incl. boundary)."""

    def __init__(self, N, a=1.0, b=0.0, eps=1e-6, kappa=0.0, lo=-1.0, hi=1.0):
        if a <= 0 or b < 0:
            raise ValueError("the scheme is written for a > 0, b >= 0")
        self.N = int(N)
        self.h = (hi - lo) / (self.N - 1)
        self.x = lo + self.h * np.arange(self.N)
        self.a, self.b, self.eps, self.kappa = float(a), float(b), float(eps), float(kappa)
        X, Y = np.meshgrid(self.x, self.x, indexing="ij")
        self.u_exact = X**4 + Y**4
        # f = (a u)_x + (b u)_y - eps Lap u for the exact solution
        self.f = self.a * 4 * X**3 + self.b * 4 * Y**3 - self.eps * 12 * (X**2 + Y**2)

    def initial(self):
        """Boundary values of the exact solution, zero inside."""
        u = self.u_exact.copy()
        u[1:-1, 1:-1] = 0.0
        return u


def face_values(u, kappa, axis):
    """F at the faces k+1/2, k = 0..N-2, along `axis` (Eq. eqn41).

    The inflow face k = 0 needs u_{-1}, outside the grid; it is the linear
    extrapolation 2 u_0 - u_1, which makes F_{1/2} = (u_0 + u_1) / 2 for every kappa.
    """
    v = np.moveaxis(u, axis, 0)
    ghost = 2.0 * v[0] - v[1]
    w = np.concatenate([ghost[None], v], axis=0)  # w[k + 1] = v[k]
    k = np.arange(1, w.shape[0] - 1)  # faces of v-nodes 0..N-2
    F = (w[k] + 0.25 * (1.0 - kappa) * (w[k] - w[k - 1])
         + 0.25 * (1.0 + kappa) * (w[k + 1] - w[k]))
    return np.moveaxis(F, 0, axis)


def apply(pb, u):
    """L_kappa u at the interior nodes ([N-2, N-2])."""
    h = pb.h
    Fx = face_values(u, pb.kappa, 0)  # [N-1, N]
    Fy = face_values(u, pb.kappa, 1)  # [N, N-1]
    conv = pb.a * (Fx[1:, 1:-1] - Fx[:-1, 1:-1]) / h + pb.b * (Fy[1:-1, 1:] - Fy[1:-1, :-1]) / h
    lap = (u[2:, 1:-1] + u[:-2, 1:-1] + u[1:-1, 2:] + u[1:-1, :-2] - 4.0 * u[1:-1, 1:-1]) / h**2
    return conv - pb.eps * lap


def residual(pb, u):
    """f - L_kappa u at the interior nodes."""
    return pb.f[1:-1, 1:-1] - apply(pb, u)


def l0_coefficient(kappa, splitting):
    """c of the upwind difference c (u_i - u_{i-1}) kept in the line operator L^0."""
    c = (2.0 - kappa) / 2.0
    if splitting == "Ls0":
        return c + (1.0 - kappa) / 4.0
    if splitting == "Ls1":
        return c
    raise ValueError(splitting)


def line_matrix(pb, splitting):
    """L^0 of one x-line: dense [N-2, N-2] (tridiagonal)."""
    n = pb.N - 2
    c = l0_coefficient(pb.kappa, splitting) * pb.a / pb.h
    d = pb.eps / pb.h**2
    A = np.zeros((n, n))
    for i in range(n):
        A[i, i] = c + 4.0 * d
        if i > 0:
            A[i, i - 1] = -c - d
        if i + 1 < n:
            A[i, i + 1] = -d
    return A


def line_relaxation(pb, splitting="Ls1", order="lexicographic", omega=1.0, sweeps=20, u0=None, tol=0.0):
    """The paper's x-line relaxation in change form; returns ``(u, hist)`` with
    ``hist[k] = ||f - L u||_inf`` after k sweeps (hist[0] at the start)."""
    u = pb.initial() if u0 is None else np.array(u0, dtype=np.float64)
    A = line_matrix(pb, splitting)
    hist = [float(np.max(np.abs(residual(pb, u))))]
    for _ in range(sweeps):
        if order == "lexicographic":
            for j in range(1, pb.N - 1):
                rj = residual(pb, u)[:, j - 1]
                u[1:-1, j] += omega * np.linalg.solve(A, rj)
        elif order == "jacobi":
            r = residual(pb, u)
            u[1:-1, 1:-1] += omega * np.linalg.solve(A, r)
        else:
            raise ValueError(order)
        hist.append(float(np.max(np.abs(residual(pb, u)))))
        if hist[-1] <= tol:
            break
    return u, hist


def operator_matrix(pb):
    """Dense L_kappa on the interior unknowns (C order [N-2, N-2]) and the boundary part
    ``L u_b`` of the boundary data, column by column from ``apply`` (small N only)."""
    n = pb.N - 2
    ub = pb.initial()
    base = apply(pb, ub).ravel()
    A = np.zeros((n * n, n * n))
    for c in range(n * n):
        u = ub.copy()
        u[1 + c // n, 1 + c % n] += 1.0
        A[:, c] = apply(pb, u).ravel() - base
    return A, base


def solve_direct(pb):
    """The discrete solution of L_kappa u = f with the boundary data, by dense LU."""
    A, base = operator_matrix(pb)
    u = pb.initial()
    u[1:-1, 1:-1] = np.linalg.solve(A, pb.f[1:-1, 1:-1].ravel() - base).reshape(pb.N - 2, pb.N - 2)
    return u
