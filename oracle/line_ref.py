"""Line-contact EHL: discrete residual, Jacobians and an independent solve (test infrastructure).

Discrete problem (Sec. 3.3 Example 6, Sec. 3.3.1, Sec. 3.3.3):
grid ``X_i = xa + i h``, ``i = 0..N-1``, ``h = (xb - xa)/(N - 1)``,
``P_0 = P_{N-1} = 0``; unknowns ``P_1..P_{N-2}`` and ``H0``.

* film ``H_i = H0 + X_i^2/2 - sum_k K[i,k] P_k + rough_i`` (Eq. eqn19, Case 1);
* ``u_k = rho_k H_k``; limited face value (Eqs. eqn64-eqn65, in the standard
  upwind form with the symmetric limiter function ``psi(a, b)``)
  ``F_{i+1/2} = u_i + psi(u_i - u_{i-1}, u_{i+1} - u_i) / 2`` for ``i >= 1``
  and the first-order ``F_{1/2} = u_0`` at the inflow face whose stencil
  leaves the grid;  minmod ``psi = sgn(a) min(|a|, |b|)`` if ``ab > 0``,
  van Leer ``psi = 2ab/(a+b)`` if ``ab > 0``, else ``psi = 0``;
* half-node coefficient ``eps_{i+1/2} = (eps_i + eps_{i+1})/2`` (Eq. eqn63);
* residual per unit length
  ``R_i = (F_{i+1/2} - F_{i-1/2})/h
         - [eps_{i+1/2}(P_{i+1}-P_i) - eps_{i-1/2}(P_i-P_{i-1})]/h^2``;
* complementarity ``P_i >= 0, R_i >= 0, P_i R_i = 0`` (Example 6) and force
  balance ``h sum_i P_i = pi/2``.

The oracle solves this by a dense semismooth Newton method on
``Phi = (min(P, R), h sum P - pi/2)`` with the exact Jacobian (every
dependence on P included) and dense LU, which is a different iteration from
the banded limiter-based Newton-Raphson method of Sec. 3.3.3-3.3.4; agreement
therefore pins the fixed point, not the path.
"""
import numpy as np

from . import kernels_ref, material_ref


class LineProblem:
    """Grid, kernel and lubricant constants of one line-contact instance."""

    def __init__(self, N, M, L, xa=-4.5, xb=1.5, alpha=1.7e-8, compressible=True,
                 elastic=True, limiter="minmod", rough=None, switch_eps_h=0.6,
                 dist_weight=0.25, kappa=0.0, splitting="frozen"):
        self.N = int(N)
        self.n = self.N - 2
        self.M, self.L = float(M), float(L)
        self.xa, self.xb = float(xa), float(xb)
        self.h = (self.xb - self.xa) / (self.N - 1)
        self.X = self.xa + self.h * np.arange(self.N)
        self.alpha = float(alpha)
        self.lam, self.abar = material_ref.moes_line(self.M, self.L)
        self.compressible = bool(compressible)
        self.elastic = bool(elastic)
        if limiter not in ("minmod", "vanleer", "kappa"):
            raise ValueError(limiter)
        if splitting not in ("frozen", "hs1", "hs2"):
            raise ValueError(splitting)
        self.limiter = limiter
        self.kappa = float(kappa)
        self.splitting = splitting
        self.rough = np.zeros(self.N) if rough is None else np.asarray(rough, dtype=np.float64)
        self.K = kernels_ref.k_line(self.N, self.h) if self.elastic else np.zeros((self.N, self.N))
        self.switch_eps_h = float(switch_eps_h)
        self.dist_weight = float(dist_weight)
        self.load = np.pi / 2.0

    # ------------------------------------------------------------------ helpers
    def full(self, P_int):
        """Interior vector (n) -> nodal vector (N) with zero Dirichlet ends."""
        P = np.zeros(self.N)
        P[1:-1] = P_int
        return P

    def hertz(self):
        """Hertzian start ``P = sqrt(max(0, 1 - X^2))`` (Sec. 4), interior part."""
        return np.sqrt(np.maximum(0.0, 1.0 - self.X**2))[1:-1]

    def film(self, P_int, H0):
        """``H = H0 + X^2/2 - K P + rough`` at all N nodes (Eq. eqn19, Case 1)."""
        return H0 + 0.5 * self.X**2 - self.K @ self.full(P_int) + self.rough

    def h0_for_min_film(self, P_int, h_init):
        """``H0`` such that ``min_i H_i = h_init`` at pressure ``P_int``."""
        H = self.film(P_int, 0.0)
        return h_init - np.min(H)


def limiter(a, b, kind, kappa=0.0):
    """``psi(a, b)`` and its partial derivatives (piecewise, exact on each branch).

    ``kind`` "minmod" or "vanleer" (limited, Sec. 3.3.3), or "kappa": van Leer's
    unlimited kappa-scheme, whose face value ``u_i + (1 - kappa)/4 a + (1 + kappa)/4 b``
    (Sec. 3.1, Eq. eqn41; Sec. 3.3.2, Eq. eqn56) is ``u_i + psi / 2`` with the linear
    ``psi = ((1 - kappa) a + (1 + kappa) b) / 2``.
    """
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if kind == "kappa":
        da = np.full(a.shape, 0.5 * (1.0 - kappa))
        db = np.full(b.shape, 0.5 * (1.0 + kappa))
        return da * a + db * b, da, db
    same = a * b > 0.0
    if kind == "minmod":
        use_a = np.abs(a) <= np.abs(b)
        psi = np.where(same, np.where(use_a, a, b), 0.0)
        da = np.where(same & use_a, 1.0, 0.0)
        db = np.where(same & ~use_a, 1.0, 0.0)
    else:
        s = np.where(same, a + b, 1.0)
        psi = np.where(same, 2.0 * a * b / s, 0.0)
        da = np.where(same, 2.0 * b * b / s**2, 0.0)
        db = np.where(same, 2.0 * a * a / s**2, 0.0)
    return psi, da, db


def state(pb, P_int, H0):
    """All nodal quantities of the discrete residual at ``(P, H0)``."""
    P = pb.full(P_int)
    H = pb.film(P_int, H0)
    rho, drho, eta, deta = material_ref.material(P, pb.abar, pb.alpha, pb.compressible)
    eps = rho * H**3 / (eta * pb.lam)
    u = rho * H
    N, h = pb.N, pb.h
    # faces i+1/2, i = 0..N-2
    a = np.zeros(N - 1)
    b = np.zeros(N - 1)
    a[1:] = u[1:-1] - u[:-2]
    b[1:] = u[2:] - u[1:-1]
    psi, pa, pbb = limiter(a, b, pb.limiter, pb.kappa)
    psi[0] = 0.0
    pa[0] = 0.0
    pbb[0] = 0.0
    F = u[:-1] + 0.5 * psi
    epsf = 0.5 * (eps[:-1] + eps[1:])
    C = (F[1:] - F[:-1]) / h
    Q = (epsf[1:] * (P[2:] - P[1:-1]) - epsf[:-1] * (P[1:-1] - P[:-2])) / h**2
    R = C - Q
    return dict(P=P, H=H, rho=rho, drho=drho, eta=eta, deta=deta, eps=eps, u=u,
                a=a, b=b, psi=psi, psi_a=pa, psi_b=pbb, F=F, epsf=epsf, R=R)


def residual(pb, P_int, H0):
    """Interior residual ``R_1..R_{N-2}`` (length n)."""
    return state(pb, P_int, H0)["R"]


def comp_residual(pb, P_int, H0):
    """``(||min(P, R)||_inf, h sum P - pi/2)``."""
    R = residual(pb, P_int, H0)
    return np.max(np.abs(np.minimum(P_int, R))), pb.h * np.sum(P_int) - pb.load


def jacobian_exact(pb, P_int, H0):
    """Exact ``dR/dP`` ([n, n]) and ``dR/dH0`` ([n]) on the current limiter branch."""
    s = state(pb, P_int, H0)
    N, n, h = pb.N, pb.n, pb.h
    H, rho, eps, P = s["H"], s["rho"], s["eps"], s["P"]
    # columns 0..n-1 correspond to nodes 1..N-2, last column is H0
    dH = np.zeros((N, n + 1))
    dH[:, :n] = -pb.K[:, 1:-1]
    dH[:, n] = 1.0
    own = np.zeros((N, n + 1))
    own[1:-1, :n] = np.eye(n)
    drho_rel = s["drho"] / rho
    deta_rel = s["deta"] / s["eta"]
    du = rho[:, None] * dH + (s["drho"] * H)[:, None] * own
    deps = (3.0 * eps / H)[:, None] * dH + (eps * (drho_rel - deta_rel))[:, None] * own
    dF = du[:-1].copy()
    pa, pbb = s["psi_a"], s["psi_b"]
    i = np.arange(1, N - 1)
    dF[1:] += 0.5 * (pa[1:, None] * (du[i] - du[i - 1]) + pbb[1:, None] * (du[i + 1] - du[i]))
    dC = (dF[1:] - dF[:-1]) / h
    depsf = 0.5 * (deps[:-1] + deps[1:])
    dP = own  # dP_j / dz
    epsf = s["epsf"]
    dQ = (depsf[1:] * (P[2:] - P[1:-1])[:, None] + epsf[1:, None] * (dP[2:] - dP[1:-1])
          - depsf[:-1] * (P[1:-1] - P[:-2])[:, None] - epsf[:-1, None] * (dP[1:-1] - dP[:-2])) / h**2
    J = dC - dQ
    return J[:, :n], J[:, n]


def split_coefficient(pb):
    """``c`` of the hybrid splittings' upwind Couette part, or None for the frozen limiter.

    Sec. 3.3.2, Eqs. eqn57-eqn61: L_hs1 keeps the kappa-scheme's first-order part
    ``(2 - kappa)/2 (H_i - H_{i-1})`` in the line operator (Ls1 / Ls4), L_hs2 also
    the ``(1 - kappa)/4 (H_i - H_{i-1})`` that Eq. eqn58 splits off the upwind
    difference (Ls0 / Ls5); the rest of the convective term stays on the right-hand
    side.  Both use the weighted-change distribution where eps/h <= switch.
    Pinned by the stencils of Eq. eqn42 and the textbook kappa differences (the coefficient of
    the upwind difference in each, and of the farther upwind one) and, for the matrix it
    scales, by central differences of the residual where the first-order upwind difference is
    exact (tests/test_oracle_line.py).
    """
    if pb.splitting == "hs1":
        return (2.0 - pb.kappa) / 2.0
    if pb.splitting == "hs2":
        return (2.0 - pb.kappa) / 2.0 + (1.0 - pb.kappa) / 4.0
    return None


def jacobian_frozen(pb, P_int, H0):
    """``dR/dP`` with eps, rho and the limiter factor frozen (Sec. 3.3.3, Eqs. eqn62-eqn66).

    The Couette face value is linearised as
    ``F_{i+1/2} = u_i + phi_i (u_i - u_{i-1}) / 2`` with the frozen factor
    ``phi_i = psi_i / (u_i - u_{i-1})`` (0 where the backward difference is 0),
    ``u = rho H`` with ``rho`` frozen and ``dH/dP = -K``; the Poiseuille term
    keeps ``eps_{i+/-1/2}`` frozen.  Returns ``[n, n]``.
    """
    s = state(pb, P_int, H0)
    N, n, h = pb.N, pb.n, pb.h
    rho = s["rho"]
    a = s["a"]
    du = -rho[:, None] * pb.K[:, 1:-1]  # [N, n]
    c = split_coefficient(pb)
    if c is not None:
        dC = c * (du[1:-1] - du[:-2]) / h
    else:
        phi = np.where(a != 0.0, s["psi"] / np.where(a != 0.0, a, 1.0), 0.0)
        phi[0] = 0.0
        dF = du[:-1].copy()
        dF[1:] += 0.5 * phi[1:, None] * (du[1:-1] - du[:-2])
        dC = (dF[1:] - dF[:-1]) / h
    epsf = s["epsf"]
    dQ = np.zeros((n, n))
    for r in range(n):  # row r <-> node r+1
        dQ[r, r] = -(epsf[r + 1] + epsf[r]) / h**2
        if r + 1 < n:
            dQ[r, r + 1] = epsf[r + 1] / h**2
        if r - 1 >= 0:
            dQ[r, r - 1] = epsf[r] / h**2
    return dC - dQ


def switch_set(pb, P_int, H0):
    """Nodes of the weighted-change subregion: ``eps_i / h <= switch`` (Sec. 3.3.2, Eq. eqn60)."""
    s = state(pb, P_int, H0)
    return (s["eps"][1:-1] / pb.h) <= pb.switch_eps_h


def distribution_matrix(pb, P_int, H0):
    """Change distribution ``dP = D sigma`` of the weighted-change method (Sec. 3.3.4, Eq. eqn69).

    A change ``sigma_k`` at a node of the weighted-change subregion adds
    ``sigma_k`` to ``P_k`` and ``-w sigma_k`` to each interior neighbour
    (``w = dist_weight``, 1/4 in the paper's formula); elsewhere it adds
    ``sigma_k`` to ``P_k`` only.
    """
    n = pb.n
    Dm = np.eye(n)
    sw = switch_set(pb, P_int, H0)
    for k in np.nonzero(sw)[0]:
        if k - 1 >= 0:
            Dm[k - 1, k] = -pb.dist_weight
        if k + 1 < n:
            Dm[k + 1, k] = -pb.dist_weight
    return Dm


def active_rows(pb, P_int, H0):
    """Cavitated rows ``P_i <= 0 and R_i > 0``: identity rows of the Newton system."""
    R = residual(pb, P_int, H0)
    return (P_int <= 0.0) & (R > 0.0)


def jacobian_band(pb, P_int, H0, beta):
    """The banded approximate Jacobian of the hybrid limiter-based Newton method.

    ``band_beta(J_frozen D)`` (Sec. 3.3.3-3.3.4: the kernel coupling truncated
    to the band, Eqs. eqn67-eqn68 for beta = 2), with cavitated rows replaced
    by identity rows.  Returns ``(band [n, 2 beta + 1], active [n] bool)`` in
    the row-major band layout ``band[i, j] = A[i, i - beta + j]``.
    """
    J = jacobian_frozen(pb, P_int, H0) @ distribution_matrix(pb, P_int, H0)
    act = active_rows(pb, P_int, H0)
    n = pb.n
    band = np.zeros((n, 2 * beta + 1))
    for i in range(n):
        if act[i]:
            band[i, beta] = 1.0
            continue
        for j in range(2 * beta + 1):
            c = i - beta + j
            if 0 <= c < n:
                band[i, j] = J[i, c]
    return band, act


def rounding_floor(pb, P_int, H0):
    """``1e3`` roundoff units times the largest term entering any ``R_i``."""
    s = state(pb, P_int, H0)
    P, F, epsf, h = s["P"], s["F"], s["epsf"], pb.h
    conv = (np.abs(F[1:]) + np.abs(F[:-1])) / h
    pois = (np.abs(epsf[1:] * (P[2:] - P[1:-1])) + np.abs(epsf[:-1] * (P[1:-1] - P[:-2]))) / h**2
    return 1e3 * np.finfo(np.float64).eps * float(np.max(conv + pois))


def solve(pb, P_init=None, H0_init=None, h_init=0.05, tol=1e-12, max_iter=200, verbose=False):
    """Dense semismooth Newton solve of the discrete complementarity problem.

    Unknowns ``z = (P_1..P_{N-2}, H0)``; equations
    ``Phi_i = min(P_i, R_i / d_i)`` (``d_i = |dR_i/dP_i|`` of the current
    iterate: a positive row scaling that leaves the solution set unchanged)
    and ``Phi_n = h sum P - pi/2``.  Each step solves ``J_Phi dz = -Phi`` by
    dense LU, where row i of ``J_Phi`` is ``e_i`` when ``P_i <= R_i / d_i``
    and the exact scaled ``(dR_i/dP, dR_i/dH0)`` otherwise, then backtracks on
    ``||Phi||_2`` and keeps ``P >= 0``.

    Stops when ``||min(P, R)||_inf <= tol`` and ``|h sum P - pi/2| <= tol``, or
    when the residual has stopped falling for five steps and lies below the
    rounding floor of R (``1e3`` units of roundoff times the largest term of
    the residual formula: the Poiseuille terms grow like ``eps / h^2``).
    Returns ``(P_int, H0, info)`` with ``info["res"] = ||min(P, R)||_inf``.
    """
    P = pb.hertz() if P_init is None else np.array(P_init, dtype=np.float64)
    H0 = pb.h0_for_min_film(P, h_init) if H0_init is None else float(H0_init)
    n = pb.n
    hist = []
    best = np.inf
    stall = 0
    for it in range(max_iter):
        R = residual(pb, P, H0)
        r_c = np.max(np.abs(np.minimum(P, R)))
        r_g = abs(pb.h * np.sum(P) - pb.load)
        hist.append((r_c, r_g))
        if verbose:
            print(f"it {it:3d}  |min(P,R)| {r_c:.3e}  |g| {r_g:.3e}  H0 {H0:.8f}")
        if r_c <= tol and r_g <= tol:
            return P, H0, dict(iters=it, hist=hist, converged=True, res=r_c, force=r_g)
        if r_c < 0.5 * best:
            best = r_c
            stall = 0
        else:
            stall += 1
        J, JH = jacobian_exact(pb, P, H0)
        d = np.abs(np.diag(J))
        d = np.where(d > 0.0, d, 1.0)

        def phi(P, H0):
            R = residual(pb, P, H0)
            return np.concatenate([np.minimum(P, R / d), [pb.h * np.sum(P) - pb.load]])

        F = phi(P, H0)
        use_p = P <= R / d
        Jp = np.zeros((n + 1, n + 1))
        Jp[:n, :n] = np.where(use_p[:, None], np.eye(n), J / d[:, None])
        Jp[:n, n] = np.where(use_p, 0.0, JH / d)
        Jp[n, :n] = pb.h
        dz = np.linalg.solve(Jp, -F)
        floor = rounding_floor(pb, P, H0)
        if stall >= 5 and r_c <= max(tol, floor) and r_g <= tol:
            return P, H0, dict(iters=it, hist=hist, converged=True, res=r_c, force=r_g, floor=floor)
        f0 = np.linalg.norm(F)
        t = 1.0
        for _ in range(40):
            Pn = np.maximum(P + t * dz[:n], 0.0)
            Hn = H0 + t * dz[n]
            Fn = phi(Pn, Hn)
            if np.all(np.isfinite(Fn)) and np.linalg.norm(Fn) <= (1.0 - 1e-4 * t) * f0:
                break
            t *= 0.5
        if not np.all(np.isfinite(Fn)):
            break
        P, H0 = Pn, Hn
    R = residual(pb, P, H0)
    r_c = np.max(np.abs(np.minimum(P, R)))
    return P, H0, dict(iters=max_iter, hist=hist, converged=False, res=r_c,
                       force=abs(pb.h * np.sum(P) - pb.load))


def solve_paper(pb, beta=2, omega=1.0, c=0.05, tol=1e-8, max_iter=4000, h_init=0.05):
    """The paper's hybrid limiter-based Newton iteration for line contact, step by step.

    From the Hertzian start with ``min H = h_init`` (Sec. 4), each iteration
    (Sec. 3.3.3-3.3.4):
    1. the residual R at the current iterate (Eqs. eqn62-eqn65);
    2. the banded approximate Jacobian ``band_beta(J_frozen D)`` with eps, rho
       and the limiter factor frozen and the change distributed by D in the
       weighted-change subregion (Eqs. eqn66-eqn69; ``jacobian_band``), the
       cavitated rows as identity rows (reading of Sec. 2.2.2);
    3. the band system for the change sigma with right-hand side -R (0 on the
       cavitated rows), solved here by dense LU in place of PAQIF;
    4. the projected distributed update ``P <- max(0, P + omega D sigma)``;
    5. the H0 relaxation ``H0 <- H0 - c (pi/2 - h sum P)`` (Eq. eqn75 with the
       line-contact load).
    Stops when ``||min(P, R)||_inf <= tol`` and ``|h sum P - pi/2| <= tol``
    (checked before each update), or at ``max_iter`` updates, or when the
    iterate stops being finite.  Returns ``(P, H0, info)`` with ``info["hist"]``
    the residual before every update.
    """
    P = pb.hertz()
    H0 = pb.h0_for_min_film(P, h_init)
    hist = []
    with np.errstate(over="ignore", invalid="ignore"):
        for it in range(max_iter):
            r_c, g = comp_residual(pb, P, H0)
            hist.append(r_c)
            if not (np.isfinite(r_c) and np.isfinite(g)):
                return P, H0, dict(iters=it, converged=False, diverged=True, hist=hist)
            if r_c <= tol and abs(g) <= tol:
                return P, H0, dict(iters=it, converged=True, diverged=False, hist=hist)
            R = residual(pb, P, H0)
            band, act = jacobian_band(pb, P, H0, beta)
            A = np.zeros((pb.n, pb.n))
            for i in range(pb.n):
                for j in range(2 * beta + 1):
                    col = i - beta + j
                    if 0 <= col < pb.n:
                        A[i, col] = band[i, j]
            sigma = np.linalg.solve(A, np.where(act, 0.0, -R))
            P = np.maximum(P + omega * (distribution_matrix(pb, P, H0) @ sigma), 0.0)
            H0 = H0 - c * (pb.load - pb.h * np.sum(P))
    return P, H0, dict(iters=max_iter, converged=False, diverged=False, hist=hist)


def solve_continuation(pb_factory, M_target, L_target, steps, **kw):
    """Solve at ``M_target, L_target`` by a sequence of loads (plain continuation).

    ``pb_factory(M, L)`` builds a problem; the load ``M`` is raised
    geometrically from ``M_target / 2^steps`` (and ``L`` with it) and each
    solution starts the next solve.
    """
    P = H0 = None
    for k in range(steps, -1, -1):
        f = 2.0 ** (-k * 0.5)
        pb = pb_factory(M_target * f, L_target)
        P, H0, info = solve(pb, P_init=P, H0_init=H0, **kw)
        if not info["converged"]:
            raise RuntimeError(f"continuation step M={M_target * f} did not converge")
    return pb, P, H0, info


# ------------------------------------------------------------ grid sequence
def grid_sequence(N, n_min=65, levels=-1):
    """Grids ``N_0 < N_1 < ... < N_L = N`` with ``N_{l+1} - 1 = 2 (N_l - 1)``.

    Coarsening halves the number of intervals while it stays even and the
    coarse grid keeps at least ``n_min`` nodes; ``levels`` (``>= 0``) caps the
    number of coarse grids, ``-1`` takes as many as the rule allows.  The
    paper computes its line- and point-contact solutions on such a sequence
    of grids (Sec. 4, coarse ``16+1`` up to fine ``1024+1`` nodes per axis).
    """
    seq = [int(N)]
    while (seq[-1] - 1) % 2 == 0 and (seq[-1] - 1) // 2 + 1 >= n_min and (levels < 0 or len(seq) <= levels):
        seq.append((seq[-1] - 1) // 2 + 1)
    return seq[::-1]


def prolong(Pc):
    """Nodal vector on a grid of ``Nc`` nodes -> ``2 Nc - 1`` nodes, linear interpolation.

    Coarse node ``i`` is fine node ``2 i``; a new fine node takes the mean of
    its two coarse neighbours.
    """
    Pc = np.asarray(Pc, dtype=np.float64)
    Pf = np.empty(2 * len(Pc) - 1)
    Pf[0::2] = Pc
    Pf[1::2] = 0.5 * (Pc[:-1] + Pc[1:])
    return Pf


def inject(vf, Nc):
    """Fine nodal vector -> its values at the ``Nc`` nodes of a coarser grid of the sequence."""
    vf = np.asarray(vf, dtype=np.float64)
    stride = (len(vf) - 1) // (Nc - 1)
    return vf[::stride].copy()


def solve_nested(pb_factory, N, n_min=65, levels=-1, coarse_tol=1e-6, tol=1e-12, **kw):
    """Nested iteration: solve on each grid of ``grid_sequence(N)``, coarse to fine.

    ``pb_factory(N_l)`` builds the problem on ``N_l`` nodes (with the
    roughness injected from the finest grid).  The coarsest solve starts from
    the Hertzian pressure; each finer one from the prolonged pressure of the
    grid below and its ``H0``.  Coarse grids are solved to ``max(tol,
    coarse_tol)``, the finest to ``tol``.  Returns ``(pb, P_int, H0, info)``
    of the finest grid, ``info["levels"]`` the ``(N_l, iterations,
    converged)`` of every grid.
    """
    seq = grid_sequence(N, n_min, levels)
    P = H0 = None
    out = []
    for l, Nl in enumerate(seq):
        pb = pb_factory(Nl)
        P0 = None if P is None else prolong(pb_prev.full(P))[1:-1]
        t = tol if l == len(seq) - 1 else max(tol, coarse_tol)
        P, H0, info = solve(pb, P_init=P0, H0_init=H0, tol=t, **kw)
        out.append((Nl, info["iters"], info["converged"]))
        pb_prev = pb
    info["levels"] = out
    return pb, P, H0, info
