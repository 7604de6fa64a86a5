"""Point-contact EHL: discrete residual, exact Jacobian and a dense solve (test infrastructure).

Discrete problem (Sec. 3.3 Example 6 in two dimensions, Sec. 3.3.1 Case 2,
Sec. 3.3.3): grid ``X_i = xa + i h``, ``Y_j = ya + j h`` (one spacing in both
directions), ``P = 0`` on the boundary nodes; unknowns ``P`` at the interior
nodes and ``H0``.  Arrays are ``[nx, ny]`` (x index first).

* film ``H = H0 + X^2/2 + Y^2/2 + D + rough`` with the direct-sum deformation
  ``D_ij = (2/pi^2) sum_kl G(i-k, j-l) P_kl`` (``kernels_ref.deform_point``);
* lubricant as in line contact, with the point-contact Moes conversion
  ``lambda = (128 pi^3/(3 M^4))^{1/3}``, ``alpha_bar = (L/pi)(3M/2)^{1/3}``;
* residual per unit area: the limited x-flux of ``u = rho H`` (the line
  contact's face value along every x-line, first order at the inflow face)
  and the 5-point Poiseuille term with arithmetic half-node ``eps``:
  ``R_ij = (F_{i+1/2,j} - F_{i-1/2,j})/h
          - [eps_{i+1/2,j}(P_{i+1,j}-P_ij) - eps_{i-1/2,j}(P_ij-P_{i-1,j})]/h^2
          - [eps_{i,j+1/2}(P_{i,j+1}-P_ij) - eps_{i,j-1/2}(P_ij-P_{i,j-1})]/h^2``;
* complementarity ``P >= 0, R >= 0, P R = 0`` and force balance
  ``h^2 sum P = 2 pi / 3`` (the Hertzian load, reading of the force
  statement: the H0 update of Sec. 3.3.4 uses 2 pi / 3).

The dense Jacobian and Newton solve are meant for grids up to 65 x 65.
"""
import numpy as np

from . import kernels_ref, line_ref, material_ref


class PointProblem:
    """Grid, kernel and lubricant constants of one point-contact instance."""

    def __init__(self, nx, ny, M, L, xa=-4.5, xb=1.5, ya=-3.0, alpha=1.7e-8, compressible=True,
                 elastic=True, limiter="minmod", rough=None, kappa=0.0):
        self.nx, self.ny = int(nx), int(ny)
        self.M, self.L = float(M), float(L)
        self.h = (xb - xa) / (self.nx - 1)
        self.xa, self.ya = float(xa), float(ya)
        self.X = self.xa + self.h * np.arange(self.nx)
        self.Y = self.ya + self.h * np.arange(self.ny)
        self.alpha = float(alpha)
        self.lam, self.abar = material_ref.moes_point(self.M, self.L)
        self.compressible = bool(compressible)
        self.elastic = bool(elastic)
        if limiter not in ("minmod", "vanleer", "kappa"):
            raise ValueError(limiter)
        self.limiter = limiter
        self.kappa = float(kappa)
        self.rough = np.zeros((self.nx, self.ny)) if rough is None else np.asarray(rough, dtype=np.float64)
        self.table = kernels_ref.g_point_table(self.nx, self.ny, self.h)
        self.load = 2.0 * np.pi / 3.0
        self.shape_int = (self.nx - 2, self.ny - 2)
        self.n = (self.nx - 2) * (self.ny - 2)

    def full(self, P_int):
        """Interior values (flattened ``[nx-2, ny-2]``) -> nodal ``[nx, ny]`` with zero boundary."""
        P = np.zeros((self.nx, self.ny))
        P[1:-1, 1:-1] = np.asarray(P_int, dtype=np.float64).reshape(self.shape_int)
        return P

    def deform(self, P):
        return kernels_ref.deform_point(P, self.h, self.table) if self.elastic else np.zeros_like(P)

    def film(self, P_int, H0):
        X, Y = np.meshgrid(self.X, self.Y, indexing="ij")
        return H0 + 0.5 * X**2 + 0.5 * Y**2 + self.deform(self.full(P_int)) + self.rough

    def hertz(self):
        """Hertzian start ``sqrt(max(0, 1 - X^2 - Y^2))``, interior values flattened."""
        X, Y = np.meshgrid(self.X, self.Y, indexing="ij")
        return np.sqrt(np.maximum(0.0, 1.0 - X**2 - Y**2))[1:-1, 1:-1].ravel()

    def h0_for_min_film(self, P_int, h_init):
        return h_init - np.min(self.film(P_int, 0.0))

    def deform_matrix(self):
        """Dense ``dD/dP_int``: ``[nx*ny, n]`` (rows nodal in C order, columns interior in C order)."""
        ii, jj = np.meshgrid(np.arange(self.nx), np.arange(self.ny), indexing="ij")
        ki, kj = np.meshgrid(np.arange(1, self.nx - 1), np.arange(1, self.ny - 1), indexing="ij")
        a = np.abs(ii.ravel()[:, None] - ki.ravel()[None, :])
        b = np.abs(jj.ravel()[:, None] - kj.ravel()[None, :])
        return self.table[a, b] if self.elastic else np.zeros((self.nx * self.ny, self.n))


def state(pb, P_int, H0):
    P = pb.full(P_int)
    H = pb.film(P_int, H0)
    rho, drho, eta, deta = material_ref.material(P, pb.abar, pb.alpha, pb.compressible)
    eps = rho * H**3 / (eta * pb.lam)
    u = rho * H
    nx, h = pb.nx, pb.h
    # x-faces i+1/2, i = 0..nx-2, on every y-line
    a = np.zeros((nx - 1, pb.ny))
    b = np.zeros((nx - 1, pb.ny))
    a[1:] = u[1:-1] - u[:-2]
    b[1:] = u[2:] - u[1:-1]
    psi, pa, pbb = line_ref.limiter(a, b, pb.limiter, pb.kappa)
    psi[0] = pa[0] = pbb[0] = 0.0
    F = u[:-1] + 0.5 * psi
    ex = 0.5 * (eps[:-1] + eps[1:])        # [nx-1, ny]
    ey = 0.5 * (eps[:, :-1] + eps[:, 1:])  # [nx, ny-1]
    C = (F[1:, 1:-1] - F[:-1, 1:-1]) / h
    Qx = (ex[1:, 1:-1] * (P[2:, 1:-1] - P[1:-1, 1:-1]) - ex[:-1, 1:-1] * (P[1:-1, 1:-1] - P[:-2, 1:-1])) / h**2
    Qy = (ey[1:-1, 1:] * (P[1:-1, 2:] - P[1:-1, 1:-1]) - ey[1:-1, :-1] * (P[1:-1, 1:-1] - P[1:-1, :-2])) / h**2
    R = C - Qx - Qy
    return dict(P=P, H=H, rho=rho, drho=drho, eta=eta, deta=deta, eps=eps, u=u, psi=psi, psi_a=pa, psi_b=pbb,
                F=F, ex=ex, ey=ey, R=R)


def residual(pb, P_int, H0):
    """Interior residual flattened ``[nx-2, ny-2]``."""
    return state(pb, P_int, H0)["R"].ravel()


def comp_residual(pb, P_int, H0):
    R = residual(pb, P_int, H0)
    return np.max(np.abs(np.minimum(P_int, R))), pb.h**2 * np.sum(P_int) - pb.load


def _tangent(pb, s, dH, dP, dlnpH=None, dlnlam=None):
    """``dR`` (interior, flattened) for the perturbations ``dH``, ``dP`` ([nx, ny, c]) of H and P,
    and optionally of ``ln p_H`` and ``ln lambda`` (``[c]``; rho and eta depend on ``P p_H``, so
    ``d/d ln p_H = P d/dP``)."""
    h = pb.h
    H, rho, eps, P = s["H"], s["rho"], s["eps"], s["P"]
    drho = s["drho"][..., None] * dP
    dlneta = (s["deta"] / s["eta"])[..., None] * dP
    if dlnpH is not None:
        drho = drho + (s["drho"] * P)[..., None] * dlnpH
        dlneta = dlneta + (s["deta"] / s["eta"] * P)[..., None] * dlnpH
    deps = eps[..., None] * (drho / rho[..., None] + 3.0 * dH / H[..., None] - dlneta)
    if dlnlam is not None:
        deps = deps - eps[..., None] * dlnlam
    du = drho * H[..., None] + rho[..., None] * dH
    dF = du[:-1].copy()
    pa, pbb = s["psi_a"], s["psi_b"]
    dF[1:] += 0.5 * (pa[1:, :, None] * (du[1:-1] - du[:-2]) + pbb[1:, :, None] * (du[2:] - du[1:-1]))
    dC = (dF[1:, 1:-1] - dF[:-1, 1:-1]) / h
    dex = 0.5 * (deps[:-1] + deps[1:])
    dey = 0.5 * (deps[:, :-1] + deps[:, 1:])
    ex, ey = s["ex"][..., None], s["ey"][..., None]
    dQx = (dex[1:, 1:-1] * (P[2:, 1:-1] - P[1:-1, 1:-1])[..., None] + ex[1:, 1:-1] * (dP[2:, 1:-1] - dP[1:-1, 1:-1])
           - dex[:-1, 1:-1] * (P[1:-1, 1:-1] - P[:-2, 1:-1])[..., None]
           - ex[:-1, 1:-1] * (dP[1:-1, 1:-1] - dP[:-2, 1:-1])) / h**2
    dQy = (dey[1:-1, 1:] * (P[1:-1, 2:] - P[1:-1, 1:-1])[..., None] + ey[1:-1, 1:] * (dP[1:-1, 2:] - dP[1:-1, 1:-1])
           - dey[1:-1, :-1] * (P[1:-1, 1:-1] - P[1:-1, :-2])[..., None]
           - ey[1:-1, :-1] * (dP[1:-1, 1:-1] - dP[1:-1, :-2])) / h**2
    return (dC - dQx - dQy).reshape(pb.n, -1)


def jacobian_exact(pb, P_int, H0, Kd=None, block=512):
    """Exact ``dR/dP_int`` ([n, n]) and ``dR/dH0`` ([n]) on the current limiter branch.

    Forward mode, ``block`` columns at a time: the film carries the deformation
    column ``dD/dP_kl`` (and 1 for H0), ``rho`` and ``eta`` the own-node
    derivative.
    """
    s = state(pb, P_int, H0)
    nx, ny, n = pb.nx, pb.ny, pb.n
    if Kd is None:
        Kd = pb.deform_matrix()
    J = np.zeros((n, n))
    ki, kj = np.meshgrid(np.arange(1, nx - 1), np.arange(1, ny - 1), indexing="ij")
    ki, kj = ki.ravel(), kj.ravel()
    for c0 in range(0, n, block):
        c1 = min(n, c0 + block)
        dH = Kd[:, c0:c1].reshape(nx, ny, c1 - c0)
        dP = np.zeros((nx, ny, c1 - c0))
        dP[ki[c0:c1], kj[c0:c1], np.arange(c1 - c0)] = 1.0
        J[:, c0:c1] = _tangent(pb, s, dH, dP)
    JH = _tangent(pb, s, np.ones((nx, ny, 1)), np.zeros((nx, ny, 1)))[:, 0]
    return J, JH


def xline_band_exact(pb, P_int, H0, beta):
    """The x-line bands of the exact Jacobian: ``[ny-2, nx-2, 2 beta + 1]``.

    Entry ``[j-1, i-1, beta + k - i]`` is ``dR_ij / dP_kj`` (Sec. 3.3.3: the
    x-line systems of the point-contact Newton matrix, one per grid row j,
    here from the exact Jacobian).  Without the dense Jacobian: the residual
    row ``(i, j)`` reads the film at x-nodes ``i-2 .. i+1`` (the limited faces)
    and at ``(i, j +/- 1)`` (eps of the y-faces), so the band entries of column
    ``(k, j)`` need the deformation column of a unit pressure at ``(k, j)``
    only on the window ``x in [k - beta - 2, k + beta + 1]``, ``y in
    [j - 1, j + 1]``.  Columns whose windows and stencils are disjoint
    (x-indices ``2 beta + 4`` apart, y-indices 3 apart) share one forward-mode
    tangent, each filled with the kernel table on its own window.
    """
    s = state(pb, P_int, H0)
    nx, ny = pb.nx, pb.ny
    px, py = 2 * beta + 4, 3
    band = np.zeros((ny - 2, nx - 2, 2 * beta + 1))
    for cx in range(px):
        ks = np.arange(1 + cx, nx - 1, px)
        for cy in range(py):
            ls = np.arange(1 + cy, ny - 1, py)
            if len(ks) == 0 or len(ls) == 0:
                continue
            dH = np.zeros((nx, ny, 1))
            dP = np.zeros((nx, ny, 1))
            K, L = np.meshgrid(ks, ls, indexing="ij")
            K, L = K.ravel(), L.ravel()
            dP[K, L, 0] = 1.0
            if pb.elastic:
                for ox in range(-beta - 2, beta + 2):
                    for oy in (-1, 0, 1):
                        mx, my = K + ox, L + oy
                        ok = (mx >= 0) & (mx < nx) & (my >= 0) & (my < ny)
                        dH[mx[ok], my[ok], 0] = pb.table[np.abs(ox), np.abs(oy)]
            t = _tangent(pb, s, dH, dP)[:, 0].reshape(nx - 2, ny - 2)  # row (i, j) -> [i-1, j-1]
            for d in range(-beta, beta + 1):
                rows = K + d  # row i = k + d, entry beta + k - i = beta - d
                ok = (rows >= 1) & (rows <= nx - 2)
                band[L[ok] - 1, rows[ok] - 1, beta - d] = t[rows[ok] - 1, L[ok] - 1]
    return band


def yline_band_exact(pb, P_int, H0, beta):
    """The y-line bands of the exact Jacobian: ``[nx-2, ny-2, 2 beta + 1]``.

    Entry ``[i-1, j-1, beta + l - j]`` is ``dR_ij / dP_il`` (Sec. 3.3.2-3.3.4: the
    y-line systems of the alternating line splitting, one per grid column i; the
    paper writes out only the x-line equations, the y-lines follow by symmetry).
    As in ``xline_band_exact``: the rows ``(i, l + d)`` of column ``(i, l)`` read
    the film at ``x in [i - 2, i + 1]``, ``y in [l - beta - 1, l + beta + 1]``, so
    columns 4 apart in x and ``2 beta + 3`` apart in y share one tangent.
    """
    s = state(pb, P_int, H0)
    nx, ny = pb.nx, pb.ny
    px, py = 4, 2 * beta + 3
    band = np.zeros((nx - 2, ny - 2, 2 * beta + 1))
    for cx in range(px):
        ks = np.arange(1 + cx, nx - 1, px)
        for cy in range(py):
            ls = np.arange(1 + cy, ny - 1, py)
            if len(ks) == 0 or len(ls) == 0:
                continue
            dH = np.zeros((nx, ny, 1))
            dP = np.zeros((nx, ny, 1))
            K, L = np.meshgrid(ks, ls, indexing="ij")
            K, L = K.ravel(), L.ravel()
            dP[K, L, 0] = 1.0
            if pb.elastic:
                for ox in range(-2, 2):
                    for oy in range(-beta - 1, beta + 2):
                        mx, my = K + ox, L + oy
                        ok = (mx >= 0) & (mx < nx) & (my >= 0) & (my < ny)
                        dH[mx[ok], my[ok], 0] = pb.table[np.abs(ox), np.abs(oy)]
            t = _tangent(pb, s, dH, dP)[:, 0].reshape(nx - 2, ny - 2)
            for d in range(-beta, beta + 1):
                rows = L + d  # row j = l + d, entry beta + l - j = beta - d
                ok = (rows >= 1) & (rows <= ny - 2)
                band[K[ok] - 1, rows[ok] - 1, beta - d] = t[K[ok] - 1, rows[ok] - 1]
    return band


def rounding_floor(pb, P_int, H0):
    """``1e3`` roundoff units times the largest term entering any ``R_ij``."""
    s = state(pb, P_int, H0)
    P, F, ex, ey, h = s["P"], s["F"], s["ex"], s["ey"], pb.h
    conv = (np.abs(F[1:, 1:-1]) + np.abs(F[:-1, 1:-1])) / h
    pois = (np.abs(ex[1:, 1:-1] * (P[2:, 1:-1] - P[1:-1, 1:-1])) + np.abs(ex[:-1, 1:-1] * (P[1:-1, 1:-1] - P[:-2, 1:-1]))
            + np.abs(ey[1:-1, 1:] * (P[1:-1, 2:] - P[1:-1, 1:-1]))
            + np.abs(ey[1:-1, :-1] * (P[1:-1, 1:-1] - P[1:-1, :-2]))) / h**2
    return 1e3 * np.finfo(np.float64).eps * float(np.max(conv + pois))


def solve(pb, P_init=None, H0_init=None, h_init=0.05, tol=1e-12, max_iter=100):
    """Dense semismooth Newton on ``Phi = (min(P, R/d), h^2 sum P - 2 pi/3)``.

    The same iteration as ``line_ref.solve`` on the two-dimensional problem:
    Jacobi row scaling ``d = |dR_ii/dP_ii|``, dense LU per step, backtracking
    on ``||Phi||_2`` with ``P >= 0``, stop at ``tol`` or at the rounding floor
    after five steps without the residual halving.
    """
    n = pb.n
    P = pb.hertz() if P_init is None else np.array(P_init, dtype=np.float64)
    H0 = pb.h0_for_min_film(P, h_init) if H0_init is None else float(H0_init)
    Kd = pb.deform_matrix()
    best, stall = np.inf, 0
    for it in range(max_iter):
        R = residual(pb, P, H0)
        r_c = np.max(np.abs(np.minimum(P, R)))
        r_g = abs(pb.h**2 * np.sum(P) - pb.load)
        if r_c <= tol and r_g <= tol:
            return P, H0, dict(iters=it, converged=True, res=r_c, force=r_g)
        if r_c < 0.5 * best:
            best, stall = r_c, 0
        else:
            stall += 1
        if stall >= 5 and r_c <= max(tol, rounding_floor(pb, P, H0)) and r_g <= tol:
            return P, H0, dict(iters=it, converged=True, res=r_c, force=r_g)
        J, JH = jacobian_exact(pb, P, H0, Kd)
        d = np.abs(np.diag(J))
        d = np.where(d > 0.0, d, 1.0)
        use_p = P <= R / d
        F = np.concatenate([np.where(use_p, P, R / d), [pb.h**2 * np.sum(P) - pb.load]])
        Jp = np.zeros((n + 1, n + 1))
        Jp[:n, :n] = np.where(use_p[:, None], np.eye(n), J / d[:, None])
        Jp[:n, n] = np.where(use_p, 0.0, JH / d)
        Jp[n, :n] = pb.h**2
        dz = np.linalg.solve(Jp, -F)
        f0 = np.linalg.norm(F)
        t = 1.0
        for _ in range(40):
            Pn = np.maximum(P + t * dz[:n], 0.0)
            Hn = H0 + t * dz[n]
            Rn = residual(pb, Pn, Hn)
            Fn = np.concatenate([np.minimum(Pn, Rn / d), [pb.h**2 * np.sum(Pn) - pb.load]])
            if np.all(np.isfinite(Fn)) and np.linalg.norm(Fn) <= (1.0 - 1e-4 * t) * f0:
                break
            t *= 0.5
        P, H0 = Pn, Hn
    R = residual(pb, P, H0)
    return P, H0, dict(iters=max_iter, converged=False, res=np.max(np.abs(np.minimum(P, R))),
                       force=abs(pb.h**2 * np.sum(P) - pb.load))


def prolong(Pc):
    """Bilinear interpolation of a nodal ``[nc_x, nc_y]`` array to ``[2 nc_x - 1, 2 nc_y - 1]``."""
    Pc = np.asarray(Pc, dtype=np.float64)
    Px = np.empty((2 * Pc.shape[0] - 1, Pc.shape[1]))
    Px[0::2] = Pc
    Px[1::2] = 0.5 * (Pc[:-1] + Pc[1:])
    Pf = np.empty((Px.shape[0], 2 * Pc.shape[1] - 1))
    Pf[:, 0::2] = Px
    Pf[:, 1::2] = 0.5 * (Px[:, :-1] + Px[:, 1:])
    return Pf


def solve_nested(pb_factory, nx, ny, n_min=17, tol=1e-12, coarse_tol=1e-6, **kw):
    """Nested iteration over grids with halved intervals in both directions (at least
    ``n_min`` nodes per direction), each grid started from the prolonged solution below."""
    seq = [(nx, ny)]
    while all((m - 1) % 2 == 0 and (m - 1) // 2 + 1 >= n_min for m in seq[-1]):
        seq.append(tuple((m - 1) // 2 + 1 for m in seq[-1]))
    seq = seq[::-1]
    P = H0 = None
    out = []
    for l, (gx, gy) in enumerate(seq):
        pb = pb_factory(gx, gy)
        P0 = None if P is None else prolong(prev.full(P))[1:-1, 1:-1].ravel()
        t = tol if l == len(seq) - 1 else max(tol, coarse_tol)
        P, H0, info = solve(pb, P_init=P0, H0_init=H0, tol=t, **kw)
        out.append(((gx, gy), info["iters"], info["converged"]))
        prev = pb
    info["levels"] = out
    return pb, P, H0, info


# ------------------------------------------------------------------- adjoint
def moes_point_log_derivatives(M, L):
    """``d ln(lambda)/d(M, L)`` and ``d ln(p_H)/d(M, L)`` for the point-contact conversion."""
    return np.array([-4.0 / (3.0 * M), 0.0]), np.array([1.0 / (3.0 * M), 1.0 / L])


def adjoint(pb, P_int, H0, gP, gH, gH0):
    """Gradient of ``J(P, H, H0)`` w.r.t. the roughness (nodal ``[nx, ny]``), ``M`` and ``L``.

    As the line-contact adjoint (``adjoint_ref.adjoint``) on the point problem:
    equation rows ``P_i > R_i / |dR_ii/dP_ii|``, bordered with the force row
    ``h^2``, dense LU of the transpose.  ``gP``, ``gH`` are nodal ``[nx, ny]``.
    Meant for small grids (the roughness tangent is dense).
    """
    nx, ny, n, NN = pb.nx, pb.ny, pb.n, pb.nx * pb.ny
    Kd = pb.deform_matrix()
    J, JH = jacobian_exact(pb, P_int, H0, Kd)
    R = residual(pb, P_int, H0)
    d = np.abs(np.diag(J))
    d = np.where(d > 0.0, d, 1.0)
    A = np.nonzero(P_int > R / d)[0]
    na = len(A)
    s = state(pb, P_int, H0)
    Trough = _tangent(pb, s, np.eye(NN).reshape(nx, ny, NN), np.zeros((nx, ny, NN)))   # [n, NN]
    dlam, dpH = moes_point_log_derivatives(pb.M, pb.L)
    TML = _tangent(pb, s, np.zeros((nx, ny, 2)), np.zeros((nx, ny, 2)), dlnpH=dpH, dlnlam=dlam)  # [n, 2]
    Fx = np.zeros((na + 1, na + 1))
    Fx[:na, :na] = J[np.ix_(A, A)]
    Fx[:na, na] = JH[A]
    Fx[na, :na] = pb.h**2
    gP = np.asarray(gP, dtype=np.float64)
    gH = np.asarray(gH, dtype=np.float64)
    gPt = gP[1:-1, 1:-1].ravel() + Kd.T @ gH.ravel()
    gH0t = float(gH0) + float(np.sum(gH))
    lam = np.linalg.solve(Fx.T, np.concatenate([gPt[A], [gH0t]]))
    grad_rough = gH.ravel() - lam[:na] @ Trough[A]
    gML = -(lam[:na] @ TML[A])
    return dict(rough=grad_rough.reshape(nx, ny), M=float(gML[0]), L=float(gML[1]), rows=A)
