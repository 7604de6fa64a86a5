"""GPU parity of the line-contact entry points (ehl_residual, ehl_jacobian_band,
ehl_solve) against the float64 oracle, through the C ABI.

Tolerances
* residual: |R_gpu - R_ref| <= 1e-12 x the row's term magnitude
  (|F_{i+1/2}| + |F_{i-1/2}|)/h + (|eps_{i+1/2} dP| + |eps_{i-1/2} dP|)/h^2 --
  both sides evaluate the same float64 formula, the deformation sum runs in
  double-float (about 1e-15 relative), so only rounding of the terms differs;
* film H: 1e-13 relative;
* band Jacobians: 1e-11 x the row's largest entry;
* converged P, H: 1e-8 relative (the target stated for converged solutions).
"""
import numpy as np
import pytest
import torch

from oracle import line_ref as lr
from paper_2008_03276_gb300 import ops

pytestmark = pytest.mark.gpu


def make(N=129, M=20.0, L=10.0, limiter=0, beta=2, method=0, compressible=1, elastic=1, n_inst=1, per=None, **kw):
    p = ops.default_params(1, nx=N, M=M, L=L, limiter=limiter, halfband=beta, method=method,
                           compressible=compressible, elastic=elastic, **kw)
    per_inst = None
    if per is not None:
        per_inst = [ops.default_params(1, nx=N, limiter=limiter, halfband=beta, method=method,
                                       compressible=compressible, elastic=elastic, **{**kw, **d}) for d in per]
    return ops.Context(p, n_inst=n_inst, per_inst=per_inst), p


def oracle_problem(N=129, M=20.0, L=10.0, limiter=0, compressible=1, elastic=1, rough=None, dist_weight=0.5):
    return lr.LineProblem(N, M, L, limiter=("minmod", "vanleer")[limiter], compressible=bool(compressible),
                          elastic=bool(elastic), rough=rough, dist_weight=dist_weight)


def row_scale(pb, P, H0):
    s = lr.state(pb, P, H0)
    F, ef, Pn, h = s["F"], s["epsf"], s["P"], pb.h
    return (np.abs(F[1:]) + np.abs(F[:-1])) / h + (np.abs(ef[1:] * (Pn[2:] - Pn[1:-1])) +
                                                   np.abs(ef[:-1] * (Pn[1:-1] - Pn[:-2]))) / h**2


def limiter_conditioning(pb, P, H0, rel=1e-14):
    """Per interior row: rel x |u| / min(|a|, |b|) over the two faces of the row.

    The limiter derivatives and the frozen factor psi/a depend on the ratio of
    the differences a = u_j - u_{j-1}, b = u_{j+1} - u_j.  Where rho H is
    nearly flat (the Hertzian zone of a converged solution) a and b are
    differences of nearly equal numbers, and a relative change `rel` in u (two
    summation orders of the deformation) moves them by rel |u| / |a|.
    """
    s = lr.state(pb, P, H0)
    u, a, b = s["u"], s["a"], s["b"]
    with np.errstate(divide="ignore", invalid="ignore"):
        c = rel * np.abs(u[:-1]) / np.minimum(np.abs(a), np.abs(b))
    c = np.where(np.isfinite(c), c, 0.0)
    c[0] = 0.0
    c = np.minimum(c, 1.0)
    return np.maximum(c[1:], c[:-1])  # faces i+1/2 and i-1/2 of interior node i


def to_dev(*arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


@pytest.fixture(scope="module")
def c1_ref():
    pb = oracle_problem()
    P, H0, info = lr.solve(pb)
    assert info["converged"]
    return pb, P, H0


def states(pb, P_ref, H0_ref):
    """Converged state, a perturbed state and the Hertzian start."""
    rng = np.random.default_rng(5)
    P2 = np.maximum(P_ref * (1 + 0.05 * rng.standard_normal(pb.n)), 0.0)
    Ph = pb.hertz()
    return [(P_ref, H0_ref), (P2, H0_ref + 0.01), (Ph, pb.h0_for_min_film(Ph, 0.1))]


@pytest.mark.parametrize("limiter,compressible,elastic,rough", [(0, 1, 1, False), (1, 1, 1, False),
                                                                (1, 0, 1, False), (0, 0, 0, False),
                                                                (1, 1, 1, True)])
def test_residual_matches_oracle(c1_ref, limiter, compressible, elastic, rough):
    _, P_ref, H0_ref = c1_ref
    N = 129
    rgh = 0.02 * np.sin(np.linspace(0, 20, N)) if rough else None
    pb = oracle_problem(N, limiter=limiter, compressible=compressible, elastic=elastic, rough=rgh)
    ctx, _ = make(N, limiter=limiter, compressible=compressible, elastic=elastic)
    for P, H0 in states(pb, P_ref, H0_ref):
        Pn = pb.full(P)
        Pd, H0d = to_dev(Pn[None], np.array([H0]))
        rd = None if rgh is None else to_dev(rgh[None])[0]
        R, H, comp = ctx.residual(Pd, H0d, rd)
        torch.cuda.synchronize()
        R, H, comp = R.cpu().numpy()[0], H.cpu().numpy()[0], comp.cpu().numpy()[0]
        s = lr.state(pb, P, H0)
        assert np.max(np.abs(H - s["H"])) <= 1e-13 * np.max(np.abs(s["H"]))
        scale = row_scale(pb, P, H0)
        assert np.all(np.abs(R[1:-1] - s["R"]) <= 1e-12 * scale + 1e-300)
        assert R[0] == 0.0 and R[-1] == 0.0
        cr, g = lr.comp_residual(pb, P, H0)
        assert abs(comp[0] - cr) <= 1e-12 * max(1.0, np.max(scale))
        assert abs(comp[1] - g) <= 1e-13


@pytest.mark.parametrize("limiter", [0, 1])
@pytest.mark.parametrize("beta", [1, 2, 4])
def test_paper_band_jacobian_matches_oracle(c1_ref, limiter, beta):
    _, P_ref, H0_ref = c1_ref
    pb = oracle_problem(limiter=limiter)
    ctx, _ = make(limiter=limiter, beta=beta)
    for P, H0 in states(pb, P_ref, H0_ref):
        Pd, H0d = to_dev(pb.full(P)[None], np.array([H0]))
        band, act = ctx.jacobian_band(Pd, H0d, kind=0)
        torch.cuda.synchronize()
        band, act = band.cpu().numpy()[0], act.cpu().numpy()[0].astype(bool)
        ref, ract = lr.jacobian_band(pb, P, H0, beta)
        assert np.array_equal(act, ract)
        # the distributed entries J_f(c) - w (J_f(c-1) + J_f(c+1)) cancel terms as large as the
        # frozen row itself: measure the rounding against the frozen row's magnitude
        Jf = lr.jacobian_frozen(pb, P, H0)
        mag = (1 + 2 * pb.dist_weight) * np.max(np.abs(Jf), axis=1, keepdims=True)
        cond = limiter_conditioning(pb, P, H0)[:, None]
        tol = (1e-12 + 10 * cond) * mag + 1e-300
        assert np.all(np.abs(band - ref) <= tol)


@pytest.mark.parametrize("limiter", [0, 1])
def test_exact_band_jacobian_matches_oracle(c1_ref, limiter):
    _, P_ref, H0_ref = c1_ref
    beta = 3
    pb = oracle_problem(limiter=limiter)
    ctx, _ = make(limiter=limiter, beta=beta)
    for P, H0 in states(pb, P_ref, H0_ref):
        Pd, H0d = to_dev(pb.full(P)[None], np.array([H0]))
        band, act = ctx.jacobian_band(Pd, H0d, kind=1)
        torch.cuda.synchronize()
        band, act = band.cpu().numpy()[0], act.cpu().numpy()[0].astype(bool)
        J, _ = lr.jacobian_exact(pb, P, H0)
        R = lr.residual(pb, P, H0)
        # row scale of the library: max(|J_ii|, max_{|j-i|<=beta} |J_ij| / 10)
        Jb = np.array([[J[i, j] if abs(i - j) <= beta else 0.0 for j in range(pb.n)] for i in range(pb.n)])
        dsc = np.maximum(np.abs(np.diag(J)), 0.1 * np.max(np.abs(Jb), axis=1))
        ract = P <= R / dsc
        assert np.array_equal(act, ract)
        n = pb.n
        cond = limiter_conditioning(pb, P, H0)
        for i in range(n):
            for j in range(2 * beta + 1):
                c = i - beta + j
                ref = 0.0 if (c < 0 or c >= n) else J[i, c]
                if ract[i]:
                    ref = 1.0 if j == beta else 0.0
                # van Leer derivatives 2b^2/(a+b)^2 amplify the relative change of a, b up to ~4x per face
                assert abs(band[i, j] - ref) <= (1e-11 + 50 * cond[i]) * np.max(np.abs(J[i]))


def test_paper_method_converges_to_oracle_fixed_point(c1_ref):
    pb, P_ref, H0_ref = c1_ref
    ctx, _ = make(method=0, tol=1e-11, max_iter=3000)
    P, H0, iters, res, code = ctx.solve()
    torch.cuda.synchronize()
    assert code == 0
    P, H0, iters, res = P.cpu().numpy()[0], H0.cpu().numpy()[0], int(iters.cpu()[0]), res.cpu().numpy()[0]
    # converged to tol, or stopped at the rounding floor of R (1e3 roundoff units of its largest term)
    assert res[0] <= max(1e-11, lr.rounding_floor(pb, P[1:-1], H0)) and abs(res[1]) <= 1e-11
    assert 10 < iters < 3000
    assert P[0] == 0 and P[-1] == 0
    assert np.max(np.abs(P[1:-1] - P_ref)) <= 1e-8 * np.max(P_ref)
    assert abs(H0 - H0_ref) <= 1e-8 * abs(H0_ref)
    H = pb.film(P[1:-1], H0)
    assert np.max(np.abs(H - pb.film(P_ref, H0_ref))) <= 1e-8 * np.max(np.abs(H))


def test_paper_method_batch_of_instances():
    per = [dict(M=15.0, L=8.0), dict(M=20.0, L=10.0), dict(M=25.0, L=12.0)]
    ctx, _ = make(method=0, tol=1e-11, max_iter=4000, n_inst=3, per=per)
    P, H0, iters, res, code = ctx.solve()
    torch.cuda.synchronize()
    assert code == 0
    P, H0 = P.cpu().numpy(), H0.cpu().numpy()
    for k, d in enumerate(per):
        pb = oracle_problem(M=d["M"], L=d["L"])
        Pr, H0r, info = lr.solve(pb)
        assert info["converged"]
        assert np.max(np.abs(P[k, 1:-1] - Pr)) <= 1e-8 * np.max(Pr)
        assert abs(H0[k] - H0r) <= 1e-8 * abs(H0r)


@pytest.mark.parametrize("limiter", [0, 1])
@pytest.mark.parametrize("N,M", [(129, 20.0), (513, 200.0)])
def test_jacobian_apply_matches_oracle(limiter, N, M):
    pb = oracle_problem(N, M=M, limiter=limiter)
    ctx, _ = make(N, M=M, limiter=limiter)
    rng = np.random.default_rng(N)
    P = pb.hertz() * (1 + 0.05 * rng.standard_normal(pb.n)).clip(0)
    H0 = pb.h0_for_min_film(P, 0.05)
    J, JH = lr.jacobian_exact(pb, P, H0)
    v = rng.standard_normal(pb.n)
    vh = 0.3
    ref = J @ v + JH * vh
    Pd, H0d, vd, vhd = to_dev(pb.full(P)[None], np.array([H0]), pb.full(v)[None], np.array([vh]))
    out = ctx.jacobian_apply(Pd, H0d, vd, vhd)
    torch.cuda.synchronize()
    out = out.cpu().numpy()[0]
    scale = np.abs(J) @ np.abs(v) + np.abs(JH) * abs(vh)
    cond = limiter_conditioning(pb, P, H0)
    assert out[0] == 0 and out[-1] == 0
    assert np.all(np.abs(out[1:-1] - ref) <= (1e-12 + 50 * cond) * scale + 1e-300)
