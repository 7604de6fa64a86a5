"""GPU parity of van Leer's kappa-schemes in the EHL residual and Jacobians (Sec. 3.1, Eq. eqn41;
Sec. 3.3.2, Eqs. eqn56-eqn61) against the float64 oracle, through the C ABI.

limiter = 2 selects the unlimited kappa-scheme (kappa in {0, 1/3, -1}); splitting = 1, 2 the
hybrid splittings L_hs1, L_hs2 of the kind-0 Newton matrix.  Tolerances as in
test_gpu_line.py: residual 1e-12 of the row's terms, exact band 1e-11 of the row's largest
entry, kind-0 band 1e-12 of the frozen row (plus the frozen factor's conditioning where the
splitting keeps psi / a), converged P, H0, H 1e-8.
"""
import numpy as np
import pytest
import torch

from oracle import line_ref as lr
from oracle import point_ref as ptr
from paper_2008_03276_gb300 import ops

pytestmark = pytest.mark.gpu
KAPPAS = [0.0, 1.0 / 3.0, -1.0]
SPLIT = {0: "frozen", 1: "hs1", 2: "hs2"}


def to_dev(*arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


def problem(kappa, N=129, splitting=0):
    return lr.LineProblem(N, 20.0, 10.0, limiter="kappa", kappa=kappa, dist_weight=0.5, splitting=SPLIT[splitting])


def context(kappa, N=129, beta=2, splitting=0, method=1, **kw):
    p = ops.default_params(1, nx=N, M=20.0, L=10.0, limiter=2, kappa=kappa, halfband=beta, splitting=splitting,
                           method=method, **kw)
    return ops.Context(p)


def row_scale(pb, P, H0):
    s = lr.state(pb, P, H0)
    F, ef, Pn, h = s["F"], s["epsf"], s["P"], pb.h
    return (np.abs(F[1:]) + np.abs(F[:-1])) / h + (np.abs(ef[1:] * (Pn[2:] - Pn[1:-1])) +
                                                   np.abs(ef[:-1] * (Pn[1:-1] - Pn[:-2]))) / h**2


def frozen_conditioning(pb, P, H0, rel=1e-14):
    s = lr.state(pb, P, H0)
    u, a = s["u"], s["a"]
    with np.errstate(divide="ignore", invalid="ignore"):
        c = rel * np.abs(u[:-1]) / np.abs(a)
    c = np.where(np.isfinite(c), c, 0.0)
    c[0] = 0.0
    c = np.minimum(c, 1.0)
    return np.maximum(c[1:], c[:-1])


@pytest.fixture(scope="module", params=KAPPAS)
def kappa_state(request):
    kappa = request.param
    pb = problem(kappa)
    P, H0, info = lr.solve(pb)
    assert info["converged"]
    rng = np.random.default_rng(3)
    P2 = np.maximum(P * (1 + 0.05 * rng.standard_normal(pb.n)), 0.0)
    Ph = pb.hertz()
    return kappa, pb, P, H0, [(P, H0), (P2, H0 + 0.01), (Ph, pb.h0_for_min_film(Ph, 0.1))]


def test_residual(kappa_state):
    kappa, pb, _, _, sts = kappa_state
    ctx = context(kappa)
    for P, H0 in sts:
        Pd, H0d = to_dev(pb.full(P)[None], np.array([H0]))
        R, H, comp = ctx.residual(Pd, H0d)
        R, H = R.cpu().numpy()[0], H.cpu().numpy()[0]
        s = lr.state(pb, P, H0)
        assert np.max(np.abs(H - s["H"])) <= 1e-13 * np.max(np.abs(s["H"]))
        assert np.all(np.abs(R[1:-1] - s["R"]) <= 1e-12 * row_scale(pb, P, H0) + 1e-300)


def test_exact_band(kappa_state):
    kappa, pb, _, _, sts = kappa_state
    beta = 3
    ctx = context(kappa, beta=beta)
    for P, H0 in sts:
        Pd, H0d = to_dev(pb.full(P)[None], np.array([H0]))
        band, act = ctx.jacobian_band(Pd, H0d, kind=1)
        band, act = band.cpu().numpy()[0], act.cpu().numpy()[0].astype(bool)
        J, _ = lr.jacobian_exact(pb, P, H0)
        n = pb.n
        for i in range(n):
            if act[i]:
                continue
            for j in range(2 * beta + 1):
                c = i - beta + j
                ref = 0.0 if (c < 0 or c >= n) else J[i, c]
                assert abs(band[i, j] - ref) <= 1e-11 * np.max(np.abs(J[i]))


@pytest.mark.parametrize("splitting", [0, 1, 2])
def test_kind0_band_of_each_splitting(kappa_state, splitting):
    kappa, _, _, _, sts = kappa_state
    pb = problem(kappa, splitting=splitting)
    beta = 2
    ctx = context(kappa, beta=beta, splitting=splitting, method=0)
    for P, H0 in sts:
        Pd, H0d = to_dev(pb.full(P)[None], np.array([H0]))
        band, act = ctx.jacobian_band(Pd, H0d, kind=0)
        band, act = band.cpu().numpy()[0], act.cpu().numpy()[0].astype(bool)
        ref, ract = lr.jacobian_band(pb, P, H0, beta)
        assert np.array_equal(act, ract)
        Jf = lr.jacobian_frozen(pb, P, H0)
        mag = (1 + 2 * pb.dist_weight) * np.max(np.abs(Jf), axis=1, keepdims=True)
        cond = frozen_conditioning(pb, P, H0)[:, None] if splitting == 0 else 0.0
        assert np.all(np.abs(band - ref) <= (1e-12 + 10 * cond) * mag + 1e-300)


def test_newton_krylov_solution(kappa_state):
    kappa, pb, P_ref, H0_ref, _ = kappa_state
    ctx = context(kappa, tol=1e-11, max_iter=100)
    P, H0, iters, res, code = ctx.solve()
    assert code == 0
    P, H0 = P.cpu().numpy()[0], float(H0.cpu()[0])
    assert np.max(np.abs(P[1:-1] - P_ref)) <= 1e-8 * np.max(P_ref)
    assert abs(H0 - H0_ref) <= 1e-8 * abs(H0_ref)
    H = pb.film(P[1:-1], H0)
    assert np.max(np.abs(H - pb.film(P_ref, H0_ref))) <= 1e-8 * np.max(np.abs(H))


@pytest.mark.parametrize("kappa", KAPPAS)
def test_point_residual(kappa):
    n = 33
    pb = ptr.PointProblem(n, n, 20.0, 10.0, limiter="kappa", kappa=kappa)
    rng = np.random.default_rng(n)
    P = pb.hertz() * (1 + 0.05 * rng.standard_normal(pb.n)).clip(0)
    H0 = pb.h0_for_min_film(P, 0.1)
    p = ops.default_params(2, nx=n, ny=n, M=20.0, L=10.0, limiter=2, kappa=kappa, method=1)
    ctx = ops.Context(p)
    Pd, H0d = to_dev(pb.full(P).T.copy()[None], np.array([H0]))
    R, H, comp = ctx.residual(Pd, H0d)
    R, H = R.cpu().numpy()[0], H.cpu().numpy()[0]
    s = ptr.state(pb, P, H0)
    assert np.max(np.abs(H - s["H"].T)) <= 1e-13 * np.max(np.abs(s["H"]))
    assert np.max(np.abs(R[1:-1, 1:-1] - s["R"].T)) <= 1e-11 * max(1.0, np.max(np.abs(s["R"])))
