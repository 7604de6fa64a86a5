"""GPU adjoint (ehl_adjoint) against the dense adjoint oracle and central differences.

The oracle's dense adjoint is evaluated at the GPU's converged state, so the
comparison isolates the transposed solve: gradients must agree to 1e-8
(normwise for the roughness profile).  Central differences of re-converged
GPU solutions (step 1e-6) must agree to 1e-5.
"""
import numpy as np
import pytest
import torch

from oracle import adjoint_ref as ar
from oracle import line_ref as lr
from paper_2008_03276_gb300 import inputs, ops

pytestmark = pytest.mark.gpu

LIM = {0: "minmod", 1: "vanleer"}


def dev(a):
    return torch.tensor(np.asarray(a, dtype=np.float64), device="cuda")


def make(N, M, L, limiter=0, beta=4, tol=1e-12, n_inst=1, per=None):
    kw = dict(nx=N, limiter=limiter, halfband=beta, method=1, tol=tol, max_iter=80, krylov_dim=40)
    p = ops.default_params(1, M=M, L=L, **kw)
    per_inst = None if per is None else [ops.default_params(1, **kw, **d) for d in per]
    return ops.Context(p, n_inst=n_inst, per_inst=per_inst)


def roughness(N, seed, amp=0.01, wavelength=0.5, sigma=0.005, corr=0.2):
    X = np.linspace(-4.5, 1.5, N)
    return inputs.sin_grf_roughness(X, seed=seed, amp=amp, wavelength=wavelength, sigma=sigma, corr=corr)


def rows(a):
    a = np.asarray(a, dtype=np.float64)
    return a[None] if a.ndim == 1 else a


def solve(ctx, rgh):
    P, H0, iters, res, code = ctx.solve(rough=dev(rows(rgh)))
    return P, H0


def seeds(pbs, P, H0, which):
    gP, gH, gH0 = [], [], []
    for k, pb in enumerate(pbs):
        _, a, b, c = ar.objective_seeds(pb, P[k, 1:pb.N - 1], H0[k], which)
        gP.append(a)
        gH.append(b)
        gH0.append(c)
    return np.array(gP), np.array(gH), np.array(gH0)


@pytest.mark.parametrize("N,M,L,limiter,beta", [(129, 20.0, 10.0, 0, 2), (257, 50.0, 10.0, 1, 4),
                                                (513, 200.0, 10.0, 1, 8)])
@pytest.mark.parametrize("which", ["H_c", "H_min", "P2"])
def test_adjoint_matches_dense_oracle(N, M, L, limiter, beta, which):
    rgh = roughness(N, seed=N)
    ctx = make(N, M, L, limiter, beta)
    P, H0 = solve(ctx, rgh)
    Pn, H0n = P.cpu().numpy(), H0.cpu().numpy()
    pb = lr.LineProblem(N, M, L, limiter=LIM[limiter], rough=rgh)
    gP, gH, gH0 = seeds([pb], Pn, H0n, which)
    gr, gml, rel, code = ctx.adjoint(P, H0, dev(gP), dev(gH), dev(gH0), rough=dev(rows(rgh)), tol=1e-11)
    assert code == 0, (code, rel.cpu().numpy())
    ref = ar.adjoint(pb, Pn[0, 1:-1], H0n[0], gP[0], gH[0], gH0[0])
    gr, gml = gr.cpu().numpy()[0], gml.cpu().numpy()[0]
    scale = np.max(np.abs(ref["rough"]))
    assert np.max(np.abs(gr - ref["rough"])) <= 1e-8 * scale, np.max(np.abs(gr - ref["rough"])) / scale
    assert abs(gml[0] - ref["M"]) <= 1e-8 * abs(ref["M"]) + 1e-12 * scale
    assert abs(gml[1] - ref["L"]) <= 1e-8 * abs(ref["L"]) + 1e-12 * scale


def test_adjoint_matches_resolved_differences():
    N, M, L = 257, 50.0, 10.0
    rgh = roughness(N, seed=7)
    ctx = make(N, M, L, 1, 4)
    P, H0 = solve(ctx, rgh)
    pb = lr.LineProblem(N, M, L, limiter="vanleer", rough=rgh)
    c = int(np.argmin(np.abs(pb.X)))

    def value(rg, M_=M, L_=L):
        cx = make(N, M_, L_, 1, 4)
        Pp, H0p, it, res, code = cx.solve(P, H0, rough=dev(rows(rg)))
        _, H, _ = cx.residual(Pp, H0p, dev(rows(rg)))
        return float(H[0, c].cpu())

    gH = np.zeros((1, N))
    gH[0, c] = 1.0
    gr, gml, rel, code = ctx.adjoint(P, H0, None, dev(gH), None, rough=dev(rows(rgh)), tol=1e-11)
    gr, gml = gr.cpu().numpy()[0], gml.cpu().numpy()[0]
    d = 1e-6
    for k in (100, 180, 200):
        rp, rm = rgh.copy(), rgh.copy()
        rp[k] += d
        rm[k] -= d
        fd = (value(rp) - value(rm)) / (2 * d)
        assert abs(fd - gr[k]) <= 1e-5 * abs(fd) + 1e-7 * np.max(np.abs(gr)), (k, fd, gr[k])
    fdM = (value(rgh, M * (1 + d)) - value(rgh, M * (1 - d))) / (2 * d * M)
    fdL = (value(rgh, L_=L * (1 + d)) - value(rgh, L_=L * (1 - d))) / (2 * d * L)
    assert abs(fdM - gml[0]) <= 1e-5 * abs(fdM)
    assert abs(fdL - gml[1]) <= 1e-5 * abs(fdL)


def test_autograd_function_batch():
    """A batch of loads and roughness profiles through torch.autograd: H_min, H_c and
    h sum P^2 summed into one loss; per-instance gradients equal the dense oracle."""
    N = 257
    per = [dict(M=20.0, L=10.0), dict(M=50.0, L=8.0), dict(M=120.0, L=12.0)]
    ctx = make(N, 20.0, 10.0, 0, 4, tol=1e-10, n_inst=3, per=per)
    rgh = np.stack([roughness(N, seed=30 + k) for k in range(3)])
    rough = dev(rgh).requires_grad_(True)
    ML = dev([[d["M"], d["L"]] for d in per]).requires_grad_(True)
    P, H, H0 = ops.solve_differentiable(ctx, rough, ML)
    X = torch.linspace(-4.5, 1.5, N, dtype=torch.float64, device="cuda")
    c = int(torch.argmin(X.abs()))
    h = 6.0 / (N - 1)
    loss = H.min(dim=1).values.sum() + 0.5 * H[:, c].sum() + 0.25 * h * (P ** 2).sum()
    loss.backward()
    gr, gml = rough.grad.cpu().numpy(), ML.grad.cpu().numpy()
    Pn, H0n = P.detach().cpu().numpy(), H0.detach().cpu().numpy()
    for k, d in enumerate(per):
        pb = lr.LineProblem(N, d["M"], d["L"], limiter="minmod", rough=rgh[k])
        tot = dict(rough=np.zeros(N), M=0.0, L=0.0)
        for which, wgt in (("H_min", 1.0), ("H_c", 0.5), ("P2", 0.25)):
            _, gP, gH, gH0 = ar.objective_seeds(pb, Pn[k, 1:-1], H0n[k], which)
            g = ar.adjoint(pb, Pn[k, 1:-1], H0n[k], gP, gH, gH0)
            for key in tot:
                tot[key] = tot[key] + wgt * g[key]
        scale = np.max(np.abs(tot["rough"]))
        assert np.max(np.abs(gr[k] - tot["rough"])) <= 1e-8 * scale
        assert abs(gml[k, 0] - tot["M"]) <= 1e-8 * abs(tot["M"])
        assert abs(gml[k, 1] - tot["L"]) <= 1e-8 * abs(tot["L"])


def c5_roughness(N, n, amp=0.1, sigma=0.05):
    """The adjoint workload's roughness: amp sin(2 pi X / 0.25) + a Gaussian random field
    (standard deviation sigma, correlation length 0.1), seeds 2, 3, ..."""
    X = np.linspace(-4.5, 1.5, N)
    return np.stack([inputs.sin_grf_roughness(X, seed=2 + k, amp=amp, wavelength=0.25, sigma=sigma, corr=0.1)
                     for k in range(n)])


def scaled_condition(pb, P_int, H0):
    """Condition number of the bordered equation-row system, rows scaled by |dR_i/dP_i|."""
    T = ar.tangent(pb, P_int, H0)
    rows = ar.equation_rows(pb, P_int, H0, T["P"])
    A = np.nonzero(rows)[0]
    F = np.zeros((len(A) + 1, len(A) + 1))
    F[:-1, :-1] = T["P"][np.ix_(A, A)]
    F[:-1, -1] = T["H0"][A]
    F[-1, :-1] = pb.h
    d = np.abs(np.diag(T["P"]))[A]
    F[:-1] /= np.where(d > 0, d, 1.0)[:, None]
    F[-1] /= pb.h
    return np.linalg.cond(F)


@pytest.mark.slow
def test_adjoint_c5_batch_matches_oracle():
    """The adjoint workload (N = 1025, M = 50, L = 10) with the roughness recipe at a
    fifth of its amplitude (0.02 sin + field sigma 0.01): at the full amplitude the
    film reaches contact in part of the batch and the bordered system of the others
    has a scaled condition number near 1e12 (see the next test)."""
    N, M, L, n = 1025, 50.0, 10.0, 8
    rgh = c5_roughness(N, n, amp=0.02, sigma=0.01)
    ctx = make(N, M, L, 1, 8, tol=1e-10, n_inst=n)
    P, H0, iters, res, code = ctx.solve(rough=dev(rgh))
    Pn, H0n = P.cpu().numpy(), H0.cpu().numpy()
    pbs = [lr.LineProblem(N, M, L, limiter="vanleer", rough=rgh[k]) for k in range(n)]
    gP, gH, gH0 = seeds(pbs, Pn, H0n, "H_min")
    gr, gml, rel, code = ctx.adjoint(P, H0, dev(gP), dev(gH), dev(gH0), rough=dev(rgh), tol=1e-11, max_cycles=20)
    gr, gml = gr.cpu().numpy(), gml.cpu().numpy()
    for k in range(3):
        ref = ar.adjoint(pbs[k], Pn[k, 1:-1], H0n[k], gP[k], gH[k], gH0[k])
        scale = np.max(np.abs(ref["rough"]))
        assert np.max(np.abs(gr[k] - ref["rough"])) <= 1e-8 * scale
        assert abs(gml[k, 0] - ref["M"]) <= 1e-8 * abs(ref["M"])
        assert abs(gml[k, 1] - ref["L"]) <= 1e-8 * abs(ref["L"])


@pytest.mark.slow
def test_adjoint_c5_full_amplitude_reports():
    """The full-amplitude recipe: instances at or near contact (H_min <= 0) and the worst
    conditioned ones may not converge to tol 1e-10; they are reported through their
    residual and the status.  The converged ones give finite gradients that agree with the
    oracle to the accuracy their conditioning allows (1e-14 x cond)."""
    N, M, L, n = 1025, 50.0, 10.0, 8
    rgh = c5_roughness(N, n)
    ctx = make(N, M, L, 1, 8, tol=1e-10, n_inst=n)
    P, H0, iters, res, code = ctx.solve(rough=dev(rgh), check=False)
    res = res.cpu().numpy()
    ok = (np.abs(res[:, 0]) <= 1e-8) & (np.abs(res[:, 1]) <= 1e-8)
    Pn, H0n = P.cpu().numpy(), H0.cpu().numpy()
    pbs = [lr.LineProblem(N, M, L, limiter="vanleer", rough=rgh[k]) for k in range(n)]
    Hmin = np.array([pbs[k].film(Pn[k, 1:-1], H0n[k]).min() for k in range(n)])
    print("converged", ok.tolist(), "H_min", np.round(Hmin, 4).tolist())
    assert ok.sum() >= 4
    assert code == (0 if ok.all() else 4)  # EHL_ENOCONV reports the unconverged instances
    assert not np.any(ok[Hmin <= 0])       # an instance in contact never reports convergence
    gP, gH, gH0 = seeds(pbs, Pn, H0n, "H_min")
    gr, gml, rel, code = ctx.adjoint(P, H0, dev(gP), dev(gH), dev(gH0), rough=dev(rgh), tol=1e-11, max_cycles=20,
                                     check=False)
    gr, gml, rel = gr.cpu().numpy(), gml.cpu().numpy(), rel.cpu().numpy()
    print("adjoint relres", rel.tolist())
    for k in np.nonzero(ok)[0][:2]:
        assert np.all(np.isfinite(gr[k])) and rel[k] <= 1e-8
        kappa = scaled_condition(pbs[k], Pn[k, 1:-1], H0n[k])
        ref = ar.adjoint(pbs[k], Pn[k, 1:-1], H0n[k], gP[k], gH[k], gH0[k])
        scale = np.max(np.abs(ref["rough"]))
        err = np.max(np.abs(gr[k] - ref["rough"])) / scale
        print(f"instance {k}: scaled condition {kappa:.2e}, gradient difference {err:.2e}")
        assert err <= max(1e-8, 1e-14 * kappa)   # forward-error bound kappa u with a constant of ~100


@pytest.mark.slow
def test_adjoint_c5_full_amplitude_matches_resolved_differences():
    """The adjoint workload at its full roughness amplitude (N = 1025, M = 50, L = 10, van Leer,
    beta 8, 0.1 sin(2 pi X / 0.25) + field (0.05, 0.1)): on the first instance of the batch whose
    forward solve converges, the adjoint gradient of the central film H_c with respect to M, L
    and three roughness nodes near the centre against central differences of re-converged
    solves.  At this amplitude the bordered system's scaled condition number is about 6e12 and
    the re-converged solves stop at their rounding floor (a residual of about 1e-9), so a
    difference with step d carries noise that falls as 1/d: with the workload's step 1e-6 (and
    1e-5) the differences are noise, with steps 1e-4 and 1e-3 they approach the adjoint gradient
    to 2e-2 and 2e-3 (the 1/d decrease is the check)."""
    N, M, L, n = 1025, 50.0, 10.0, 8
    rgh = c5_roughness(N, n)
    ctx = make(N, M, L, 1, 8, tol=1e-12, n_inst=n)
    P, H0, iters, res, code = ctx.solve(rough=dev(rgh), check=False)
    r = np.abs(res.cpu().numpy())
    ok = np.nonzero((r[:, 0] <= 1e-8) & (r[:, 1] <= 1e-8))[0]
    assert len(ok) > 0
    k = int(ok[0])
    rk = rgh[k]
    pb = lr.LineProblem(N, M, L, limiter="vanleer", rough=rk)
    c = int(np.argmin(np.abs(pb.X)))
    P1, H01 = P[k:k + 1].contiguous(), H0[k:k + 1].contiguous()
    single = make(N, M, L, 1, 8, tol=1e-12)
    Ps, H0s, _, rs, code = single.solve(P1, H01, rough=dev(rows(rk)), check=False)
    assert float(rs.abs().max()) <= 1e-8

    def value(rg, M_=M, L_=L):
        cx = make(N, M_, L_, 1, 8, tol=1e-12)
        Pp, H0p, it, res_, code_ = cx.solve(Ps, H0s, rough=dev(rows(rg)), check=False)
        assert float(res_.abs().max()) <= 1e-8
        _, H, _ = cx.residual(Pp, H0p, dev(rows(rg)))
        return float(H[0, c].cpu())

    gH = np.zeros((1, N))
    gH[0, c] = 1.0
    gr, gml, rel, code = single.adjoint(Ps, H0s, None, dev(gH), None, rough=dev(rows(rk)), tol=1e-12, max_cycles=20,
                                        check=False)
    gr, gml = gr.cpu().numpy()[0], gml.cpu().numpy()[0]
    assert float(rel.cpu()[0]) <= 1e-8  # the transposed solve stalls near 1e-10 at this conditioning
    kappa = scaled_condition(pb, Ps.cpu().numpy()[0, 1:-1], float(H0s.cpu()[0]))
    print(f"instance {k}: scaled condition {kappa:.2e}, H_min {pb.film(Ps.cpu().numpy()[0, 1:-1], float(H0s.cpu()[0])).min():.4e}")
    # the differences' noise falls as 1/d (measured at d = 1e-6 .. 1e-3 on a GB300: worst relative
    # difference 2.9, 6.3e-2, 9.2e-3, 5.7e-4 on one instance, 11.5, 0.35 at d = 1e-6, 1e-5 on
    # another): the adjoint is the limit they approach.  Which instance converges first, and the
    # noise of its re-converged solves, move with any change of the solver's summation order, so
    # the two noise-dominated steps are printed, not checked
    for d, tol in ((1e-6, 1e9), (1e-5, 1e9), (1e-4, 2e-2), (1e-3, 2e-3)):
        errs = []
        for node in (c - 40, c - 10, c + 20):
            rp, rm = rk.copy(), rk.copy()
            rp[node] += d
            rm[node] -= d
            fd = (value(rp) - value(rm)) / (2 * d)
            errs.append(abs(fd - gr[node]) / (abs(fd) + 1e-2 * np.max(np.abs(gr))))
        fdM = (value(rk, M * (1 + d)) - value(rk, M * (1 - d))) / (2 * d * M)
        fdL = (value(rk, L_=L * (1 + d)) - value(rk, L_=L * (1 - d))) / (2 * d * L)
        errs += [abs(fdM - gml[0]) / abs(fdM), abs(fdL - gml[1]) / abs(fdL)]
        print(f"instance {k}, step {d:g}: relative differences {[f'{e:.2e}' for e in errs]}")
        assert max(errs) <= tol
