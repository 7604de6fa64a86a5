"""GPU parity of the point-contact path (dim = 2) with the point oracle, through the C ABI.

Oracle arrays are [nx, ny] (x first); the library's are [instance][ny][nx].
"""
import numpy as np
import pytest
import torch

from oracle import point_ref as pr
from paper_2008_03276_gb300 import inputs, ops

pytestmark = pytest.mark.gpu

LIM = {0: "minmod", 1: "vanleer"}


def dev(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def make(n, M=20.0, L=10.0, limiter=0, beta=2, tol=1e-11, n_inst=1, per=None, levels=-1, **kw):
    q = dict(nx=n, ny=n, limiter=limiter, halfband=beta, method=1, tol=tol, max_iter=80, levels=levels,
             coarse_min_nodes=17)
    q.update({"krylov_dim": 40, **kw})
    p = ops.default_params(2, M=M, L=L, **q)
    per_inst = None if per is None else [ops.default_params(2, **q, **d) for d in per]
    return ops.Context(p, n_inst=n_inst, per_inst=per_inst)


def perturbed_state(pb, seed):
    rng = np.random.default_rng(seed)
    P = pb.hertz() * (1 + 0.05 * rng.standard_normal(pb.n)).clip(0)
    return P, pb.h0_for_min_film(P, 0.1)


def to_gpu_nodal(pb, P_int):
    return pb.full(P_int).T.copy()      # [ny, nx]


def rough2(n, seed, amp=0.01):
    X = np.linspace(-4.5, 1.5, n)
    rx = inputs.sin_grf_roughness(X, seed=seed, amp=amp, wavelength=0.5, sigma=amp / 2, corr=0.2)
    ry = np.cos(2 * np.pi * np.linspace(-3, 3, n) / 0.7)
    return amp * 0.5 * np.outer(ry, np.ones(n)) + rx[None, :]   # [ny, nx]


@pytest.mark.parametrize("limiter,rough", [(0, False), (1, False), (1, True)])
@pytest.mark.parametrize("n", [33, 65])
def test_point_residual_matches_oracle(n, limiter, rough):
    rg = rough2(n, seed=n) if rough else None
    pb = pr.PointProblem(n, n, 20.0, 10.0, limiter=LIM[limiter], rough=None if rg is None else rg.T)
    ctx = make(n, limiter=limiter)
    P, H0 = perturbed_state(pb, n)
    R, H, comp = ctx.residual(dev(to_gpu_nodal(pb, P)[None]), dev([H0]), None if rg is None else dev(rg[None]))
    R, H, comp = R.cpu().numpy()[0], H.cpu().numpy()[0], comp.cpu().numpy()[0]
    s = pr.state(pb, P, H0)
    assert np.max(np.abs(H - s["H"].T)) <= 1e-13 * np.max(np.abs(s["H"]))
    Rr = s["R"]                                   # [nx-2, ny-2]
    scale = max(1.0, np.max(np.abs(Rr)))
    assert np.max(np.abs(R[1:-1, 1:-1] - Rr.T)) <= 1e-11 * scale
    assert np.all(R[0] == 0) and np.all(R[:, 0] == 0)
    cr, g = pr.comp_residual(pb, P, H0)
    assert abs(comp[0] - cr) <= 1e-11 * scale
    assert abs(comp[1] - g) <= 1e-13


@pytest.mark.parametrize("limiter", [0, 1])
def test_point_band_and_jacobian_apply_match_oracle(limiter):
    n, beta = 33, 3
    pb = pr.PointProblem(n, n, 20.0, 10.0, limiter=LIM[limiter])
    ctx = make(n, limiter=limiter, beta=beta)
    P, H0 = perturbed_state(pb, 7)
    J, JH = pr.jacobian_exact(pb, P, H0)
    Pd, H0d = dev(to_gpu_nodal(pb, P)[None]), dev([H0])
    band, act = ctx.jacobian_band(Pd, H0d, kind=1)
    band, act = band.cpu().numpy()[0], act.cpu().numpy()[0]    # [ny-2][nx-2][bw]
    R = pr.residual(pb, P, H0)
    ni = n - 2
    scale = np.max(np.abs(J))
    for jr in range(0, ni, 5):                # grid row j = jr + 1
        for ir in range(ni):
            r_or = ir * ni + jr               # oracle interior index (x major)
            cols = [ic * ni + jr for ic in range(max(0, ir - beta), min(ni, ir + beta + 1))]
            d = max(abs(J[r_or, r_or]), 0.1 * np.max(np.abs(J[r_or, cols]))) or 1.0
            identity = P[r_or] <= R[r_or] / d
            assert bool(act[jr, ir]) == identity
            for t in range(2 * beta + 1):
                ic = ir - beta + t
                if identity:
                    ref = 1.0 if t == beta else 0.0
                elif 0 <= ic < ni:
                    ref = J[r_or, ic * ni + jr]
                else:
                    ref = 0.0
                assert abs(band[jr, ir, t] - ref) <= 1e-11 * scale, (jr, ir, t)
    rng = np.random.default_rng(3)
    v = rng.standard_normal(pb.n)
    vh = 0.7
    ref = J @ v + JH * vh
    out = ctx.jacobian_apply(Pd, H0d, dev(to_gpu_nodal(pb, v)[None]), dev([vh])).cpu().numpy()[0]
    sc = np.abs(J) @ np.abs(v) + np.abs(JH) * vh
    assert np.all(np.abs(out[1:-1, 1:-1] - ref.reshape(ni, ni).T) <= 1e-11 * sc.reshape(ni, ni).T + 1e-300)


@pytest.fixture(scope="module")
def oracle_33():
    pb = pr.PointProblem(33, 33, 20.0, 10.0)
    P, H0, info = pr.solve(pb, tol=1e-11)
    assert info["converged"]
    return pb, P, H0


@pytest.mark.parametrize("levels,beta,precision", [(0, 2, 0), (-1, 2, 0), (-1, 4, 0), (-1, 2, 2), (-1, 2, 3)])
def test_point_solve_matches_oracle(oracle_33, levels, beta, precision):
    """precision > 0: the Krylov products as one tensor-core GEMM per instance (the residual stays float64)."""
    pb, Pr, H0r = oracle_33
    ctx = make(33, levels=levels, beta=beta, precision=precision)
    P, H0, iters, res, code = ctx.solve(check=False)
    print(f"levels {levels} beta {beta} precision {precision}: code {code} iters {iters.tolist()} res {res.tolist()}")
    assert code == 0
    P, H0 = P.cpu().numpy()[0], float(H0.cpu()[0])
    assert np.max(np.abs(P[1:-1, 1:-1] - pb.full(Pr)[1:-1, 1:-1].T)) <= 1e-8 * np.max(Pr)
    assert abs(H0 - H0r) <= 1e-8 * abs(H0r)


@pytest.mark.slow
def test_point_solve_129_properties():
    n = 129
    # the x-line preconditioner leaves the y-coupling to GMRES: at 129^2 a 40-vector basis is
    # marginal (the Newton iteration can stall at |Phi| ~ 1e-11), 100 vectors suffice
    ctx = make(n, M=100.0, L=10.0, limiter=1, beta=4, tol=1e-8, krylov_dim=100)
    P, H0, iters, res, code = ctx.solve(check=False)
    print(f"129^2: code {code} iters {iters.tolist()} res {res.tolist()}")
    assert code == 0
    Pn, H0n = P.cpu().numpy()[0], float(H0.cpu()[0])
    pb = pr.PointProblem(n, n, 100.0, 10.0, limiter="vanleer")
    Pint = Pn.T[1:-1, 1:-1].ravel()
    R = pr.residual(pb, Pint, H0n)       # the oracle's residual at the GPU's solution
    assert np.max(np.abs(np.minimum(Pint, R))) <= 2e-8
    assert abs(pb.h**2 * Pint.sum() - 2 * np.pi / 3) <= 1e-8
    assert np.max(np.abs(Pn - Pn[::-1, :])) <= 1e-6 * np.max(Pn)       # Y -> -Y


# ---------------------------------------------------------------- point-contact adjoint
@pytest.mark.parametrize("which", ["H_c", "P2"])
def test_point_adjoint_matches_dense_oracle(which):
    n, M, L = 33, 20.0, 10.0
    rg = rough2(n, seed=5, amp=0.005)                     # [ny, nx]
    ctx = make(n, M=M, L=L, tol=1e-12)
    P, H0, iters, res, code = ctx.solve(rough=dev(rg[None]), check=False)
    assert code == 0
    Pn, H0n = P.cpu().numpy()[0], float(H0.cpu()[0])
    pb = pr.PointProblem(n, n, M, L, rough=rg.T)
    Pint = Pn.T[1:-1, 1:-1].ravel()
    gP, gH = np.zeros((n, n)), np.zeros((n, n))          # oracle layout [nx, ny]
    if which == "H_c":
        gH[int(np.argmin(np.abs(pb.X))), int(np.argmin(np.abs(pb.Y)))] = 1.0
    else:
        gP[:] = 2.0 * pb.h**2 * pb.full(Pint)
    ref = pr.adjoint(pb, Pint, H0n, gP, gH, 0.0)
    gr, gml, rel, code = ctx.adjoint(P, H0, dev(gP.T[None]), dev(gH.T[None]), None, rough=dev(rg[None]), tol=1e-11,
                                     max_cycles=20)
    assert code == 0, rel.tolist()
    gr, gml = gr.cpu().numpy()[0].T, gml.cpu().numpy()[0]  # back to [nx, ny]
    scale = np.max(np.abs(ref["rough"]))
    assert np.max(np.abs(gr - ref["rough"])) <= 1e-8 * scale, np.max(np.abs(gr - ref["rough"])) / scale
    assert abs(gml[0] - ref["M"]) <= 1e-8 * abs(ref["M"])
    assert abs(gml[1] - ref["L"]) <= 1e-8 * abs(ref["L"])


@pytest.mark.slow
def test_point_adjoint_129_vs_resolved_differences():
    """The adjoint workload's point-contact backward: 129 x 129, M = 100, L = 10."""
    n, M, L = 129, 100.0, 10.0
    rg = rough2(n, seed=9, amp=0.005)
    ctx = make(n, M=M, L=L, beta=4, tol=1e-11, krylov_dim=100)
    P, H0, iters, res, code = ctx.solve(rough=dev(rg[None]), check=False)
    assert code == 0, (iters.tolist(), res.tolist())
    X, Y = np.linspace(-4.5, 1.5, n), np.linspace(-3, 3, n)
    ci, cj = int(np.argmin(np.abs(X))), int(np.argmin(np.abs(Y)))
    gH = np.zeros((n, n))
    gH[cj, ci] = 1.0                                       # H_c, GPU layout [ny, nx]
    gr, gml, rel, code = ctx.adjoint(P, H0, None, dev(gH[None]), None, rough=dev(rg[None]), tol=1e-11, max_cycles=20)
    assert code == 0, rel.tolist()
    gr, gml = gr.cpu().numpy()[0], gml.cpu().numpy()[0]

    def hc(rgx, M_=M, L_=L):
        cx = make(n, M=M_, L=L_, beta=4, tol=1e-12, krylov_dim=100)
        Pp, H0p, it, rs, cd = cx.solve(P, H0, rough=dev(rgx[None]), check=False)
        _, H, _ = cx.residual(Pp, H0p, dev(rgx[None]))
        return float(H[0, cj, ci].cpu())

    # a re-solve to tol 1e-12 reproduces H_c to a few 1e-11 (its rounding floor: 2.8e-11
    # measured), so a central difference with step d carries an error up to eps_h / d: the
    # small off-centre gradient (1e-3 of the central one) takes a wider step
    eps_h = 5e-11
    for node, d in (((cj, ci), 1e-6), ((cj + 3, ci - 4), 1e-4)):
        rp, rm = rg.copy(), rg.copy()
        rp[node] += d
        rm[node] -= d
        fd = (hc(rp) - hc(rm)) / (2 * d)
        assert abs(fd - gr[node]) <= 1e-5 * abs(fd) + eps_h / d, (node, fd, gr[node])
    # M enters smoothly; a wider step keeps the re-solves' rounding floor (~1e-11 in H_c) out of the difference
    dm = 1e-4
    fd = (hc(rg, M_=M * (1 + dm)) - hc(rg, M_=M * (1 - dm))) / (2 * dm * M)
    assert abs(fd - gml[0]) <= 1e-5 * abs(fd), (fd, gml[0])
