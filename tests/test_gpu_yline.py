"""GPU parity of the y-line stage of the point-contact preconditioner (ehl_params.yline = 1).

The alternating line splitting of Sec. 3.3.2-3.3.4 solves x-line and then y-line systems; the
library's preconditioner for the Newton-Krylov solve applies the bordered x-line solve and
then the bordered y-line solve of the remaining residual.  Checked against the oracle:
the y-line bands (ehl_jacobian_band kind 2) entry by entry against point_ref.yline_band_exact
(1e-11 of the row's largest exact entry), and the converged solution with the y-line stage on
(1e-8 at 33^2).  The stage is not a better preconditioner: at 65^2 and 257^2 with M = 100 it
stalls GMRES (the y-line systems of the Hertzian zone, where eps vanishes, couple only
through the kernel's Couette differences and are far from dominant), so these sizes are
measured, not tested.
"""
import numpy as np
import pytest
import torch

from oracle import point_ref as pr
from paper_2008_03276_gb300 import ops

pytestmark = pytest.mark.gpu
LIM = {0: "minmod", 1: "vanleer"}


def dev(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


@pytest.mark.parametrize("limiter,beta", [(0, 2), (1, 3)])
def test_yline_bands_match_oracle(limiter, beta):
    n = 33
    pb = pr.PointProblem(n, n, 20.0, 10.0, limiter=LIM[limiter])
    rng = np.random.default_rng(11)
    P = pb.hertz() * (1 + 0.05 * rng.standard_normal(pb.n)).clip(0)
    H0 = pb.h0_for_min_film(P, 0.1)
    ctx = ops.Context(ops.default_params(2, nx=n, ny=n, M=20.0, L=10.0, limiter=limiter, halfband=beta, method=1))
    Pd, H0d = dev(pb.full(P).T[None]), dev([H0])
    band, act = ctx.jacobian_band(Pd, H0d, kind=2)
    _, actx = ctx.jacobian_band(Pd, H0d, kind=1)
    band, act = band.cpu().numpy()[0], act.cpu().numpy()[0].astype(bool)  # band [x][y][t], act [y][x]
    assert np.array_equal(act, actx.cpu().numpy()[0].astype(bool))
    ref = pr.yline_band_exact(pb, P, H0, beta)  # [x][y][t]
    J, _ = pr.jacobian_exact(pb, P, H0)
    rowmax = np.max(np.abs(J), axis=1).reshape(n - 2, n - 2)  # oracle rows x-major
    for i in range(n - 2):
        for j in range(n - 2):
            if act[j, i]:
                want = np.zeros(2 * beta + 1)
                want[beta] = 1.0
                assert np.array_equal(band[i, j], want)
            else:
                assert np.max(np.abs(band[i, j] - ref[i, j])) <= 1e-11 * rowmax[i, j], (i, j)


@pytest.mark.parametrize("deform", [0, 1])
def test_solve_with_yline_stage_matches_oracle(deform):
    pb = pr.PointProblem(33, 33, 20.0, 10.0)
    Pr, H0r, info = pr.solve(pb, tol=1e-11)
    assert info["converged"]
    p = ops.default_params(2, nx=33, ny=33, M=20.0, L=10.0, method=1, tol=1e-11, max_iter=80, coarse_min_nodes=17,
                           krylov_dim=40, yline=1, deform=deform)
    ctx = ops.Context(p)
    P, H0, iters, res, code = ctx.solve(check=False)
    assert code == 0
    P, H0 = P.cpu().numpy()[0], float(H0.cpu()[0])
    assert np.max(np.abs(P[1:-1, 1:-1] - pb.full(Pr)[1:-1, 1:-1].T)) <= 1e-8 * np.max(Pr)
    assert abs(H0 - H0r) <= 1e-8 * abs(H0r)
