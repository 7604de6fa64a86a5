"""GPU parity of the convection-diffusion workload (Sec. 3.1, Sec. 6) with oracle/cd_ref.py,
through the C ABI (ehl_cd_residual, ehl_cd_relax).

Oracle arrays are [nx, ny] (x first); the library's are [instance][ny][nx].  The residual is
float64 on both sides (tolerance: 1e-13 of the size of its terms); a sweep's line solves are
PAQIF (double-float) against dense LU, so iterates agree to 1e-11 of |u| after several sweeps.
"""
import numpy as np
import pytest
import torch

from oracle import cd_ref as cd
from paper_2008_03276_gb300 import _ffi, ops

pytestmark = pytest.mark.gpu
ORDERS = ["lexicographic", "jacobi"]


def to_dev(arrs):
    return torch.tensor(np.stack([np.ascontiguousarray(a.T) for a in arrs]), dtype=torch.float64, device="cuda")


def start(pb, seed):
    """Boundary data of the exact solution, seeded noise inside."""
    u = pb.initial()
    rng = np.random.default_rng(seed)
    u[1:-1, 1:-1] = rng.uniform(-1.0, 1.0, (pb.N - 2, pb.N - 2))
    return u


def term_scale(pb, u):
    return np.max(np.abs(pb.f)) + 4 * (pb.a + pb.b) / pb.h * np.max(np.abs(u)) + 8 * pb.eps / pb.h**2 * np.max(
        np.abs(u))


@pytest.mark.parametrize("N", [5, 17, 33, 50, 65, 130])
@pytest.mark.parametrize("kappa", [0.0, 1.0 / 3.0, -1.0, 1.0])
@pytest.mark.parametrize("b", [0.0, 0.5])
def test_residual_matches_oracle(N, kappa, b):
    pb = cd.CDProblem(N, a=1.0, b=b, eps=1e-6, kappa=kappa)
    us = [start(pb, N + s) for s in range(3)]
    p = ops.cd_params(N, a=pb.a, b=b, eps=pb.eps, kappa=kappa)
    u = to_dev(us)
    f = to_dev([pb.f] * 3)
    r, rmax = ops.cd_residual(p, u, f)
    r, rmax = r.cpu().numpy(), rmax.cpu().numpy()
    for k in range(3):
        ref = cd.residual(pb, us[k])  # [N-2, N-2] x first
        tol = 1e-13 * term_scale(pb, us[k])
        assert np.max(np.abs(r[k][1:-1, 1:-1] - ref.T)) <= tol
        assert np.all(r[k][0, :] == 0) and np.all(r[k][-1, :] == 0) and np.all(r[k][:, 0] == 0)
        assert abs(rmax[k] - np.max(np.abs(ref))) <= tol


@pytest.mark.parametrize("N", [17, 50, 65])
@pytest.mark.parametrize("kappa", [0.0, 1.0 / 3.0, -1.0])
@pytest.mark.parametrize("splitting", ["Ls0", "Ls1"])
@pytest.mark.parametrize("order", ORDERS)
def test_relaxation_matches_oracle(N, kappa, splitting, order):
    pb = cd.CDProblem(N, kappa=kappa)
    sweeps = 6
    u0 = [pb.initial(), start(pb, 7)]
    refs = [cd.line_relaxation(pb, splitting, order=order, sweeps=sweeps, u0=u) for u in u0]
    p = ops.cd_params(N, kappa=kappa, splitting=splitting, order=order)
    u = to_dev(u0)
    f = to_dev([pb.f] * 2)
    hist, info = ops.cd_relax(p, u, f, sweeps)
    torch.cuda.synchronize()
    u, hist, info = u.cpu().numpy(), hist.cpu().numpy(), info.cpu().numpy()
    assert np.all(info == 0)
    for k, (ur, hr) in enumerate(refs):
        assert np.max(np.abs(u[k] - ur.T)) <= 1e-11 * np.max(np.abs(ur))
        # boundary untouched
        assert np.array_equal(u[k][0, :], u0[k].T[0, :]) and np.array_equal(u[k][:, -1], u0[k].T[:, -1])
        assert np.allclose(hist[:, k], hr[1:], rtol=1e-6, atol=1e-11 * hr[0])


def test_relaxation_converges_to_the_discrete_solution():
    pb = cd.CDProblem(33, kappa=1.0 / 3.0, eps=1e-3)
    ud = cd.solve_direct(pb)
    p = ops.cd_params(33, kappa=1.0 / 3.0, eps=1e-3, splitting="Ls1")
    u = to_dev([pb.initial()])
    hist, info = ops.cd_relax(p, u, to_dev([pb.f]), 60)
    torch.cuda.synchronize()
    assert hist.cpu().numpy()[-1, 0] <= 1e-11
    assert np.max(np.abs(u.cpu().numpy()[0] - ud.T)) <= 1e-11 * np.max(np.abs(ud))


def test_zero_sweeps_and_argument_checks():
    N = 17
    pb = cd.CDProblem(N)
    p = ops.cd_params(N)
    u = to_dev([start(pb, 1)])
    before = u.clone()
    f = to_dev([pb.f])
    hist, info = ops.cd_relax(p, u, f, 0)
    torch.cuda.synchronize()
    assert torch.equal(u, before) and int(info.cpu()[0]) == 0
    bad = ops.cd_params(N, a=-1.0)
    with pytest.raises(_ffi.EhlError):
        ops.cd_residual(bad, u, f)
    with pytest.raises(_ffi.EhlError):
        ops.cd_relax(ops.cd_params(N, kappa=1.5), u, f, 1)
    # a caller workspace one byte short is refused
    need = ops.cd_workspace_size(p, 1)
    ws = torch.empty(need - 1, dtype=torch.uint8, device="cuda")
    with pytest.raises(_ffi.EhlError):
        ops.cd_relax(p, u, f, 1, workspace=ws)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    ops.cd_relax(p, u, f, 1, workspace=ws)


def test_full_size_all_lines_against_the_oracle():
    """n = 1025 (1023 x-lines per sweep, the size the bench times), kappa = 0, Ls0."""
    N = 1025
    pb = cd.CDProblem(N, kappa=0.0)
    ur, hr = cd.line_relaxation(pb, "Ls0", order="jacobi", sweeps=3)
    p = ops.cd_params(N, kappa=0.0, splitting="Ls0", order="jacobi")
    u = to_dev([pb.initial()])
    hist, info = ops.cd_relax(p, u, to_dev([pb.f]), 3)
    torch.cuda.synchronize()
    assert int(info.cpu()[0]) == 0
    assert np.max(np.abs(u.cpu().numpy()[0] - ur.T)) <= 1e-11 * np.max(np.abs(ur))
    assert np.allclose(hist.cpu().numpy()[:, 0], hr[1:], rtol=1e-6, atol=1e-11 * hr[0])
