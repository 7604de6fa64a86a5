"""Edge cases of the EHL path on the GPU: the smallest grid, the largest line grid of the
high-load configuration, the rigid and isoviscous limit, rectangular point grids, a ragged
batch with one instance per grid size, and invalid arguments rejected before any launch."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import line_ref as lr
from oracle import point_ref as pr
from paper_2008_03276_gb300 import _ffi, ops

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def test_smallest_line_grid_residual_and_solve():
    N = 5  # three unknowns
    pb = lr.LineProblem(N, 20.0, 10.0)
    ctx = ops.Context(ops.default_params(1, nx=N, halfband=1, method=1, tol=1e-12, max_iter=60, levels=0))
    P = pb.hertz()
    H0 = pb.h0_for_min_film(P, 0.3)
    R, H, comp = ctx.residual(dev(pb.full(P)[None]), dev([H0]))
    s = lr.state(pb, P, H0)
    assert np.max(np.abs(H.cpu().numpy()[0] - s["H"])) <= 1e-13 * np.max(np.abs(s["H"]))
    assert np.max(np.abs(R.cpu().numpy()[0, 1:-1] - s["R"])) <= 1e-12 * max(1.0, np.max(np.abs(s["R"])))
    Pg, H0g, iters, res, code = ctx.solve(check=False)
    assert code in (0, _ffi.EHL_ENOCONV)           # a status, never a fault
    assert np.all(np.isfinite(Pg.cpu().numpy()))


def test_rigid_isoviscous_limit_matches_oracle():
    N = 257
    kw = dict(nx=N, M=2.0, L=0.0, compressible=0, elastic=0, halfband=2, method=1, tol=1e-11, max_iter=60)
    ctx = ops.Context(ops.default_params(1, **kw))
    P, H0, iters, res, code = ctx.solve(check=False)
    assert code == 0, (iters.tolist(), res.tolist())
    pb = lr.LineProblem(N, 2.0, 0.0, compressible=False, elastic=False)
    Pr, H0r, info = lr.solve(pb)
    assert info["converged"]
    P, H0 = P.cpu().numpy()[0], float(H0.cpu()[0])
    assert np.max(np.abs(P[1:-1] - Pr)) <= 1e-8 * np.max(Pr)
    assert abs(H0 - H0r) <= 1e-8 * abs(H0r)


@pytest.mark.slow
def test_high_load_line_4097_matches_oracle():
    """The largest line grid of the high-load configuration: N = 4097, M = 200, L = 10, van Leer."""
    N, M, L = 4097, 200.0, 10.0
    ctx = ops.Context(ops.default_params(1, nx=N, M=M, L=L, limiter=1, halfband=8, method=1, tol=1e-9, max_iter=80))
    P, H0, iters, res, code = ctx.solve(check=False)
    assert code == 0, (iters.tolist(), res.tolist())
    P, H0 = P.cpu().numpy()[0], float(H0.cpu()[0])
    pb, Pr, H0r, info = lr.solve_nested(lambda n: lr.LineProblem(n, M, L, limiter="vanleer"), N, n_min=513, tol=1e-9)
    assert info["converged"], info["levels"]
    assert np.max(np.abs(P[1:-1] - Pr)) <= 1e-8 * np.max(Pr)
    assert abs(H0 - H0r) <= 1e-8 * abs(H0r)


def test_rectangular_point_grid_residual_matches_oracle():
    nx, ny, h = 65, 33, 6.0 / 64
    ya = -0.5 * (ny - 1) * h
    pb = pr.PointProblem(nx, ny, 20.0, 10.0, ya=ya, limiter="vanleer")
    ctx = ops.Context(ops.default_params(2, nx=nx, ny=ny, ya=ya, yb=-ya, limiter=1, halfband=2, method=1))
    rng = np.random.default_rng(4)
    P = pb.hertz() * (1 + 0.05 * rng.standard_normal(pb.n)).clip(0)
    H0 = pb.h0_for_min_film(P, 0.1)
    R, H, comp = ctx.residual(dev(pb.full(P).T[None]), dev([H0]))
    s = pr.state(pb, P, H0)
    assert np.max(np.abs(H.cpu().numpy()[0] - s["H"].T)) <= 1e-13 * np.max(np.abs(s["H"]))
    Rr = s["R"]
    assert np.max(np.abs(R.cpu().numpy()[0, 1:-1, 1:-1] - Rr.T)) <= 1e-11 * max(1.0, np.max(np.abs(Rr)))


def test_ragged_batch_one_instance_per_grid():
    sizes = [129, 257, 65, 513]
    per = [ops.default_params(1, nx=n, M=20.0 + 10 * k, L=10.0, halfband=4, method=1, tol=1e-10, max_iter=60)
           for k, n in enumerate(sizes)]
    ctx = ops.Context(per[0], n_inst=len(per), per_inst=per)
    P, H0, iters, res, code = ctx.solve(check=False)
    assert code == 0
    P, H0 = P.cpu().numpy(), H0.cpu().numpy()
    for k, n in enumerate(sizes):
        pb = lr.LineProblem(n, 20.0 + 10 * k, 10.0)
        Pr, H0r, info = lr.solve(pb)
        assert info["converged"]
        assert np.max(np.abs(P[k, 1:n - 1] - Pr)) <= 1e-8 * np.max(Pr)
        assert np.all(P[k, n:] == 0.0)


def test_invalid_arguments_are_rejected():
    lib = _ffi.load()
    p = ops.default_params(1)
    q = ops.default_params(2)
    h = ctypes.c_void_p(0)
    arr = (_ffi.EhlParams * 2)(p, q)                       # mixed dimensions
    assert lib.ehl_create(ctypes.byref(p), 2, arr, None, ctypes.byref(h)) == _ffi.EHL_EINVAL
    q.ny = 77                                              # grid spacing differs in y
    assert lib.ehl_create(ctypes.byref(q), 1, None, None, ctypes.byref(h)) == _ffi.EHL_EINVAL
    ctx = ops.Context(ops.default_params(1, nx=65))
    P = torch.zeros((1, 65), dtype=torch.float64, device="cuda")
    H0 = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert lib.ehl_solve(ctx._h, ctypes.c_void_p(P.data_ptr()), ctypes.c_void_p(H0.data_ptr()), None, 7, None,
                         None) == _ffi.EHL_EINVAL
    with pytest.raises(ValueError):
        ctx.residual(torch.zeros((1, 64), dtype=torch.float64, device="cuda"), H0)
