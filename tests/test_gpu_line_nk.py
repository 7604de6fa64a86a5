"""GPU parity of the Newton-Krylov line-contact solve (method 1) with the oracle.

Both solve the same discrete complementarity problem with force balance; the
oracle by dense semismooth Newton with LU, the GPU by PAQIF-preconditioned
GMRES.  Converged P and H0 must agree to 1e-8 relative.  Each GPU solve is run
to a residual a little above its float64 rounding floor (which grows with
eps/h^2 at fine grids and high loads).
"""
import time

import numpy as np
import pytest
import torch

from oracle import line_ref as lr
from paper_2008_03276_gb300 import inputs, ops

pytestmark = pytest.mark.gpu


def gpu_solve(N, M, L, limiter, beta, tol, n_inst=1, per=None, max_iter=60, krylov_dim=40, levels=-1, rough=None):
    kw = dict(limiter=limiter, halfband=beta, method=1, tol=tol, max_iter=max_iter, krylov_dim=krylov_dim,
              levels=levels)
    p = ops.default_params(1, nx=N, M=M, L=L, **kw)
    per_inst = None
    if per is not None:
        per_inst = [ops.default_params(1, nx=N, **kw, **d) for d in per]
    ctx = ops.Context(p, n_inst=n_inst, per_inst=per_inst)
    rd = None if rough is None else torch.tensor(np.asarray(rough, dtype=np.float64).reshape(n_inst, N), device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    P, H0, iters, res, code = ctx.solve(rough=rd, check=False)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return P.cpu().numpy(), H0.cpu().numpy(), iters.cpu().numpy(), res.cpu().numpy(), code, dt


def check(P, H0, pb, Pr, H0r):
    assert P[0] == 0 and P[-1] == 0
    assert np.max(np.abs(P[1:-1] - Pr)) <= 1e-8 * np.max(Pr)
    assert abs(H0 - H0r) <= 1e-8 * abs(H0r)
    H, Hr = pb.film(P[1:-1], H0), pb.film(Pr, H0r)
    assert np.max(np.abs(H - Hr)) <= 1e-8 * np.max(np.abs(Hr))


@pytest.mark.parametrize("levels", [0, -1])
@pytest.mark.parametrize("beta", [2, 4, 8])
def test_c1_newton_krylov(beta, levels):
    pb = lr.LineProblem(129, 20.0, 10.0, limiter="minmod")
    Pr, H0r, info = lr.solve(pb)
    assert info["converged"]
    P, H0, iters, res, code, dt = gpu_solve(129, 20.0, 10.0, 0, beta, tol=1e-11, levels=levels)
    print(f"beta {beta} levels {levels}: {iters[0]} Newton steps, {dt * 1e3:.1f} ms, res {res[0]}")
    assert code == 0 and iters[0] < 30
    check(P[0], H0[0], pb, Pr, H0r)


@pytest.mark.slow
def test_high_load_newton_krylov():
    N, M = 1025, 200.0
    pb = lr.LineProblem(N, M, 10.0, limiter="vanleer")
    Pr, H0r, info = lr.solve(pb)
    assert info["converged"]
    P, H0, iters, res, code, dt = gpu_solve(N, M, 10.0, 1, 8, tol=3e-10)
    print(f"N {N} M {M}: {iters[0]} Newton steps, {dt * 1e3:.1f} ms, res {res[0]}")
    assert code == 0 and iters[0] < 40
    check(P[0], H0[0], pb, Pr, H0r)


def test_batch_of_loads_newton_krylov():
    per = [dict(M=10.0, L=5.0), dict(M=50.0, L=10.0), dict(M=150.0, L=15.0), dict(M=400.0, L=8.0)]
    P, H0, iters, res, code, dt = gpu_solve(257, 20.0, 10.0, 0, 4, tol=1e-10, n_inst=4, per=per)
    print(f"batch of 4: iters {iters.tolist()}, {dt * 1e3:.1f} ms")
    assert code == 0
    for k, d in enumerate(per):
        pb = lr.LineProblem(257, d["M"], d["L"], limiter="minmod")
        Pr, H0r, info = lr.solve(pb)
        assert info["converged"]
        check(P[k], H0[k], pb, Pr, H0r)


@pytest.mark.parametrize("rough", [False, True])
def test_nested_iteration_low_load_van_leer(rough):
    """Low load, strong piezoviscosity, van Leer: Newton from the Hertzian start on the
    target grid stalls (oracle and GPU alike); the grid sequence 65-129-257 converges."""
    M, L, N = 10.068856862228834, 19.478471312560632, 257
    X = np.linspace(-4.5, 1.5, N)
    rgh = inputs.sin_grf_roughness(X, seed=11, amp=0.02, wavelength=0.4, sigma=0.01) if rough else np.zeros(N)
    pb, Pr, H0r, info = lr.solve_nested(
        lambda n: lr.LineProblem(n, M, L, limiter="vanleer", rough=lr.inject(rgh, n)), N, tol=1e-11)
    assert info["converged"], info["levels"]
    P, H0, iters, res, code, dt = gpu_solve(N, M, L, 1, 8, tol=1e-10, rough=rgh if rough else None)
    print(f"nested: {iters[0]} Newton steps on the target grid, {dt * 1e3:.1f} ms, res {res[0]}; "
          f"oracle levels {info['levels']}")
    assert code == 0 and iters[0] < 20
    check(P[0], H0[0], pb, Pr, H0r)


@pytest.mark.parametrize("precision", [1, 2, 3])
def test_mixed_precision_krylov_products(precision):
    """Krylov products as a float32-output GEMM (1 float32, 2 float32 on BF16 tensor cores, 3 TF32):
    the residual stays float64, so the converged solution matches the oracle as tightly."""
    N, M, L = 513, 200.0, 10.0
    pb = lr.LineProblem(N, M, L, limiter="vanleer")
    Pr, H0r, info = lr.solve(pb)
    assert info["converged"]
    per = [dict(M=M, L=L)] * 4
    kw = dict(limiter=1, halfband=8, method=1, tol=1e-10, max_iter=60, krylov_dim=40, precision=precision)
    p = ops.default_params(1, nx=N, M=M, L=L, **kw)
    ctx = ops.Context(p, n_inst=4, per_inst=[ops.default_params(1, nx=N, **kw, **d) for d in per])
    P, H0, iters, res, code = ctx.solve(check=False)
    assert code == 0, (code, iters.tolist())
    P, H0 = P.cpu().numpy(), H0.cpu().numpy()
    for k in range(4):
        check(P[k], H0[k], pb, Pr, H0r)
