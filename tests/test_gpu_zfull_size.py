"""GPU parity at the full sizes and in the launch configurations the bench times.

The dense oracle cannot solve every full-size workload, so each is checked on what the
oracle can compute there: sampled instances solved by the oracle (the high-load line batch),
or the oracle's residual evaluated at the GPU's solution together with invariants that hold at
any size (the ragged batch, point contact at 257^2).  These tests sit in a file of their own,
after the other GPU tests and before the allocation-free one, which runs last.
"""
import time

import numpy as np
import pytest
import torch

from oracle import line_ref as lr
from oracle import point_ref as pr
from paper_2008_03276_gb300 import inputs, ops

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def check_line(P, H0, pb, Pr, H0r):
    assert P[0] == 0 and P[-1] == 0
    assert np.max(np.abs(P[1:-1] - Pr)) <= 1e-8 * np.max(Pr)
    assert abs(H0 - H0r) <= 1e-8 * abs(H0r)
    H, Hr = pb.film(P[1:-1], H0), pb.film(Pr, H0r)
    assert np.max(np.abs(H - Hr)) <= 1e-8 * np.max(np.abs(Hr))


def test_high_load_batch_of_512_in_the_bench_configuration():
    """The bench's line batch (512 instances of N = 1025, M = 200, L = 10, van Leer, band 8,
    Krylov basis 40, the library's nested iteration and partition count for 512 systems),
    solved to 3e-10: sampled instances match the oracle, and the 512 identical problems,
    solved side by side, return the same solution."""
    N, M, L = 1025, 200.0, 10.0
    pb = lr.LineProblem(N, M, L, limiter="vanleer")
    Pr, H0r, info = lr.solve(pb)
    assert info["converged"]
    p = ops.default_params(1, nx=N, M=M, L=L, limiter=1, halfband=8, method=1, tol=3e-10, max_iter=60,
                           krylov_dim=40)
    ctx = ops.Context(p, n_inst=512)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    P, H0, iters, res, code = ctx.solve(check=False)
    torch.cuda.synchronize()
    it = iters.cpu().numpy()
    print(f"batch of 512: iters {it.min()}-{it.max()}, {(time.perf_counter() - t0) * 1e3:.1f} ms")
    assert code == 0
    P, H0 = P.cpu().numpy(), H0.cpu().numpy()
    for k in (0, 255, 511):
        check_line(P[k], H0[k], pb, Pr, H0r)
    assert np.max(np.abs(P - P[0])) <= 1e-12 * np.max(np.abs(P[0]))
    assert np.max(np.abs(H0 - H0[0])) <= 1e-12 * abs(H0[0])


def test_c3_full_batch_solutions_satisfy_the_oracles_problem():
    """C3 as the bench runs it (512 instances, N from {257, 513, 1025, 2049}, M log-uniform on
    [10, 1000], L on [5, 20], minmod, band 2, tol 1e-8): for the first and last instance of every
    grid size the oracle's residual at the GPU's solution meets the convergence test the bench
    counts (complementarity and force residual within 10 tol, or the rounding floor)."""
    per = inputs.batched_line_params(512, seed=1)
    kw = dict(limiter=0, halfband=2, method=1, tol=1e-8, max_iter=60, precision=0)
    pp = [ops.default_params(1, nx=q["N"], M=q["M"], L=q["L"], **kw) for q in per]
    ctx = ops.Context(pp[0], n_inst=len(pp), per_inst=pp)
    P, H0, iters, res, code = ctx.solve(check=False)
    assert code == 0, code
    P, H0 = P.cpu().numpy(), H0.cpu().numpy()
    picks = []
    for N in (257, 513, 1025, 2049):
        ks = [k for k, q in enumerate(per) if q["N"] == N]
        picks += [ks[0], ks[-1]]
    for k in picks:
        q = per[k]
        n = q["N"]
        pb = lr.LineProblem(n, q["M"], q["L"], limiter="minmod")
        assert P[k, 0] == 0.0 and P[k, n - 1] == 0.0 and np.all(P[k, n:] == 0.0)
        rc, g = lr.comp_residual(pb, P[k, 1:n - 1], H0[k])
        floor = lr.rounding_floor(pb, P[k, 1:n - 1], H0[k])
        assert rc <= max(1e-7, floor) and abs(g) <= 1e-7, (k, q, rc, g, floor)


def test_point_solve_257_in_the_bench_configuration():
    """C4 as the bench runs it (257^2, M = 100, L = 10, minmod, band 2, nested from 33^2,
    tol 1e-8, the library's Krylov basis): the oracle's residual at the GPU's solution, the
    force balance and the Y-mirror symmetry (the dense oracle does not reach this size)."""
    n = 257
    p = ops.default_params(2, nx=n, ny=n, M=100.0, L=10.0, limiter=0, halfband=2, method=1, tol=1e-8,
                           max_iter=60, coarse_min_nodes=33)
    ctx = ops.Context(p)
    P, H0, iters, res, code = ctx.solve(check=False)
    print(f"257^2: code {code} iters {iters.tolist()} res {res.tolist()}")
    assert code == 0
    Pn, H0n = P.cpu().numpy()[0], float(H0.cpu()[0])
    pb = pr.PointProblem(n, n, 100.0, 10.0, limiter="minmod")
    Pint = Pn.T[1:-1, 1:-1].ravel()
    R = pr.residual(pb, Pint, H0n)       # the oracle's residual at the GPU's solution
    assert np.max(np.abs(np.minimum(Pint, R))) <= 2e-8
    assert abs(pb.h**2 * Pint.sum() - 2 * np.pi / 3) <= 1e-8
    assert np.max(np.abs(Pn - Pn[::-1, :])) <= 1e-6 * np.max(Pn)       # Y -> -Y
