"""The partition-count autotuner (ehl_paqif_autotune, ehl_params.autotune).

Sec. 2.2.4 leaves the number r of blocks per system free; the library's rule picks it from the
batch shape, the autotuner times every admissible r on the GPU.  Checked: the returned r is
admissible and the fastest of the times it reports; the solve with it matches dense LU to
1e-12 like every other r; a line-contact context created with autotune = 1 converges to the
solution of one created without (1e-9 relative: the preconditioner's rounding differs).
"""
import numpy as np
import pytest
import torch

from oracle import paqif_ref as pr
from paper_2008_03276_gb300 import inputs, ops

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n_sys,n,beta", [(4096, 1024, 4), (512, 1023, 8), (255, 255, 2)])
def test_autotune_picks_the_fastest_admissible_r(n_sys, n, beta):
    band_h, rhs_h = inputs.dd_band_systems(n_sys, n, beta, seed=n_sys + n)
    band, rhs = torch.from_numpy(band_h).cuda(), torch.from_numpy(rhs_h).cuda()
    r, ms = ops.paqif_autotune(band, rhs, beta, mode=1, reps=3)
    assert ops.paqif_partitions(n_sys, n, beta, r) == r
    timed = [(k + 1, t) for k, t in enumerate(ms) if t >= 0]
    assert len(timed) >= 2
    assert ms[r - 1] == min(t for _, t in timed)
    print(f"{n_sys} x {n}, beta {beta}: r = {r}, auto = {ops.paqif_partitions(n_sys, n, beta, 0)}, "
          f"ms = {[(k, round(t, 4)) for k, t in timed]}")
    x, _, info = ops.paqif_solve(band, rhs, beta, 1, partitions=r)
    torch.cuda.synchronize()
    assert bool((info == 0).all())
    idx = [0, n_sys // 2, n_sys - 1]
    ref = pr.paqif_reference(band_h[idx], rhs_h[idx], beta, 1)
    assert np.max(np.abs(x.cpu().numpy()[idx] - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_context_with_autotuned_preconditioner():
    kw = dict(nx=1025, M=200.0, L=10.0, limiter=1, halfband=8, method=1, tol=1e-10, max_iter=60)
    c1 = ops.Context(ops.default_params(1, autotune=1, **kw), n_inst=64)
    c0 = ops.Context(ops.default_params(1, autotune=0, **kw), n_inst=64)
    P1, H1, it1, r1, code1 = c1.solve(check=False)
    P0, H0, it0, r0, code0 = c0.solve(check=False)
    assert code1 == 0 and code0 == 0
    assert float((P1 - P0).abs().max() / P0.abs().max()) <= 1e-9


def test_point_context_with_autotuned_xlines():
    """257^2 point contact (the bench's configuration) with the FFT deformation and the x-line
    partition count autotuned: converged, and the oracle's own residual at the solution is small."""
    from oracle import point_ref as ptr
    n = 257
    p = ops.default_params(2, nx=n, ny=n, M=100.0, L=10.0, limiter=0, halfband=2, method=1, tol=1e-8, max_iter=60,
                           coarse_min_nodes=33, deform=1, autotune=1)
    ctx = ops.Context(p)
    P, H0, iters, res, code = ctx.solve(check=False)
    assert code == 0
    Pn, H0n = P.cpu().numpy()[0], float(H0.cpu()[0])
    pb = ptr.PointProblem(n, n, 100.0, 10.0)
    Pint = Pn.T[1:-1, 1:-1].ravel()
    R = ptr.residual(pb, Pint, H0n)
    assert np.max(np.abs(np.minimum(Pint, R))) <= max(2e-8, ptr.rounding_floor(pb, Pint, H0n))
