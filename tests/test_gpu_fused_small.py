"""One-CTA stages of small line-contact instances against the multi-kernel stages.

For an instance of at most 256 nodes the state evaluation (film from the float64 deformation
chunks, lubricant model, limited faces, residual and its reductions) runs in one CTA, and for
at most 257 nodes so does a Krylov step of the Newton-Krylov solve (preconditioned vector,
double-float deformation of the film derivative, exact directional derivative, Arnoldi step).
Both do the multi-kernel stages' operations in the same order.  The one-CTA state agrees with
the stage kernels (``EHL_FUSE=0``) bit for bit: residual, film and reductions, and so every
iterate of the paper's iteration, whose linear solve is PAQIF alone.  The one-CTA Krylov step,
the same operations compiled into one kernel, differs in the last bits (most likely products
contracted into FMAs differently), so Newton-Krylov solves are compared as two solves to the
same tolerance: the same Newton iteration counts, and
converged pressures and H0 within 1e-9 relative (measured on a GB300: at most 3.5e-11, against
the solve tolerance 1e-8).
"""
import os

import numpy as np
import pytest
import torch

from paper_2008_03276_gb300 import ops

pytestmark = pytest.mark.gpu


def _context(fuse, p, n_inst=1, per_inst=None):
    old = os.environ.get("EHL_FUSE")
    os.environ["EHL_FUSE"] = "1" if fuse else "0"
    try:
        return ops.Context(p, n_inst=n_inst, per_inst=per_inst)
    finally:
        if old is None:
            del os.environ["EHL_FUSE"]
        else:
            os.environ["EHL_FUSE"] = old


def _both(p, n_inst=1, per_inst=None, rough=None):
    out = []
    for fuse in (True, False):
        ctx = _context(fuse, p, n_inst, per_inst)
        n0 = ops.kernel_launches()
        P, H0, iters, res, code = ctx.solve(rough=rough, check=False)
        torch.cuda.synchronize()
        out.append((P.cpu().numpy(), H0.cpu().numpy(), iters.cpu().numpy(), int(code),
                    ops.kernel_launches() - n0))
    return out


@pytest.mark.parametrize("N", [65, 129, 256])
def test_residual_and_film_bitwise(N):
    p = ops.default_params(1, nx=N, M=20.0, L=10.0, limiter=1, halfband=2, method=1)
    X = np.linspace(-4.5, 1.5, N)
    P = torch.tensor(np.sqrt(np.clip(1.0 - X ** 2, 0.0, None))[None, :], device="cuda")
    P[:, 0] = 0.0
    P[:, -1] = 0.0
    H0 = torch.tensor([-0.3], dtype=torch.float64, device="cuda")
    rough = torch.tensor((0.01 * np.sin(2 * np.pi * X / 0.5))[None, :], device="cuda")
    res = []
    for fuse in (True, False):
        ctx = _context(fuse, p)
        R, H, comp = ctx.residual(P, H0, rough)
        res.append((R.cpu().numpy(), H.cpu().numpy(), comp.cpu().numpy()))
    np.testing.assert_array_equal(res[0][0], res[1][0])
    np.testing.assert_array_equal(res[0][1], res[1][1])
    np.testing.assert_array_equal(res[0][2], res[1][2])


def _close(Pf, Pu, Hf, Hu, rel=1e-9):
    for k in range(Pf.shape[0]):
        assert np.max(np.abs(Pf[k] - Pu[k])) <= rel * np.max(np.abs(Pu[k]))
    assert np.max(np.abs(Hf - Hu)) <= rel * np.max(np.abs(Hu))


@pytest.mark.parametrize("graph", [0, 2])
def test_c1_newton_krylov_matches_stage_kernels(graph):
    p = ops.default_params(1, nx=129, M=20.0, L=10.0, limiter=0, halfband=2, method=1, tol=1e-8, max_iter=60,
                           graph=graph)
    (Pf, Hf, itf, cf, lf), (Pu, Hu, itu, cu, lu) = _both(p)
    assert cf == 0 and cu == 0
    np.testing.assert_array_equal(itf, itu)
    _close(Pf, Pu, Hf, Hu)
    assert lf < lu  # fewer kernels for the same iterations


def test_c1_paper_iteration_bitwise():
    p = ops.default_params(1, nx=129, M=20.0, L=10.0, limiter=0, halfband=2, method=0, tol=1e-8, max_iter=4000,
                           levels=0, graph=2)
    (Pf, Hf, itf, cf, _), (Pu, Hu, itu, cu, _) = _both(p)
    assert cf == 0 and cu == 0
    np.testing.assert_array_equal(itf, itu)
    np.testing.assert_array_equal(Pf, Pu)
    np.testing.assert_array_equal(Hf, Hu)


def test_ragged_batch_with_roughness_matches_stage_kernels():
    """Grids of 129, 257 and 513 nodes in one context (the last runs the stage kernels either
    way, its coarse grids the one-CTA stages), van Leer, roughness."""
    per = [dict(nx=n, M=m) for n, m in ((129, 20.0), (257, 50.0), (513, 100.0), (257, 20.0))]
    base = dict(M=20.0, L=10.0, limiter=1, halfband=4, method=1, tol=1e-8, max_iter=60, graph=2)
    pp = [ops.default_params(1, **{**base, **d}) for d in per]
    p = ops.default_params(1, **{**base, "nx": 513})
    rough = np.zeros((4, 513))
    for k, q in enumerate(per):
        x = np.linspace(-4.5, 1.5, q["nx"])
        rough[k, :q["nx"]] = 0.01 * np.sin(2 * np.pi * x / 0.5)
    rt = torch.tensor(rough, device="cuda")
    (Pf, Hf, itf, cf, _), (Pu, Hu, itu, cu, _) = _both(p, n_inst=4, per_inst=pp, rough=rt)
    assert cf == 0 and cu == 0
    np.testing.assert_array_equal(itf, itu)
    _close(Pf, Pu, Hf, Hu)
