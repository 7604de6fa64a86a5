"""The hand-written tcgen05 tensor-core product of the Krylov vectors (precision = 5).

The Krylov products of the line-contact Newton-Krylov method need the deformation K v of every
instance's vector (Sec. 3.3.1: the film's change; K the Toeplitz matrix of the closed-form
kernel).  precision = 5 computes it for a whole grid-size batch as one TF32x3 GEMM on the
tensor cores (K and the vectors split into tf32 hi + lo parts, three tcgen05.mma products,
float32 accumulation).  Checked through ehl_jacobian_apply against the oracle's exact Jacobian
(1e-5 of the row's |J| |v| scale: the product's relative error is about 2^-21 per term plus the
float32 accumulation over N terms), on grids with partial tiles in both dimensions, batches
that span several column tiles, and K-splits; then a full solve against the float64 path.
"""
import numpy as np
import pytest
import torch

from oracle import line_ref as lr
from paper_2008_03276_gb300 import ops

pytestmark = pytest.mark.gpu


def to_dev(*arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


@pytest.mark.parametrize("N,n_inst", [(129, 3), (257, 130), (1025, 200), (2049, 5)])
def test_product_matches_the_exact_jacobian(N, n_inst):
    M, L = 50.0, 10.0
    pb = lr.LineProblem(N, M, L, limiter="vanleer")
    rng = np.random.default_rng(N + n_inst)
    P = pb.hertz() * (1 + 0.05 * rng.standard_normal(pb.n)).clip(0)
    H0 = pb.h0_for_min_film(P, 0.1)
    J, JH = lr.jacobian_exact(pb, P, H0)
    p = ops.default_params(1, nx=N, M=M, L=L, limiter=1, halfband=2, method=1, precision=5)
    ctx = ops.Context(p, n_inst=n_inst)
    V = rng.standard_normal((n_inst, pb.n))
    vh = rng.standard_normal(n_inst)
    Pn = np.tile(pb.full(P), (n_inst, 1))
    Vn = np.zeros((n_inst, N))
    Vn[:, 1:-1] = V
    Pd, H0d, Vd, vhd = to_dev(Pn, np.full(n_inst, H0), Vn, vh)
    out = ctx.jacobian_apply(Pd, H0d, Vd, vhd).cpu().numpy()
    for k in range(n_inst):
        ref = J @ V[k] + JH * vh[k]
        scale = np.abs(J) @ np.abs(V[k]) + np.abs(JH) * abs(vh[k])
        err = np.abs(out[k, 1:-1] - ref) / scale
        assert np.max(err) <= 1e-5, (k, np.max(err))


def test_solve_with_the_tensor_core_products():
    """The high-load batch (N = 1025, M = 200, van Leer, beta 8) with the tcgen05 Krylov products
    and the device-driven loop: converged, H within 1e-6 of the float64 path."""
    B = 64
    base = dict(nx=1025, M=200.0, L=10.0, limiter=1, halfband=8, method=1, tol=1e-8, max_iter=60, krylov_dim=40,
                graph=2)
    c5 = ops.Context(ops.default_params(1, precision=5, **base), n_inst=B)
    c0 = ops.Context(ops.default_params(1, precision=0, **base), n_inst=B)
    P5, H05, it5, r5, code5 = c5.solve(check=False)
    P0, H00, it0, r0, code0 = c0.solve(check=False)
    assert code5 == 0 and code0 == 0
    assert float(r5.abs().max()) <= 1e-8
    _, H5, _ = c5.residual(P5, H05)
    _, H0v, _ = c0.residual(P0, H00)
    assert float((H5 - H0v).abs().max() / H0v.abs().max()) <= 1e-6
