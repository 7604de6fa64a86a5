"""GPU parity of factor once / resolve many (Sec. 2.2.1-2.2.3: W0 and Z0 do not depend on the
right-hand side) through the C ABI: ehl_paqif_factor solves for its rhs, ehl_paqif_resolve for
new ones with the stored factorization, both against dense LU (oracle) at the tolerance of the
PAQIF tests (1e-12 relative), on the partitioned and unpartitioned shapes, modes 0 and 1.
"""
import numpy as np
import pytest
import torch

from oracle import paqif_ref as pr
from paper_2008_03276_gb300 import _ffi, inputs, ops

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n_sys,n,beta", [(3, 37, 1), (5, 130, 2), (4, 257, 4), (2, 1025, 8), (64, 1023, 8)])
@pytest.mark.parametrize("mode", [0, 1])
def test_resolve_matches_dense_lu(n_sys, n, beta, mode):
    band, rhs = inputs.dd_band_systems(n_sys, n, beta, seed=n + beta)
    rng = np.random.default_rng(7)
    rhs2 = rng.uniform(-1, 1, rhs.shape)
    bd = torch.from_numpy(band).cuda()
    x1, info1, fac = ops.paqif_factor(bd, torch.from_numpy(rhs).cuda(), beta, mode)
    x2, info2 = ops.paqif_resolve(fac, torch.from_numpy(rhs2).cuda(), beta, mode)
    x3, info3 = ops.paqif_resolve(fac, torch.from_numpy(rhs).cuda(), beta, mode)  # the factor stays usable
    torch.cuda.synchronize()
    for xs, r, inf in ((x1, rhs, info1), (x2, rhs2, info2), (x3, rhs, info3)):
        assert int((inf != 0).sum()) == 0
        xs = xs.cpu().numpy()
        for s in range(n_sys):
            ref = pr.solve_dense(pr.band_to_dense(band[s], beta), r[s])
            if mode == 1:
                ref = np.maximum(ref, 0.0)
            assert np.max(np.abs(xs[s] - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))
    # the resolve kernel sums in another order than the factor kernel's sweeps: same tolerance
    assert float((x1 - x3).abs().max()) <= 1e-12 * max(1.0, float(x1.abs().max()))


def test_resolve_agrees_with_the_solve_entry():
    n_sys, n, beta = 16, 513, 4
    band, rhs = inputs.dd_band_systems(n_sys, n, beta, seed=3)
    bd, rd = torch.from_numpy(band).cuda(), torch.from_numpy(rhs).cuda()
    x0, _, _ = ops.paqif_solve(bd, rd, beta, 0)
    _, _, fac = ops.paqif_factor(bd, torch.zeros_like(rd), beta, 0)
    x1, _ = ops.paqif_resolve(fac, rd, beta, 0)
    assert torch.allclose(x0, x1, rtol=0, atol=1e-12 * float(x0.abs().max()))


def test_argument_checks():
    n_sys, n, beta = 2, 65, 2
    band, rhs = inputs.dd_band_systems(n_sys, n, beta, seed=1)
    bd, rd = torch.from_numpy(band).cuda(), torch.from_numpy(rhs).cuda()
    need = ops.paqif_factor_size(n_sys, n, beta)
    short = torch.empty(need - 1, dtype=torch.uint8, device="cuda")
    with pytest.raises(_ffi.EhlError):
        ops.paqif_factor(bd, rd, beta, 0, factor=short)
    with pytest.raises(_ffi.EhlError):
        ops.paqif_factor(bd, rd, beta, 2)  # no LCP loop on a stored factorization
    _, _, fac = ops.paqif_factor(bd, rd, beta, 0)
    with pytest.raises(_ffi.EhlError):
        ops.paqif_resolve(fac[1:], rd, beta, 0)  # misaligned and short
