"""GPU parity of the partitioned PAQIF (ehl_paqif_solve_partitioned, through the C ABI).

With the projection applied after the full solve, every admissible partition
count r computes A^{-1} b (mode 0), its projection (mode 1) or the LCP
solution (mode 2) up to rounding, so the reference is the same float64 oracle
as for one block per system, at the same tolerance.  The cases put blocks of
every size class on the systems (one interior level up to hundreds), the
reduced system at its smallest (r = 2) and largest (r = groups per CTA), odd n
with the padding row in the last block, and active rows next to block
boundaries.
"""
import numpy as np
import pytest
import torch

from oracle import paqif_ref as pr
from paper_2008_03276_gb300 import inputs, ops

pytestmark = pytest.mark.gpu
TOL = 1e-12
GPC = {1: 32, 2: 20, 3: 16, 4: 12, 5: 8, 6: 8, 7: 8, 8: 8}  # lane groups per CTA


def admissible(beta, n, r):
    npart = 2 * ((n + 2 * r - 1) // (2 * r))
    return GPC[beta] % r == 0 and (r == 1 or (npart >= 2 * beta + 2 and (r - 1) * npart < n))


def parts_for(beta, n):
    rs = [r for r in range(2, GPC[beta] + 1) if admissible(beta, n, r)]
    return sorted(set([rs[0], rs[len(rs) // 2], rs[-1]])) if rs else []


def run(band, rhs, beta, mode, parts, active=None):
    dev = torch.device("cuda")
    b = torch.from_numpy(band).to(dev)
    r = torch.from_numpy(rhs).to(dev)
    a = None if active is None else torch.from_numpy(active.astype(np.uint8)).to(dev)
    x, iters, info = ops.paqif_solve(b, r, beta, mode, active=a, partitions=parts)
    torch.cuda.synchronize()
    return x.cpu().numpy(), iters.cpu().numpy(), info.cpu().numpy()


def relerr(x, ref):
    return np.max(np.abs(x - ref), axis=-1) / np.maximum(np.max(np.abs(ref), axis=-1), 1e-300)


@pytest.mark.parametrize("beta", [1, 2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("n", [40, 101, 257, 1024])
def test_partitioned_mode0_matches_dense_lu(n, beta):
    rs = parts_for(beta, n)
    assert rs, "every case has an admissible partition count"
    band, rhs = inputs.dd_band_systems(7, n, beta, seed=7000 + 100 * beta + n)
    ref = pr.paqif_reference(band, rhs, beta, 0)
    for r in rs:
        x, iters, info = run(band, rhs, beta, 0, r)
        assert np.all(info == 0), (r, info.tolist())
        assert np.all(iters == 1)
        assert np.max(relerr(x, ref)) <= TOL, r


@pytest.mark.parametrize("beta", [2, 4, 8])
def test_partitioned_mode1_projects_after_the_solve(beta):
    """Steps 5 and 7 deferred: the result is max(0, A^{-1} b), as with one block."""
    n = 300
    band, rhs = inputs.dd_band_systems(9, n, beta, seed=71 + beta)
    ref = pr.paqif_reference(band, rhs, beta, 1)
    x1, _, _ = run(band, rhs, beta, 1, 1)
    for r in parts_for(beta, n):
        x, _, info = run(band, rhs, beta, 1, r)
        assert np.all(info == 0)
        assert np.all(x >= 0)
        assert np.max(np.abs(x - ref)) <= TOL * np.max(np.abs(ref))
        assert np.max(np.abs(x - x1)) <= TOL * np.max(np.abs(ref))


@pytest.mark.parametrize("beta", [1, 4, 8])
def test_partitioned_mode2_lcp(beta):
    n = 200
    band, rhs = inputs.dd_band_systems(5, n, beta, seed=90 + beta)
    ref = pr.paqif_reference(band, rhs, beta, 2)
    for r in parts_for(beta, n):
        x, iters, info = run(band, rhs, beta, 2, r)
        assert np.all(info == 0) and np.all(iters >= 1) and np.all(iters < 64)
        assert np.max(np.abs(x - ref)) <= TOL * np.max(np.abs(ref)), r
        for s in range(5):
            A = pr.band_to_dense(band[s], beta)
            w = A @ x[s] - rhs[s]
            assert np.all(x[s] >= 0) and np.all(w >= -1e-12) and abs(x[s] @ w) <= 1e-11


@pytest.mark.parametrize("beta", [3, 8])
def test_partitioned_active_rows_at_block_boundaries(beta):
    n = 257
    band, rhs = inputs.dd_band_systems(6, n, beta, seed=13 + beta)
    rng = np.random.default_rng(beta)
    for r in parts_for(beta, n):
        npart = 2 * ((n + 2 * r - 1) // (2 * r))
        act = rng.random((6, n)) < 0.1
        for m in range(1, r):  # rows on both sides of every block boundary
            for d in (-2, -1, 0, 1):
                if 0 <= m * npart + d < n:
                    act[m % 6, m * npart + d] = True
        x, _, info = run(band, rhs, beta, 0, r, active=act)
        ref = pr.paqif_reference(band, rhs, beta, 0, active=act)
        assert np.all(info == 0)
        assert np.all(x[act] == 0.0)
        assert np.max(relerr(x, ref)) <= TOL, r


def test_partitioned_nonfinite_is_reported_per_system():
    beta, n = 2, 120
    band, rhs = inputs.dd_band_systems(3, n, beta, seed=5)
    rhs[1, 70] = np.nan  # inside the third of four blocks (rows 60..89)
    x, _, info = run(band, rhs, beta, 0, 4)
    assert info[0] == ops.INFO_OK and info[2] == ops.INFO_OK
    assert info[1] == ops.INFO_NONFINITE


def test_partitioned_full_size_standalone_batch():
    """The standalone workload (4096 x n = 1024, beta 4, mode 1) with two and four
    blocks per system, checked on sampled systems against the oracle."""
    beta, n, n_sys = 4, 1024, 4096
    band, rhs = inputs.dd_band_systems(n_sys, n, beta, seed=2024)
    pick = np.array([0, 1, 977, 2048, 4095])
    ref = pr.paqif_reference(band[pick], rhs[pick], beta, 1)
    for r in (2, 4):
        x, _, info = run(band, rhs, beta, 1, r)
        assert np.all(info == 0)
        assert np.max(np.abs(x[pick] - ref)) <= TOL * np.max(np.abs(ref))


@pytest.mark.parametrize("beta,r", [(2, 4), (4, 3), (8, 2)])
def test_partitioned_matches_the_stepwise_oracle(beta, r):
    """Against the dense walk-through of Sec. 2.2.4 Steps 1-7 (oracle/aqif_ref.py) on blocks of
    the same order as the kernel's (n divisible by 2r)."""
    from oracle import aqif_ref as aq

    n = 2 * r * 24
    band, rhs = inputs.dd_band_systems(3, n, beta, seed=31 + beta)
    x, _, info = run(band, rhs, beta, 1, r)
    assert np.all(info == 0)
    for s in range(3):
        A = pr.band_to_dense(band[s], beta)
        ref = aq.paqif_partitioned(A, rhs[s], beta, r, mode=1)
        assert np.max(np.abs(x[s] - ref)) <= TOL * np.max(np.abs(ref))
