"""Pins of the banded-solve / LCP oracle against things outside itself.

* dense LU on the expanded band vs scipy's LAPACK banded solver (gbsv), an
  independent factorization that reads the band in its own layout;
* a hand-checked 4x4 tridiagonal system (tests/golden/tridiag4.txt);
* PGS vs brute-force support enumeration (P-matrix: unique LCP solution);
* closed-form LCP special cases (A = I, b <= 0);
* complementarity conditions checked directly.
"""
import os

import numpy as np
import pytest
import scipy.linalg

from oracle import paqif_ref as pr
from paper_2008_03276_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def to_lapack_ab(band, beta):
    """Row-major band[i, j] = A[i, i-beta+j]  ->  LAPACK ab[beta + i - c, c] = A[i, c]."""
    n = band.shape[0]
    ab = np.zeros((2 * beta + 1, n))
    for i in range(n):
        for j in range(2 * beta + 1):
            c = i - beta + j
            if 0 <= c < n:
                ab[beta + i - c, c] = band[i, j]
    return ab


@pytest.mark.parametrize("n,beta", [(7, 1), (16, 2), (33, 4), (64, 8)])
def test_dense_lu_matches_lapack_banded(n, beta):
    band, rhs = inputs.dd_band_systems(3, n, beta, seed=n + beta)
    for s in range(3):
        A = pr.band_to_dense(band[s], beta)
        x = pr.solve_dense(A, rhs[s])
        xb = scipy.linalg.solve_banded((beta, beta), to_lapack_ab(band[s], beta), rhs[s])
        assert np.max(np.abs(x - xb)) <= 1e-13 * max(1.0, np.max(np.abs(xb)))
        assert np.max(np.abs(A @ x - rhs[s])) <= 1e-13


def test_golden_tridiagonal():
    # A = tridiag(-1, 4, -1), x = (1, 2, 3, 4) -> b = (2, 4, 6, 13); solved by hand.
    data = np.loadtxt(os.path.join(GOLDEN, "tridiag4.txt"))
    band = data[:, :3]
    b = data[:, 3]
    x_expected = data[:, 4]
    x = pr.paqif_reference(band[None], b[None], 1, mode=0)[0]
    assert np.allclose(x, x_expected, rtol=0, atol=1e-14)


def test_band_layout_ignores_outside_entries():
    band = np.full((5, 5), 7.0)  # beta = 2, every entry 7
    A = pr.band_to_dense(band, 2)
    assert A[0, 0] == 7.0 and A[0, 2] == 7.0 and A[0, 3] == 0.0
    assert np.count_nonzero(A) == 5 + 2 * 4 + 2 * 3


def test_mode1_is_projection():
    band, rhs = inputs.dd_band_systems(4, 20, 2, seed=5)
    x0 = pr.paqif_reference(band, rhs, 2, mode=0)
    x1 = pr.paqif_reference(band, rhs, 2, mode=1)
    assert np.array_equal(x1, np.maximum(x0, 0.0))
    assert np.any(x0 < 0)


def test_active_rows_pin_zero():
    band, rhs = inputs.dd_band_systems(2, 12, 2, seed=6)
    act = np.zeros((2, 12), dtype=np.uint8)
    act[0, [0, 5, 11]] = 1
    act[1, 3] = 1
    x = pr.paqif_reference(band, rhs, 2, mode=0, active=act)
    assert np.all(x[act.astype(bool)] == 0.0)
    # the remaining rows satisfy their equations exactly
    for s in range(2):
        A = pr.band_to_dense(band[s], 2)
        r = A @ x[s] - rhs[s]
        assert np.max(np.abs(r[~act[s].astype(bool)])) < 1e-13


@pytest.mark.parametrize("n", [1, 2, 5, 9, 12])
def test_lcp_pgs_matches_enumeration(n):
    beta = 2
    band, rhs = inputs.dd_band_systems(5, n, beta, seed=100 + n)
    for s in range(5):
        A = pr.band_to_dense(band[s], beta)
        sols = pr.lcp_enumerate(A, rhs[s])
        assert len(sols) == 1, "strictly diagonally dominant => P-matrix => unique"
        x, _ = pr.lcp_pgs(A, rhs[s], tol=1e-15)
        assert np.max(np.abs(x - sols[0])) <= 1e-12
        w = A @ x - rhs[s]
        assert np.all(x >= 0) and np.all(w >= -1e-12) and abs(x @ w) <= 1e-12


def test_lcp_closed_forms():
    rng = np.random.default_rng(0)
    b = rng.uniform(-1, 1, 10)
    x, _ = pr.lcp_pgs(np.eye(10), b)
    assert np.array_equal(x, np.maximum(b, 0.0))
    band, _ = inputs.dd_band_systems(1, 10, 2, seed=1)
    A = pr.band_to_dense(band[0], 2)
    x, _ = pr.lcp_pgs(A, -np.abs(b))
    assert np.all(x == 0.0)


def test_planted_mistake_is_caught():
    """A transposed band (a plausible layout slip) must fail the LAPACK pin."""
    band, rhs = inputs.dd_band_systems(1, 16, 2, seed=3)
    A = pr.band_to_dense(band[0], 2).T
    x = pr.solve_dense(A, rhs[0])
    xb = scipy.linalg.solve_banded((2, 2), to_lapack_ab(band[0], 2), rhs[0])
    assert np.max(np.abs(x - xb)) > 1e-6
