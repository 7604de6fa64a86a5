"""The seeded input generators follow the stated recipes (CPU).

Band systems: row-major band ``band[s, i, j] = A_s[i, i - beta + j]``, zero outside the
matrix, off-diagonals U(-1, 1), diagonal 1.5 x the row's absolute off-diagonal sum within the
matrix, rhs U(-1, 1).  Roughness: a sine of the given wavelength plus a Gaussian field of
covariance sigma^2 exp(-d^2 / corr^2).  Batched line parameters: M log-uniform on [10, 1000],
L uniform on [5, 20], N from the listed sizes.  Every generator is reproducible from its seed.
"""
import numpy as np

from oracle import paqif_ref as pr
from paper_2008_03276_gb300 import inputs


def test_band_systems_layout_and_dominance():
    n, beta = 23, 3
    band, rhs = inputs.dd_band_systems(4, n, beta, seed=7)
    assert band.shape == (4, n, 2 * beta + 1) and rhs.shape == (4, n)
    b2, r2 = inputs.dd_band_systems(4, n, beta, seed=7)
    assert np.array_equal(band, b2) and np.array_equal(rhs, r2)
    assert not np.array_equal(band, inputs.dd_band_systems(4, n, beta, seed=8)[0])
    for s in range(4):
        A = pr.band_to_dense(band[s], beta)
        off = np.abs(A).sum(axis=1) - np.abs(np.diag(A))
        assert np.allclose(np.diag(A), 1.5 * off)
        # entries beyond the matrix edge are zero in the band, entries beyond the band zero in A
        for i in range(n):
            for j in range(2 * beta + 1):
                c = i - beta + j
                if c < 0 or c >= n:
                    assert band[s, i, j] == 0.0
                else:
                    assert A[i, c] == band[s, i, j]
        ii, jj = np.indices(A.shape)
        assert np.all(A[np.abs(ii - jj) > beta] == 0.0)
    offd = band[:, :, [j for j in range(2 * beta + 1) if j != beta]]
    assert np.all(np.abs(offd) < 1.0) and np.all(np.abs(rhs) < 1.0)
    assert np.all(band[:, :, beta] > 0.0)


def test_band_systems_of_order_one_stay_nonsingular():
    band, _ = inputs.dd_band_systems(3, 1, 2, seed=1)
    assert np.all(band[:, 0, 2] == 1e-3)
    assert np.all(np.delete(band[:, 0, :], 2, axis=1) == 0.0)


def test_roughness_is_sine_plus_a_field_of_the_stated_covariance():
    X = np.linspace(-1.0, 1.0, 21)
    sine = 0.1 * np.sin(2.0 * np.pi * X / 0.25)
    r0 = inputs.sin_grf_roughness(X, seed=3)
    assert np.array_equal(r0, inputs.sin_grf_roughness(X, seed=3))
    fields = np.stack([inputs.sin_grf_roughness(X, seed=s) - sine for s in range(2000)])
    d = X[:, None] - X[None, :]
    C = 0.05**2 * np.exp(-(d / 0.1) ** 2)
    emp = fields.T @ fields / len(fields)
    # sample covariance of 2000 draws: a few percent of sigma^2 off at most
    assert np.max(np.abs(emp - C)) <= 0.15 * 0.05**2
    assert np.max(np.abs(fields.mean(axis=0))) <= 0.2 * 0.05


def test_batched_line_parameters():
    per = inputs.batched_line_params(512, seed=1)
    assert per == inputs.batched_line_params(512, seed=1)
    M = np.array([q["M"] for q in per])
    L = np.array([q["L"] for q in per])
    N = np.array([q["N"] for q in per])
    assert np.all((M >= 10.0) & (M <= 1000.0)) and np.all((L >= 5.0) & (L <= 20.0))
    assert set(N.tolist()) == {257, 513, 1025, 2049}
    # log-uniform M: log10 M spreads evenly over [1, 3]
    q = np.histogram(np.log10(M), bins=4, range=(1.0, 3.0))[0]
    assert np.all(q > 0.15 * len(M))
