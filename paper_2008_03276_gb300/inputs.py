"""Seeded synthetic inputs shared by the tests, the bench and the smoke check.

This module holds no arithmetic of the method: it only draws random numbers
and builds parameter sets.  Both the CUDA path and the oracle receive the
arrays it returns.
"""
import numpy as np


def dd_band_systems(n_sys, n, beta, seed=0, dominance=1.5):
    """Strictly diagonally dominant banded systems in the row-major band layout.

    ``band[s, i, j] = A_s[i, i - beta + j]``: off-diagonals ``U(-1, 1)``
    (entries whose column falls outside the matrix are zero), diagonal
    ``dominance`` times the row's absolute off-diagonal sum (at least 1e-3 so
    rows with no off-diagonal stay nonsingular), rhs ``U(-1, 1)``.  PCG64.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    band = rng.uniform(-1.0, 1.0, size=(n_sys, n, 2 * beta + 1))
    rhs = rng.uniform(-1.0, 1.0, size=(n_sys, n))
    cols = np.arange(n)[:, None] - beta + np.arange(2 * beta + 1)[None, :]
    outside = (cols < 0) | (cols >= n)
    band[:, outside] = 0.0
    band[:, :, beta] = 0.0
    off = np.abs(band).sum(axis=2)
    band[:, :, beta] = np.maximum(dominance * off, 1e-3)
    return band, rhs


def sin_grf_roughness(X, seed, amp=0.1, wavelength=0.25, sigma=0.05, corr=0.1, jitter=1e-12):
    """Roughness ``amp sin(2 pi X / wavelength)`` plus a Gaussian random field.

    The field has covariance ``sigma^2 exp(-d^2 / corr^2)`` on the grid and is
    sampled by a Cholesky factor of that covariance (plus ``jitter`` on the
    diagonal).  PCG64 with the given seed.
    """
    X = np.asarray(X, dtype=np.float64)
    d = X[:, None] - X[None, :]
    C = sigma**2 * np.exp(-(d / corr) ** 2) + jitter * np.eye(len(X))
    Lc = np.linalg.cholesky(C)
    rng = np.random.Generator(np.random.PCG64(seed))
    return amp * np.sin(2.0 * np.pi * X / wavelength) + Lc @ rng.standard_normal(len(X))


def batched_line_params(n_inst, seed=1, sizes=(257, 513, 1025, 2049)):
    """Instance parameters of the batched line-contact workload.

    ``M`` log-uniform on [10, 1000], ``L`` uniform on [5, 20], ``N`` uniform on
    ``sizes``.  Returns a list of dicts.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    M = 10.0 ** rng.uniform(1.0, 3.0, n_inst)
    L = rng.uniform(5.0, 20.0, n_inst)
    N = rng.choice(np.asarray(sizes), n_inst)
    return [dict(M=float(M[k]), L=float(L[k]), N=int(N[k])) for k in range(n_inst)]
