"""Reference for the banded linear / complementarity solves (test infrastructure).

What PAQIF computes has a plain definition, so the oracle writes out that
definition instead of the factorization:

* mode 0  ``x = A^{-1} b``                         (Sec. 2.2.2, the solution of
  ``W0 Y = F``, ``Z0 U = Y`` is the solution of ``L0 U = F``);
* mode 1  ``x = max(0, A^{-1} b)``                 (Sec. 2.2.2 / Sec. 2.2.4
  Steps 5 and 7: project the computed solution onto ``U >= 0``, with one
  partition the projection follows the full solve);
* mode 2  the linear complementarity problem of Sec. 2.1 (Eq. eqn14 with
  ``L = A``, ``f = b``):  ``x >= 0``, ``w = A x - b >= 0``, ``x^T w = 0``.

Rows flagged in ``active`` are replaced by identity rows with zero right-hand
side, i.e. ``x_i = 0`` (the cavitated rows of the Newton step).

Band layout: ``band[i, j] = A[i, i - beta + j]`` for ``0 <= j <= 2 beta``;
entries whose column falls outside ``[0, n)`` are ignored.

Pins (tests/test_oracle_paqif.py): the dense LU result is checked by its
residual and against scipy's independent banded solver; the LCP solvers are
checked against each other (PGS vs enumeration) and against the three
complementarity conditions directly.
"""
import itertools

import numpy as np


def band_to_dense(band, beta):
    """Expand one row-major band ``[n, 2 beta + 1]`` to a dense ``[n, n]`` matrix."""
    band = np.asarray(band, dtype=np.float64)
    n = band.shape[0]
    A = np.zeros((n, n))
    for i in range(n):
        for j in range(2 * beta + 1):
            c = i - beta + j
            if 0 <= c < n:
                A[i, c] = band[i, j]
    return A


def apply_active(A, b, active):
    """Replace rows with ``active[i] != 0`` by identity rows with rhs 0."""
    if active is None:
        return A, b
    A = A.copy()
    b = b.copy()
    for i in np.nonzero(np.asarray(active))[0]:
        A[i, :] = 0.0
        A[i, i] = 1.0
        b[i] = 0.0
    return A, b


def solve_dense(A, b):
    """``A^{-1} b`` by LU with partial pivoting (LAPACK getrf/getrs)."""
    return np.linalg.solve(A, b)


def lcp_pgs(A, b, tol=1e-15, max_sweeps=100000, x0=None):
    """Projected Gauss-Seidel for ``x >= 0, A x - b >= 0, x^T (A x - b) = 0``.

    The projected splitting iteration whose convergence Sec. 3.2 quotes from
    Cryer (Theorem on projected splittings): sweep i = 0..n-1,
    ``x_i <- max(0, x_i - (A x - b)_i / A_ii)``.  Stops when a sweep changes no
    component by more than ``tol * max(1, |x|_inf)``.  Returns ``(x, sweeps)``.
    """
    n = len(b)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    for sweep in range(1, max_sweeps + 1):
        change = 0.0
        for i in range(n):
            r = A[i] @ x - b[i]
            xi = max(0.0, x[i] - r / A[i, i])
            change = max(change, abs(xi - x[i]))
            x[i] = xi
        if change <= tol * max(1.0, np.max(np.abs(x))):
            return x, sweep
    return x, max_sweeps


def lcp_enumerate(A, b):
    """Exact LCP solution by trying every support set (n <= 12).

    For a P-matrix (e.g. strictly diagonally dominant with positive diagonal)
    exactly one support S gives ``x_S = A_SS^{-1} b_S >= 0`` and
    ``(A x - b)_i >= 0`` off S; that is the unique solution.  Returns the
    list of all feasible solutions found (length 1 for a P-matrix).
    """
    n = len(b)
    if n > 12:
        raise ValueError("enumeration is limited to n <= 12")
    sols = []
    for k in range(n + 1):
        for S in itertools.combinations(range(n), k):
            x = np.zeros(n)
            if k:
                S = list(S)
                x[S] = np.linalg.solve(A[np.ix_(S, S)], b[S])
                if np.any(x[S] < -1e-13):
                    continue
            w = A @ x - b
            off = np.ones(n, dtype=bool)
            off[list(S)] = False
            if np.any(w[off] < -1e-13):
                continue
            sols.append(np.maximum(x, 0.0))
    return sols


def paqif_reference(band, rhs, beta, mode, active=None, pgs_tol=1e-15):
    """Reference result of one batched call: ``band [n_sys, n, 2b+1]``, ``rhs [n_sys, n]``.

    Returns ``x [n_sys, n]``.  Mode 2 uses projected Gauss-Seidel (valid for
    the strictly diagonally dominant matrices the tests generate).
    """
    band = np.asarray(band, dtype=np.float64)
    rhs = np.asarray(rhs, dtype=np.float64)
    out = np.empty_like(rhs)
    for s in range(band.shape[0]):
        A = band_to_dense(band[s], beta)
        act = None if active is None else active[s]
        A, b = apply_active(A, rhs[s], act)
        if mode == 0:
            out[s] = solve_dense(A, b)
        elif mode == 1:
            out[s] = np.maximum(solve_dense(A, b), 0.0)
        elif mode == 2:
            out[s], _ = lcp_pgs(A, b, tol=pgs_tol)
        else:
            raise ValueError("mode must be 0, 1 or 2")
    return out
