"""Pins of the dense AQIF / partitioned-PAQIF reference (oracle/aqif_ref.py).

The factorization is checked by the product it must reproduce and by the zero
patterns Sec. 2.2.1 states for W0 (unit diagonal; column j of the left half is
zero in rows j+1 .. n-1-j, column j of the right half in rows n-1-j .. j-1,
0-based) and that the middle-out order implies for Z0 (the row of a pivot at
level k is zero in the columns eliminated before it); the solves are checked
against LU with partial pivoting, and the partitioned method's reduced system
against the LU solution at the blocks' outer rows.  A dropped coupling block
or a sign error in Step 4 changes every partitioned result (r > 1)."""
import numpy as np
import pytest

from oracle import aqif_ref as aq
from oracle import paqif_ref as pr
from paper_2008_03276_gb300 import inputs


def dense(n, beta, seed):
    band, rhs = inputs.dd_band_systems(1, n, beta, seed=seed)
    return pr.band_to_dense(band[0], beta), rhs[0]


@pytest.mark.parametrize("n,beta", [(2, 1), (8, 1), (16, 2), (30, 4), (40, 8)])
def test_factor_reproduces_matrix_with_the_stated_patterns(n, beta):
    A, _ = dense(n, beta, 10 * n + beta)
    W, Z = aq.aqif_factor(A)
    assert np.max(np.abs(W @ Z - A)) <= 1e-13 * np.max(np.abs(A))
    s = n // 2
    assert np.all(np.diag(W) == 1.0)
    for j in range(n):
        rows = range(j + 1, n - j) if j < s else range(n - 1 - j, j)
        for i in rows:
            assert W[i, j] == 0.0, (i, j)
    for k in range(s):
        p, q = s - 1 - k, s + k
        assert np.all(Z[p, p + 1:q] == 0.0) and np.all(Z[q, p + 1:q] == 0.0)


@pytest.mark.parametrize("n,beta", [(8, 1), (16, 2), (30, 4), (40, 8)])
def test_aqif_solve_matches_lu(n, beta):
    A, f = dense(n, beta, 7 * n + beta)
    W, Z = aq.aqif_factor(A)
    u = aq.aqif_solve(W, Z, f)
    ref = np.linalg.solve(A, f)
    assert np.max(np.abs(u - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("beta", [1, 2, 4])
@pytest.mark.parametrize("r", [1, 2, 4])
def test_partitioned_matches_lu_and_its_reduced_system(beta, r):
    n = 48 if beta < 4 else 80
    A, f = dense(n, beta, 100 * r + beta)
    ref = np.linalg.solve(A, f)
    u, uO = aq.paqif_partitioned(A, f, beta, r, return_reduced=True)
    assert np.max(np.abs(u - ref)) <= 1e-12 * np.max(np.abs(ref))
    nb = n // r
    outer = [m * nb + i for m in range(r) for i in list(range(beta)) + list(range(nb - beta, nb))]
    assert np.max(np.abs(uO - ref[outer])) <= 1e-12 * np.max(np.abs(ref))
    u1 = aq.paqif_partitioned(A, f, beta, r, mode=1)
    assert np.array_equal(u1, np.maximum(u, 0.0))


def test_partitioned_needs_the_coupling_blocks():
    """With the couplings of Step 4 dropped the blocks decouple: the result is block-Jacobi's,
    measurably different from A^-1 f -- the pin above would catch a dropped term."""
    beta, r, n = 2, 4, 48
    A, f = dense(n, beta, 5)
    nb = n // r
    Ab = np.zeros_like(A)
    for m in range(r):
        sl = slice(m * nb, (m + 1) * nb)
        Ab[sl, sl] = A[sl, sl]
    ub = aq.paqif_partitioned(Ab, f, beta, r)
    assert np.max(np.abs(ub - np.linalg.solve(A, f))) > 1e-6
    assert np.max(np.abs(ub - np.linalg.solve(Ab, f))) <= 1e-12 * np.max(np.abs(ub))
