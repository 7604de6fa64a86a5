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


@pytest.mark.parametrize("beta", [1, 2, 4])
@pytest.mark.parametrize("r", [2, 4])
def test_normal_equations_of_step_4_give_the_same_solution(beta, r):
    """Step 4 as printed (R_d^T R_d U_d = R_d^T F_d by Cholesky) and the direct solve the GPU
    path takes (reading A18) agree on well-conditioned systems."""
    n = 48 if beta < 4 else 80
    A, f = dense(n, beta, 300 * r + beta)
    ref = np.linalg.solve(A, f)
    u_n, uO_n = aq.paqif_partitioned(A, f, beta, r, return_reduced=True, reduced="normal")
    u_d, uO_d = aq.paqif_partitioned(A, f, beta, r, return_reduced=True)
    assert np.max(np.abs(u_n - ref)) <= 1e-11 * np.max(np.abs(ref))
    assert np.max(np.abs(uO_n - uO_d)) <= 1e-11 * np.max(np.abs(uO_d))


def test_normal_equations_square_the_conditioning():
    """On the 1-D Laplacian shifted to within 0.1 % of its smallest eigenvalue (condition number
    about 1e6) the direct solve keeps about 11 digits and the normal equations about 8: they
    square the reduced system's conditioning (why the GPU path eliminates it instead, reading
    A18)."""
    beta, r, n = 1, 4, 48
    lmin = 2.0 - 2.0 * np.cos(np.pi / (n + 1))
    A = 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1) - lmin * (1.0 - 1e-3) * np.eye(n)
    f = np.random.default_rng(3).uniform(-1.0, 1.0, n)
    ref = np.linalg.solve(A, f)
    err_d = np.max(np.abs(aq.paqif_partitioned(A, f, beta, r) - ref)) / np.max(np.abs(ref))
    err_n = np.max(np.abs(aq.paqif_partitioned(A, f, beta, r, reduced="normal") - ref)) / np.max(np.abs(ref))
    assert err_d <= 1e-9
    assert err_n > 100 * err_d


def test_stepwise_projection_equals_projection_after_for_a_positive_solution():
    """Steps 5-7 (project U_F, U_L, solve the interiors from them, project) and the projection
    after the full solve (reading A17) coincide when the outer unknowns are nonnegative."""
    beta, n = 2, 48
    A, _ = dense(n, beta, 21)
    xt = np.random.default_rng(21).uniform(0.5, 1.5, n)
    f = A @ xt
    for r in (1, 2, 4):
        us = aq.paqif_partitioned(A, f, beta, r, mode=1, projection="steps")
        ua = aq.paqif_partitioned(A, f, beta, r, mode=1)
        assert np.max(np.abs(us - xt)) <= 1e-12 and np.max(np.abs(ua - xt)) <= 1e-12


def test_stepwise_projection_depends_on_the_partition_count():
    """With negative outer unknowns the stepwise projection feeds clipped values into the
    interior solves, so its result changes with r; the projection after the solve does not."""
    beta, n = 2, 48
    A, f = dense(n, beta, 23)
    u = np.linalg.solve(A, f)
    assert np.min(u) < 0 and np.max(u) > 0
    after = [aq.paqif_partitioned(A, f, beta, r, mode=1) for r in (2, 4)]
    steps = [aq.paqif_partitioned(A, f, beta, r, mode=1, projection="steps") for r in (2, 4)]
    assert np.max(np.abs(after[0] - after[1])) <= 1e-12 * np.max(np.abs(u))
    assert np.array_equal(after[0], np.maximum(aq.paqif_partitioned(A, f, beta, 2), 0.0))
    assert np.max(np.abs(steps[0] - steps[1])) > 1e-6
