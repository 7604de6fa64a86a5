"""The PAQIF algorithm itself on dense matrices (test infrastructure).

`paqif_ref.py` writes out what PAQIF computes (A^{-1} b, its projection, the
LCP); this module follows the paper's steps, so that the factorization and
the partitioned method have a reference of their own:

* `aqif_factor` -- Sec. 2.2.1 / 2.2.3: L0 = W0 Z0 with 2x2 pivots taken from
  the middle of the matrix outwards.  Level k (0-based) pivots on rows and
  columns p = s-1-k and q = s+k of the current Schur complement; its rows are
  rows p, q of Z0, and the multipliers of every row outside [p, q] (the rows
  not yet eliminated) are columns p, q of W0.
* `aqif_solve` -- Sec. 2.2.2: W0 Y = F from the middle outwards, then
  Z0 U = Y from both ends towards the middle, one 2x2 solve per level.
* `paqif_partitioned` -- Sec. 2.1 (Eqs. eqn15, eqnn16) and Sec. 2.2.4
  Steps 1-7: r diagonal blocks L0^(m) of equal even order, each factored
  (Step 1) and swept (Step 2); the outer 2 beta x 2 beta block of W0^-1
  (Step 3); the reduced system of order 2 beta r for the first and last beta
  unknowns of every block in the paper's form, Z0's outer rows plus W0^-1's
  outer block times the coupling blocks L_-, L_+ (Step 4); the interiors from
  Z0 U_M = Y_M - Z0[M, outer] U_outer (Step 6).  By default the reduced system
  is solved directly (numpy LU), not through the normal equations of Step 4,
  and the projection of Steps 5 and 7 is applied once after the full solve
  (the readings of the paper the GPU path takes).  The paper's own forms are
  options: ``reduced="normal"`` forms R_d^T R_d U_d = R_d^T F_d and solves it
  by Cholesky (Step 4), ``projection="steps"`` projects the outer unknowns
  before the interiors are solved from them (Step 5) and the interiors after
  (Step 7).

Dense and O(n^3): small sizes only.  Pins (tests/test_oracle_aqif.py): W0 Z0
reproduces the matrix; W0 has unit diagonal and the zero pattern of
Sec. 2.2.1; Z0's rows have the zero pattern the middle-out order implies;
every solve matches LU with partial pivoting; the reduced system's solution
is the LU solution at the blocks' outer rows; the normal equations give the
same solution (to their squared conditioning); the stepwise projection equals
the projection after the solve when the outer unknowns are nonnegative, and
otherwise depends on r.
"""
import numpy as np


def _check_even(n):
    if n % 2:
        raise ValueError("AQIF pairs rows: the order must be even (pad with an identity row)")


def aqif_factor(A):
    """``(W0, Z0)`` with ``W0 @ Z0 == A`` by middle-out 2x2 pivoting (Sec. 2.2.1)."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    _check_even(n)
    s = n // 2
    L = A.copy()  # the current Schur complement, eliminated rows and columns kept in place
    W = np.eye(n)
    Z = np.zeros((n, n))
    for k in range(s):
        p, q = s - 1 - k, s + k
        piv = [p, q]
        Z[piv, :] = L[piv, :]
        Pi = L[np.ix_(piv, piv)]
        rest = [i for i in range(n) if i < p or i > q]  # rows not yet eliminated
        if rest:
            Wr = L[np.ix_(rest, piv)] @ np.linalg.inv(Pi)  # [w_ip, w_iq] solves Pi^T w = [l_ip, l_iq]
            W[np.ix_(rest, piv)] = Wr
            L[rest, :] -= Wr @ L[piv, :]
            L[np.ix_(rest, piv)] = 0.0  # eliminated: zero by construction, not by rounding
    return W, Z


def aqif_solve(W, Z, f):
    """``U`` with ``W0 Z0 U = f``: W0 Y = F middle-out, Z0 U = Y ends-inwards (Sec. 2.2.2)."""
    n = W.shape[0]
    _check_even(n)
    s = n // 2
    y = np.array(f, dtype=np.float64)
    for k in range(s):  # W0 Y = F: the pivot pair of a level is final, the outer rows take its terms
        p, q = s - 1 - k, s + k
        rest = [i for i in range(n) if i < p or i > q]
        if rest:
            y[rest] -= W[np.ix_(rest, [p, q])] @ y[[p, q]]
    u = np.zeros(n)
    for k in range(s - 1, -1, -1):  # Z0 U = Y: outer pairs first
        p, q = s - 1 - k, s + k
        outer = [i for i in range(n) if i < p or i > q]
        rhs = y[[p, q]] - (Z[np.ix_([p, q], outer)] @ u[outer] if outer else 0.0)
        u[[p, q]] = np.linalg.solve(Z[np.ix_([p, q], [p, q])], rhs)
    return u


def paqif_partitioned(A, f, beta, r, mode=0, return_reduced=False, reduced="lu", projection="after"):
    """The partitioned PAQIF of Sec. 2.2.4 on a dense banded ``A`` (half-band ``beta``).

    ``r`` blocks of equal even order ``n / r >= 2 beta + 2``.  mode 0 returns
    U, mode 1 ``max(0, U)``.  ``reduced``: "lu" solves the reduced system
    R_d U_d = F_d directly, "normal" through its normal equations by Cholesky
    (Step 4 as printed).  ``projection`` (mode 1): "after" projects the full
    solution once, "steps" projects U_F, U_L (Step 5), solves the interiors
    from the projected values (Step 6) and projects them (Step 7).  With
    ``return_reduced`` also the reduced system's solution before any
    projection, ordered ``[U_F^(1), U_L^(1), U_F^(2), ...]``.
    """
    if reduced not in ("lu", "normal") or projection not in ("after", "steps"):
        raise ValueError("reduced is 'lu' or 'normal', projection 'after' or 'steps'")
    A = np.asarray(A, dtype=np.float64)
    f = np.asarray(f, dtype=np.float64)
    n = A.shape[0]
    if n % r or (n // r) % 2 or n // r < 2 * beta + 2:
        raise ValueError("blocks of equal even order >= 2 beta + 2 required")
    nb = n // r
    b = beta
    F = list(range(b))               # first beta rows of a block
    Lr = list(range(nb - b, nb))     # last beta rows
    O = F + Lr                       # outer rows, in this order
    M = list(range(b, nb - b))       # interior rows
    blocks = []
    for m in range(r):
        sl = slice(m * nb, (m + 1) * nb)
        W, Z = aqif_factor(A[sl, sl])                       # Step 1
        # Step 2: W0 Y = F (the W-sweep of aqif_solve alone)
        y = f[sl].copy()
        s = nb // 2
        for k in range(s):
            p, q = s - 1 - k, s + k
            rest = [i for i in range(nb) if i < p or i > q]
            if rest:
                y[rest] -= W[np.ix_(rest, [p, q])] @ y[[p, q]]
        Winv = np.linalg.inv(W)
        Wout = Winv[np.ix_(O, O)]                           # Step 3: W0^-1's outer 2b x 2b block
        blocks.append(dict(W=W, Z=Z, y=y, Wout=Wout))
    # Step 4: for block m,  Z0[O, O] u_O^(m) + Wout^(m) [L_- u_L^(m-1); L_+ u_F^(m+1)] = y_O^(m)
    R = np.zeros((2 * b * r, 2 * b * r))
    g = np.zeros(2 * b * r)
    for m in range(r):
        bm = blocks[m]
        rows = slice(2 * b * m, 2 * b * (m + 1))
        R[rows, rows] = bm["Z"][np.ix_(O, O)]
        g[rows] = bm["y"][O]
        if m > 0:  # L_-: the block's first rows, the previous block's last columns
            Lm = A[np.ix_([m * nb + i for i in F], [(m - 1) * nb + i for i in Lr])]
            C = np.zeros((2 * b, b))
            C[:b, :] = Lm
            R[rows, 2 * b * (m - 1) + b:2 * b * m] += bm["Wout"] @ C
        if m < r - 1:  # L_+: the block's last rows, the next block's first columns
            Lp = A[np.ix_([m * nb + i for i in Lr], [(m + 1) * nb + i for i in F])]
            C = np.zeros((2 * b, b))
            C[b:, :] = Lp
            R[rows, 2 * b * (m + 1):2 * b * (m + 1) + b] += bm["Wout"] @ C
    if reduced == "lu":
        uO = np.linalg.solve(R, g)
    else:  # R_d^T R_d U_d = R_d^T F_d, symmetric positive definite: Cholesky without pivoting
        C = np.linalg.cholesky(R.T @ R)
        uO = np.linalg.solve(C.T, np.linalg.solve(C, R.T @ g))
    stepwise = mode == 1 and projection == "steps"
    uO_used = np.maximum(uO, 0.0) if stepwise else uO  # Step 5
    # Step 6: the interiors, Z0[M, M] u_M = y_M - Z0[M, O] u_O
    u = np.zeros(n)
    for m in range(r):
        bm = blocks[m]
        uo = uO_used[2 * b * m:2 * b * (m + 1)]
        um = np.linalg.solve(bm["Z"][np.ix_(M, M)], bm["y"][M] - bm["Z"][np.ix_(M, O)] @ uo)
        u[m * nb + np.array(O)] = uo
        u[m * nb + np.array(M)] = um
    if mode == 1:  # Step 7 (with Step 5 above), or the projection of the full solution
        u = np.maximum(u, 0.0)
    return (u, uO) if return_reduced else u
