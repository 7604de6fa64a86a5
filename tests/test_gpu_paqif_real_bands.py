"""GPU parity of PAQIF on the band systems the EHL method itself solves (Sec. 2.2.1-2.2.4).

The other PAQIF tests use strictly diagonally dominant seeded bands.  Here the bands come
from the oracle's Jacobians at states of the configurations (the C ABI's ehl_jacobian_band
computes the same bands, GPU parity in test_gpu_line.py / test_gpu_point.py):

* line contact N = 129, M = 20, L = 10, beta = 2: the paper's frozen Newton matrix with the
  weighted-change distribution (kind 0, Sec. 3.3.3-3.3.4) and the row-scaled band of the exact
  Jacobian (kind 1, the Newton-Krylov preconditioner), at the converged solution and at the
  Hertzian start, cavitated rows active;
* line contact N = 4097, M = 200, L = 10, van Leer, beta = 2, 4, 8 (kinds 0 and 1) at the
  start of the finest grid of the nested iteration (the N = 1025 solution prolonged twice),
  every admissible partition count r;
* the 255 x-line systems of the 257^2 point contact (M = 100, L = 10) at the prolonged 65^2
  solution, row-scaled exact bands, every admissible r;
* seeded bands that are not diagonally dominant (positive and indefinite diagonals), and
  bands whose middle 2x2 pivot is singular, which must be reported as EHL_INFO_SINGULAR.

Reference: dense LU with partial pivoting (oracle/paqif_ref.py).  Bounds, per system, with
u = 2^-48 (the double-float unit roundoff) and kappa the infinity-norm condition number of
the system with its active rows replaced by identity rows:
  normwise backward error  ||A x - b|| / (||A|| ||x|| + ||b||)  <= 5e-13,
  normwise forward error   ||x - x_LU|| / ||x_LU||             <= max(1e-12, 64 u kappa).
The frozen kind-0 matrices have kappa up to 1e15 (the distribution matrix of the weighted-
change method is nearly singular), so the backward error is the binding check there; the
largest errors seen are printed.
"""
import numpy as np
import pytest
import torch

from oracle import line_ref as lr
from oracle import paqif_ref as pq
from oracle import point_ref as ptr
from paper_2008_03276_gb300 import inputs, ops

pytestmark = pytest.mark.gpu
U_DF = 2.0**-48
BWD_TOL = 5e-13
EHL_INFO_SINGULAR = 1  # include/ehl.h
GPC = {1: 32, 2: 20, 3: 16, 4: 12, 5: 8, 6: 8, 7: 8, 8: 8}  # lane groups per CTA


def admissible(beta, n, r):
    npart = 2 * ((n + 2 * r - 1) // (2 * r))
    return GPC[beta] % r == 0 and (r == 1 or (npart >= 2 * beta + 2 and (r - 1) * npart < n))


def all_parts(beta, n):
    return [r for r in range(1, GPC[beta] + 1) if admissible(beta, n, r)]


def exact_band(J, beta):
    n = J.shape[0]
    band = np.zeros((n, 2 * beta + 1))
    for d in range(-beta, beta + 1):
        i = np.arange(max(0, -d), min(n, n - d))
        band[i, beta + d] = J[i, i + d]
    return band


def scaled(band, beta, P, R):
    """Row scale d_i = max(|J_ii|, max_j |J_ij| / 10); rows with P_i <= R_i / d_i active."""
    d = np.maximum(np.abs(band[:, beta]), np.max(np.abs(band), axis=1) / 10.0)
    return band / d[:, None], P <= R / d, -R / d


def check(label, band, rhs, act, beta, parts):
    """Every partition count in `parts` against dense LU; returns the worst errors."""
    n_sys, n, _ = band.shape
    x_ref = pq.paqif_reference(band, rhs, beta, 0, active=act)
    kappa = np.empty(n_sys)
    dense = []
    for s in range(n_sys):
        A, b = pq.apply_active(pq.band_to_dense(band[s], beta), rhs[s], act[s])
        kappa[s] = np.linalg.cond(A, np.inf)
        dense.append((A, b))
    dev = torch.device("cuda")
    tb = torch.from_numpy(np.ascontiguousarray(band)).to(dev)
    tr = torch.from_numpy(np.ascontiguousarray(rhs)).to(dev)
    ta = torch.from_numpy(np.ascontiguousarray(act.astype(np.uint8))).to(dev)
    worst_f = worst_b = 0.0
    for r in parts:
        x, iters, info = ops.paqif_solve(tb, tr, beta, 0, active=ta, partitions=r)
        torch.cuda.synchronize()
        x, info = x.cpu().numpy(), info.cpu().numpy()
        assert np.all(info == 0), (label, r, info.tolist())
        for s in range(n_sys):
            A, b = dense[s]
            xs, xr = x[s], x_ref[s]
            fwd = np.max(np.abs(xs - xr)) / max(np.max(np.abs(xr)), 1e-300)
            bwd = np.max(np.abs(A @ xs - b)) / (np.linalg.norm(A, np.inf) * np.max(np.abs(xs)) + np.max(np.abs(b)))
            assert bwd <= BWD_TOL, (label, r, s, bwd)
            assert fwd <= max(1e-12, 64 * U_DF * kappa[s]), (label, r, s, fwd, kappa[s])
            worst_f, worst_b = max(worst_f, fwd), max(worst_b, bwd)
    print(f"{label}: kappa <= {np.max(kappa):.2e}, forward <= {worst_f:.2e}, backward <= {worst_b:.2e}, r in {parts}")
    return worst_f, worst_b


# ---- line contact, N = 129 (C1) -------------------------------------------------------------

@pytest.fixture(scope="module")
def c1_states():
    pb = lr.LineProblem(129, 20.0, 10.0, limiter="minmod")
    P, H0, info = lr.solve(pb, tol=1e-12)
    assert info["converged"]
    Ph = pb.hertz()
    return pb, {"converged": (P, H0), "hertz": (Ph, pb.h0_for_min_film(Ph, 0.05))}


@pytest.mark.parametrize("where", ["converged", "hertz"])
def test_c1_bands(c1_states, where):
    pb, states = c1_states
    P, H0 = states[where]
    R = lr.residual(pb, P, H0)
    beta = 2
    b0, a0 = lr.jacobian_band(pb, P, H0, beta)
    J, _ = lr.jacobian_exact(pb, P, H0)
    b1, a1, r1 = scaled(exact_band(J, beta), beta, P, R)
    assert a0.any() and a1.any()
    band = np.stack([b0, b1])
    rhs = np.stack([np.where(a0, 0.0, -R), r1])
    act = np.stack([a0, a1])
    check(f"C1 {where} kinds 0/1", band, rhs, act, beta, all_parts(beta, pb.n))


# ---- line contact, N = 4097, M = 200 (C2a) --------------------------------------------------

@pytest.fixture(scope="module")
def c2a_state():
    fac = lambda N: lr.LineProblem(N, 200.0, 10.0, limiter="vanleer")
    pbc, Pc, H0c, info = lr.solve_nested(fac, 1025, tol=1e-10)
    assert info["converged"]
    pb = fac(4097)
    P = np.maximum(lr.prolong(lr.prolong(pbc.full(Pc)))[1:-1], 0.0)
    R = lr.residual(pb, P, H0c)
    J, _ = lr.jacobian_exact(pb, P, H0c)
    return pb, P, H0c, R, J


@pytest.mark.parametrize("beta", [2, 4, 8])
def test_c2a_bands_every_partition_count(c2a_state, beta):
    pb, P, H0, R, J = c2a_state
    b0, a0 = lr.jacobian_band(pb, P, H0, beta)
    b1, a1, r1 = scaled(exact_band(J, beta), beta, P, R)
    band = np.stack([b0, b1])
    rhs = np.stack([np.where(a0, 0.0, -R), r1])
    act = np.stack([a0, a1])
    parts = all_parts(beta, pb.n)
    assert 1 in parts and len(parts) >= 3
    check(f"C2a beta={beta} kinds 0/1", band, rhs, act, beta, parts)


# ---- point contact, the 257^2 x-lines (C4) --------------------------------------------------

def test_point_257_xline_bands_every_partition_count():
    fac = lambda nx, ny: ptr.PointProblem(nx, ny, 100.0, 10.0)
    pbc, Pc, H0, info = ptr.solve_nested(fac, 65, 65, tol=1e-10)
    assert info["converged"]
    pb = fac(257, 257)
    P = np.maximum(ptr.prolong(ptr.prolong(pbc.full(Pc)))[1:-1, 1:-1], 0.0)  # [255, 255] (x, y)
    beta = 2
    band = ptr.xline_band_exact(pb, P.ravel(), H0, beta)  # [y-line][x][2 beta + 1]
    R = ptr.residual(pb, P.ravel(), H0).reshape(255, 255)
    bs, acts, rhss = [], [], []
    for j in range(255):
        b, a, r = scaled(band[j], beta, P[:, j], R[:, j])
        bs.append(b)
        acts.append(a)
        rhss.append(r)
    act = np.stack(acts)
    assert act.any() and not act.all()
    check("257^2 x-lines", np.stack(bs), np.stack(rhss), act, beta, all_parts(beta, 255))


# ---- seeded bands that are not diagonally dominant ------------------------------------------

def nondominant(kind, n_sys, n, beta, seed):
    rng = np.random.default_rng(seed)
    band = rng.uniform(-1.0, 1.0, (n_sys, n, 2 * beta + 1))
    for d in range(-beta, beta + 1):
        i = np.arange(n)
        band[:, (i + d < 0) | (i + d >= n), beta + d] = 0.0
    off = np.sum(np.abs(band), axis=2) - np.abs(band[:, :, beta])
    mag = (0.5 + 0.5 * rng.random((n_sys, n))) * off
    sign = 1.0 if kind == "positive" else rng.choice([-1.0, 1.0], (n_sys, n))
    band[:, :, beta] = sign * mag
    rhs = rng.uniform(-1.0, 1.0, (n_sys, n))
    return band, rhs


@pytest.mark.parametrize("kind", ["positive", "indefinite"])
@pytest.mark.parametrize("beta,n", [(2, 64), (2, 1024), (4, 301), (8, 1024)])
def test_nondominant_seeded_bands(kind, beta, n):
    band, rhs = nondominant(kind, 16, n, beta, seed=1000 * beta + n + (kind == "indefinite"))
    act = np.zeros(rhs.shape, dtype=bool)
    parts = all_parts(beta, n)
    check(f"non-dominant {kind} beta={beta} n={n}", band, rhs, act, beta, sorted({parts[0], parts[-1]}))


@pytest.mark.parametrize("beta", [1, 2, 4, 8])
@pytest.mark.parametrize("rel_det", [0.0, 1e-15])
def test_singular_middle_pivot_is_reported(beta, rel_det):
    """With one block per system the first 2x2 pivot is the middle pair of rows (s-1, s);
    a pivot with |det| far below the rounding of |a d| + |b c| must set EHL_INFO_SINGULAR.
    The other systems of the batch (diagonally dominant) are solved as usual."""
    n = 128
    band, rhs = inputs.dd_band_systems(3, n, beta, seed=7 + beta)
    s = n // 2
    # pivot block [[1, 2], [2, 4 (1 + rel_det)]] in rows / columns (s-1, s) of system 1
    band[1, s - 1, beta] = 1.0
    band[1, s - 1, beta + 1] = 2.0
    band[1, s, beta - 1] = 2.0
    band[1, s, beta] = 4.0 * (1.0 + rel_det)
    dev = torch.device("cuda")
    x, iters, info = ops.paqif_solve(torch.from_numpy(band).to(dev), torch.from_numpy(rhs).to(dev), beta, 0,
                                     partitions=1)
    torch.cuda.synchronize()
    info = info.cpu().numpy()
    assert info[1] == EHL_INFO_SINGULAR
    assert info[0] == 0 and info[2] == 0
    ref = pq.paqif_reference(band[[0, 2]], rhs[[0, 2]], beta, 0)
    xs = x.cpu().numpy()[[0, 2]]
    assert np.max(np.abs(xs - ref)) <= 1e-12 * np.max(np.abs(ref))
