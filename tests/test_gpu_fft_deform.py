"""GPU parity of the FFT evaluation of the point-contact deformation (ehl_params.deform = 1).

The deformation sum of Sec. 3.3.1 Case 2 is a 2-D discrete convolution of the interior
pressures with the cell kernel; deform = 1 evaluates it through a float64 FFT of cyclic length
2^ceil(log2(2 n - 3)) per direction.  Against the oracle (the direct sum in numpy): the film
to 1e-13 of max |H| and the residual to 1e-11 of its scale, on power-of-two and other grid
sizes; the Krylov product (ehl_jacobian_apply) against the oracle's exact Jacobian; the
converged solution at 33^2 to 1e-8; at 257^2 (the bench's point-contact configuration) the
oracle's residual at the GPU's solution, the force balance and the y-mirror symmetry.
"""
import numpy as np
import pytest
import torch

from oracle import point_ref as pr

from paper_2008_03276_gb300 import ops

pytestmark = pytest.mark.gpu
LIM = {0: "minmod", 1: "vanleer"}


def dev(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def make(n, M=20.0, L=10.0, limiter=0, beta=2, tol=1e-11, **kw):
    q = dict(nx=n, ny=n, limiter=limiter, halfband=beta, method=1, tol=tol, max_iter=80, levels=-1,
             coarse_min_nodes=17, krylov_dim=40, deform=1)
    q.update(kw)
    return ops.Context(ops.default_params(2, M=M, L=L, **q))


def perturbed_state(pb, seed):
    rng = np.random.default_rng(seed)
    P = pb.hertz() * (1 + 0.05 * rng.standard_normal(pb.n)).clip(0)
    return P, pb.h0_for_min_film(P, 0.1)


@pytest.mark.parametrize("n", [9, 33, 50, 65, 129])
@pytest.mark.parametrize("limiter", [0, 1])
def test_film_and_residual_match_oracle(n, limiter):
    pb = pr.PointProblem(n, n, 20.0, 10.0, limiter=LIM[limiter])
    ctx = make(n, limiter=limiter)
    P, H0 = perturbed_state(pb, n)
    R, H, comp = ctx.residual(dev(pb.full(P).T[None]), dev([H0]))
    R, H = R.cpu().numpy()[0], H.cpu().numpy()[0]
    s = pr.state(pb, P, H0)
    assert np.max(np.abs(H - s["H"].T)) <= 1e-13 * np.max(np.abs(s["H"]))
    scale = max(1.0, np.max(np.abs(s["R"])))
    assert np.max(np.abs(R[1:-1, 1:-1] - s["R"].T)) <= 1e-11 * scale


def test_nonzero_boundary_pressure_is_not_a_source():
    """The sum runs over interior cells (the oracle's P is zero on the boundary nodes)."""
    n = 33
    pb = pr.PointProblem(n, n, 20.0, 10.0)
    ctx = make(n)
    P, H0 = perturbed_state(pb, 1)
    Pn = pb.full(P).T.copy()
    _, H1, _ = ctx.residual(dev(Pn[None]), dev([H0]))
    Pn[0, :] = 5.0
    Pn[:, -1] = 7.0
    _, H2, _ = ctx.residual(dev(Pn[None]), dev([H0]))
    assert torch.equal(H1, H2)


def test_krylov_product_matches_the_exact_jacobian():
    n = 33
    pb = pr.PointProblem(n, n, 20.0, 10.0, limiter="vanleer")
    ctx = make(n, limiter=1)
    P, H0 = perturbed_state(pb, 7)
    J, JH = pr.jacobian_exact(pb, P, H0)
    rng = np.random.default_rng(3)
    v = rng.standard_normal(pb.n)
    vh = 0.7
    ref = J @ v + JH * vh
    out = ctx.jacobian_apply(dev(pb.full(P).T[None]), dev([H0]), dev(pb.full(v).T[None]), dev([vh]))
    out = out.cpu().numpy()[0]
    ni = n - 2
    sc = np.abs(J) @ np.abs(v) + np.abs(JH) * vh
    assert np.all(np.abs(out[1:-1, 1:-1] - ref.reshape(ni, ni).T) <= 1e-11 * sc.reshape(ni, ni).T + 1e-300)


def test_solve_33_matches_oracle():
    pb = pr.PointProblem(33, 33, 20.0, 10.0)
    Pr, H0r, info = pr.solve(pb, tol=1e-11)
    assert info["converged"]
    ctx = make(33)
    P, H0, iters, res, code = ctx.solve(check=False)
    assert code == 0
    P, H0 = P.cpu().numpy()[0], float(H0.cpu()[0])
    assert np.max(np.abs(P[1:-1, 1:-1] - pb.full(Pr)[1:-1, 1:-1].T)) <= 1e-8 * np.max(Pr)
    assert abs(H0 - H0r) <= 1e-8 * abs(H0r)


def test_solve_257_in_the_bench_configuration():
    n = 257
    p = ops.default_params(2, nx=n, ny=n, M=100.0, L=10.0, limiter=0, halfband=2, method=1, tol=1e-8,
                           max_iter=60, coarse_min_nodes=33, deform=1)
    ctx = ops.Context(p)
    P, H0, iters, res, code = ctx.solve(check=False)
    print(f"257^2 FFT: code {code} iters {iters.tolist()} res {res.tolist()}")
    assert code == 0
    Pn, H0n = P.cpu().numpy()[0], float(H0.cpu()[0])
    pb = pr.PointProblem(n, n, 100.0, 10.0)
    Pint = Pn.T[1:-1, 1:-1].ravel()
    R = pr.residual(pb, Pint, H0n)
    assert np.max(np.abs(np.minimum(Pint, R))) <= max(2e-8, pr.rounding_floor(pb, Pint, H0n))
    assert abs(pb.h**2 * Pint.sum() - 2 * np.pi / 3) <= 1e-8
    # Y in [-3, 3] is symmetric about y = 0: the solution is mirror symmetric
    assert np.max(np.abs(Pn - Pn[::-1, :])) <= 1e-6 * np.max(Pn)
