"""The device-driven solve (ehl_params.graph = 2) against the host-driven one and the oracle.

With graph = 2 the whole iteration of a grid -- Newton steps, their GMRES iterations and their
line-search trials -- is one CUDA graph whose while-loops are controlled on the device; the
kernels are the host-driven path's, so the converged P, H0 agree with graph = 0 to rounding
(1e-12 relative) and with the oracle to 1e-8, for one instance, a batch of different loads and
a ragged batch of grid sizes; the iteration counts agree too.
"""
import numpy as np
import pytest
import torch

from oracle import line_ref as lr
from paper_2008_03276_gb300 import ops

pytestmark = pytest.mark.gpu


def solve(graph, n_inst=1, per=None, rough=None, **kw):
    q = dict(nx=129, M=20.0, L=10.0, limiter=0, halfband=2, method=1, tol=1e-10, max_iter=60)
    q.update(kw)
    p = ops.default_params(1, graph=graph, **q)
    per_inst = None if per is None else [ops.default_params(1, graph=graph, **{**q, **d}) for d in per]
    ctx = ops.Context(p, n_inst=n_inst, per_inst=per_inst)
    n0 = ops.kernel_launches()
    P, H0, iters, res, code = ctx.solve(rough=rough, check=False)
    torch.cuda.synchronize()
    return P.cpu().numpy(), H0.cpu().numpy(), iters.cpu().numpy(), res.cpu().numpy(), code, \
        ops.kernel_launches() - n0, ctx


def test_c1_matches_host_driven_and_oracle():
    pb = lr.LineProblem(129, 20.0, 10.0, limiter="minmod")
    Pr, H0r, info = lr.solve(pb)
    assert info["converged"]
    P2, H2, it2, r2, c2, l2, _ = solve(2)
    P0, H00, it0, r0, c0, l0, _ = solve(0)
    assert c2 == 0 and c0 == 0
    assert np.array_equal(it2, it0)
    assert np.max(np.abs(P2 - P0)) <= 1e-12 * np.max(P0)
    assert np.max(np.abs(P2[0, 1:-1] - Pr)) <= 1e-8 * np.max(Pr)
    assert abs(H2[0] - H0r) <= 1e-8 * abs(H0r)
    # every kernel the replay ran is counted (no host-side launches inside the loops)
    assert l2 > 0


def test_batch_of_loads_and_second_solve_reuses_the_graph():
    per = [dict(M=m, L=l) for m, l in ((10.0, 5.0), (20.0, 10.0), (50.0, 10.0), (100.0, 12.0))]
    P2, H2, it2, r2, c2, _, ctx = solve(2, n_inst=4, per=per, nx=257)
    P0, H00, it0, r0, c0, _, _ = solve(0, n_inst=4, per=per, nx=257)
    assert c2 == 0 and c0 == 0
    assert np.array_equal(it2, it0)
    assert np.max(np.abs(P2 - P0)) <= 1e-12 * np.max(P0)
    assert np.max(np.abs(H2 - H00)) <= 1e-12 * np.max(np.abs(H00))
    P3, H3, it3, r3, c3 = ctx.solve(check=False)  # the graph is replayed
    assert int(c3) == 0 and np.array_equal(P3.cpu().numpy(), P2)


def test_ragged_batch_and_roughness():
    per = [dict(nx=n, M=m) for n, m in ((129, 20.0), (257, 50.0), (513, 200.0), (257, 20.0))]
    X = [np.linspace(-4.5, 1.5, q["nx"]) for q in per]
    rough = np.zeros((4, 513))
    for k, x in enumerate(X):
        rough[k, :len(x)] = 0.01 * np.sin(2 * np.pi * x / 0.5)
    rt = torch.tensor(rough, device="cuda")
    P2, H2, it2, r2, c2, _, _ = solve(2, n_inst=4, per=per, rough=rt, nx=513, limiter=1, halfband=4)
    P0, H00, it0, r0, c0, _, _ = solve(0, n_inst=4, per=per, rough=rt, nx=513, limiter=1, halfband=4)
    assert c2 == 0 and c0 == 0
    assert np.array_equal(it2, it0)
    for k, q in enumerate(per):
        n = q["nx"]
        assert np.max(np.abs(P2[k, :n] - P0[k, :n])) <= 1e-12 * np.max(P0[k, :n])


def test_high_load_nested_grids():
    P2, H2, it2, r2, c2, _, _ = solve(2, nx=1025, M=200.0, limiter=1, halfband=8, tol=1e-8)
    assert c2 == 0
    assert np.max(np.abs(r2)) <= 1e-8


def point_solve(graph, n=33, **kw):
    q = dict(nx=n, ny=n, M=20.0, L=10.0, limiter=0, halfband=2, method=1, tol=1e-11, max_iter=80,
             coarse_min_nodes=17, krylov_dim=40)
    q.update(kw)
    ctx = ops.Context(ops.default_params(2, graph=graph, **q))
    P, H0, iters, res, code = ctx.solve(check=False)
    torch.cuda.synchronize()
    return P.cpu().numpy(), H0.cpu().numpy(), iters.cpu().numpy(), res.cpu().numpy(), code


@pytest.mark.parametrize("deform,yline", [(0, 0), (1, 0), (1, 1)])
def test_point_matches_host_driven_and_oracle(deform, yline):
    from oracle import point_ref as pr
    pb = pr.PointProblem(33, 33, 20.0, 10.0)
    Pr, H0r, info = pr.solve(pb, tol=1e-11)
    assert info["converged"]
    P2, H2, it2, r2, c2 = point_solve(2, deform=deform, yline=yline)
    P0, H00, it0, r0, c0 = point_solve(0, deform=deform, yline=yline)
    assert c2 == 0 and c0 == 0
    assert np.array_equal(it2, it0)
    assert np.max(np.abs(P2 - P0)) <= 1e-12 * np.max(P0)
    assert np.max(np.abs(P2[0, 1:-1, 1:-1] - pb.full(Pr)[1:-1, 1:-1].T)) <= 1e-8 * np.max(Pr)
    assert abs(H2[0] - H0r) <= 1e-8 * abs(H0r)


def test_point_257_fft_device_driven():
    from oracle import point_ref as pr
    n = 257
    P, H0, it, res, code = point_solve(2, n=n, M=100.0, tol=1e-8, max_iter=60, coarse_min_nodes=33, krylov_dim=200,
                                       deform=1, autotune=1)
    assert code == 0
    pb = pr.PointProblem(n, n, 100.0, 10.0)
    Pint = P[0].T[1:-1, 1:-1].ravel()
    R = pr.residual(pb, Pint, float(H0[0]))
    assert np.max(np.abs(np.minimum(Pint, R))) <= max(2e-8, pr.rounding_floor(pb, Pint, float(H0[0])))


def paper_solve(graph, n_inst=1, per=None, **kw):
    q = dict(nx=129, M=20.0, L=10.0, limiter=0, halfband=2, method=0, tol=1e-8, max_iter=4000, levels=0)
    q.update(kw)
    p = ops.default_params(1, graph=graph, **q)
    per_inst = None if per is None else [ops.default_params(1, graph=graph, **{**q, **d}) for d in per]
    ctx = ops.Context(p, n_inst=n_inst, per_inst=per_inst)
    P, H0, iters, res, code = ctx.solve(check=False)
    torch.cuda.synchronize()
    return P.cpu().numpy(), H0.cpu().numpy(), iters.cpu().numpy(), res.cpu().numpy(), code, ctx


def test_paper_iteration_device_driven_matches_host_driven():
    """Method 0 (the paper's iteration, Sec. 3.3.3-3.3.4) as one device-side loop: the same
    kernels in the same order, so the same iteration count and the same iterate bit for bit;
    and the oracle's restatement of the iteration to the tolerance of its own test."""
    P2, H2, it2, r2, c2, ctx = paper_solve(2)
    P0, H00, it0, r0, c0, _ = paper_solve(0)
    assert c2 == 0 and c0 == 0
    assert np.array_equal(it2, it0)
    assert np.array_equal(P2, P0) and np.array_equal(H2, H00)
    pb = lr.LineProblem(129, 20.0, 10.0, limiter="minmod", dist_weight=0.5)
    Pr, H0r, info = lr.solve_paper(pb, tol=1e-8)
    assert info["converged"] and abs(int(it2[0]) - info["iters"]) <= 3
    P3, H3, it3, r3, c3 = ctx.solve(check=False)  # the graph is replayed
    assert int(c3) == 0 and np.array_equal(P3.cpu().numpy(), P2)


def test_paper_iteration_device_driven_batch():
    """A batch of loads, each instance leaving the device loop when it converges."""
    per = [dict(M=m, L=l) for m, l in ((10.0, 5.0), (15.0, 8.0), (25.0, 10.0))]
    P2, H2, it2, r2, c2, _ = paper_solve(2, n_inst=3, per=per)
    P0, H00, it0, r0, c0, _ = paper_solve(0, n_inst=3, per=per)
    assert c2 == 0 and c0 == 0
    assert np.array_equal(it2, it0) and len(set(it2.tolist())) > 1
    assert np.array_equal(P2, P0) and np.array_equal(H2, H00)
