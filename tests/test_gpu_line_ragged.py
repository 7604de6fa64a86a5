"""Ragged batches: one context over line-contact instances of different grid sizes.

The caller's arrays are [n_inst][nx_max]; instance k uses the first nx_k
entries of its row.  Every per-instance result of a ragged context must equal
bit for bit the result of a context holding that instance alone (the same
kernels run on the same compact data), the padding must stay untouched, and
the converged solves must match the oracle.
"""
import numpy as np
import pytest
import torch

from oracle import line_ref as lr
from paper_2008_03276_gb300 import inputs, ops

pytestmark = pytest.mark.gpu

# interleaved sizes so that the gather/scatter index maps are not monotone blocks
PER = [dict(nx=257, M=20.0, L=10.0), dict(nx=129, M=50.0, L=5.0), dict(nx=257, M=150.0, L=12.0),
       dict(nx=129, M=10.0, L=15.0), dict(nx=193, M=80.0, L=8.0), dict(nx=129, M=300.0, L=10.0)]


def params(d, **kw):
    return ops.default_params(1, nx=d["nx"], M=d["M"], L=d["L"], **kw)


def ragged_state(seed=5):
    """Hertzian-like pressures plus noise, and roughness, padded to nx_max with a marker."""
    nx_max = max(d["nx"] for d in PER)
    rng = np.random.Generator(np.random.PCG64(seed))
    P = np.full((len(PER), nx_max), 7.25)
    R = np.full((len(PER), nx_max), -3.5)
    H0 = np.empty(len(PER))
    for k, d in enumerate(PER):
        pb = lr.LineProblem(d["nx"], d["M"], d["L"])
        p = np.sqrt(np.clip(1.0 - pb.X ** 2, 0.0, None)) * (1.0 + 0.05 * rng.standard_normal(pb.N))
        p[0] = p[-1] = 0.0
        P[k, :d["nx"]] = np.clip(p, 0.0, None)
        R[k, :d["nx"]] = inputs.sin_grf_roughness(pb.X, amp=0.02, wavelength=0.3, seed=seed + k)
        H0[k] = -0.4 + 0.1 * k
    return P, H0, R


def single(k, **kw):
    return ops.Context(params(PER[k], **kw), n_inst=1)


def test_ragged_residual_equals_single_contexts():
    P, H0, R = ragged_state()
    Pd, H0d, Rd = (torch.tensor(a, device="cuda") for a in (P, H0, R))
    ctx = ops.Context(params(PER[0]), n_inst=len(PER), per_inst=[params(d) for d in PER])
    assert ctx.ragged and ctx.nx == 257
    Rg, Hg, cg = ctx.residual(Pd, H0d, Rd)
    Rg, Hg, cg = Rg.cpu().numpy(), Hg.cpu().numpy(), cg.cpu().numpy()
    for k, d in enumerate(PER):
        n = d["nx"]
        c1 = single(k)
        R1, H1, cc1 = c1.residual(Pd[k:k + 1, :n].contiguous(), H0d[k:k + 1].contiguous(), Rd[k:k + 1, :n].contiguous())
        assert np.array_equal(Rg[k, :n], R1.cpu().numpy()[0])
        assert np.array_equal(Hg[k, :n], H1.cpu().numpy()[0])
        assert np.array_equal(cg[k], cc1.cpu().numpy()[0])
        assert np.all(Rg[k, n:] == 0.0) and np.all(Hg[k, n:] == 0.0)
        # against the oracle as well: H to 1e-13, R to 1e-12 of the magnitude of its terms
        pb = lr.LineProblem(n, d["M"], d["L"], rough=R[k, :n])
        s = lr.state(pb, P[k, 1:n - 1], H0[k])
        assert np.max(np.abs(Hg[k, :n] - s["H"])) <= 1e-13 * np.max(np.abs(s["H"]))
        F, ef, Pn, h = s["F"], s["epsf"], s["P"], pb.h
        scale = (np.abs(F[1:]) + np.abs(F[:-1])) / h + (np.abs(ef[1:] * (Pn[2:] - Pn[1:-1])) +
                                                       np.abs(ef[:-1] * (Pn[1:-1] - Pn[:-2]))) / h ** 2
        assert np.all(np.abs(Rg[k, 1:n - 1] - s["R"]) <= 1e-12 * scale + 1e-300)


@pytest.mark.parametrize("kind", [0, 1])
def test_ragged_band_jacobian_equals_single_contexts(kind):
    P, H0, R = ragged_state(seed=9)
    Pd, H0d, Rd = (torch.tensor(a, device="cuda") for a in (P, H0, R))
    beta = 4
    ctx = ops.Context(params(PER[0], halfband=beta), n_inst=len(PER), per_inst=[params(d, halfband=beta) for d in PER])
    band, act = ctx.jacobian_band(Pd, H0d, kind=kind, rough=Rd)
    band, act = band.cpu().numpy(), act.cpu().numpy()
    for k, d in enumerate(PER):
        n = d["nx"] - 2
        c1 = single(k, halfband=beta)
        b1, a1 = c1.jacobian_band(Pd[k:k + 1, :n + 2].contiguous(), H0d[k:k + 1].contiguous(), kind=kind,
                                  rough=Rd[k:k + 1, :n + 2].contiguous())
        assert np.array_equal(band[k, :n], b1.cpu().numpy()[0])
        assert np.array_equal(act[k, :n], a1.cpu().numpy()[0])
        assert np.all(band[k, n:] == 0.0) and np.all(act[k, n:] == 0)


def test_ragged_jacobian_apply_equals_single_contexts():
    P, H0, R = ragged_state(seed=13)
    rng = np.random.Generator(np.random.PCG64(4))
    v = rng.standard_normal(P.shape)
    for k, d in enumerate(PER):
        v[k, 0] = 0.0
        v[k, d["nx"] - 1:] = 0.0
    vh = rng.standard_normal(len(PER))
    Pd, H0d, Rd, vd, vhd = (torch.tensor(a, device="cuda") for a in (P, H0, R, v, vh))
    ctx = ops.Context(params(PER[0]), n_inst=len(PER), per_inst=[params(d) for d in PER])
    out = ctx.jacobian_apply(Pd, H0d, vd, vhd, rough=Rd).cpu().numpy()
    for k, d in enumerate(PER):
        n = d["nx"]
        c1 = single(k)
        o1 = c1.jacobian_apply(Pd[k:k + 1, :n].contiguous(), H0d[k:k + 1].contiguous(), vd[k:k + 1, :n].contiguous(),
                               vhd[k:k + 1].contiguous(), rough=Rd[k:k + 1, :n].contiguous())
        assert np.array_equal(out[k, :n], o1.cpu().numpy()[0])
        assert np.all(out[k, n:] == 0.0)


def test_ragged_newton_krylov_solve_matches_oracle():
    kw = dict(limiter=0, halfband=4, method=1, tol=1e-10, max_iter=60, krylov_dim=40)
    ctx = ops.Context(params(PER[0], **kw), n_inst=len(PER), per_inst=[params(d, **kw) for d in PER])
    n0 = ops.kernel_launches()
    P, H0, iters, res, code = ctx.solve(check=False)
    assert ops.kernel_launches() > n0
    assert code == 0, (code, iters.tolist(), res.tolist())
    P, H0 = P.cpu().numpy(), H0.cpu().numpy()
    for k, d in enumerate(PER):
        n = d["nx"]
        pb = lr.LineProblem(n, d["M"], d["L"], limiter="minmod")
        Pr, H0r, info = lr.solve(pb)
        assert info["converged"]
        assert P[k, 0] == 0.0 and P[k, n - 1] == 0.0
        assert np.max(np.abs(P[k, 1:n - 1] - Pr)) <= 1e-8 * np.max(Pr)
        assert abs(H0[k] - H0r) <= 1e-8 * abs(H0r)
        assert np.all(P[k, n:] == 0.0)


def test_ragged_paper_method_runs_per_group():
    """The paper's relaxation (method 0) on a ragged batch: each instance equals its single-context run."""
    kw = dict(limiter=0, halfband=4, method=0, tol=1e-9, max_iter=24)
    per = PER[:4]
    ctx = ops.Context(params(per[0], **kw), n_inst=len(per), per_inst=[params(d, **kw) for d in per])
    P, H0, iters, res, code = ctx.solve(check=False)
    P, H0, iters = P.cpu().numpy(), H0.cpu().numpy(), iters.cpu().numpy()
    for k, d in enumerate(per):
        n = d["nx"]
        c1 = ops.Context(params(d, **kw), n_inst=1)
        P1, H01, it1, res1, code1 = c1.solve(check=False)
        assert it1.cpu().numpy()[0] == iters[k]
        assert np.array_equal(P[k, :n], P1.cpu().numpy()[0])
        assert H0[k] == H01.cpu().numpy()[0]
