"""Pins of the convection-diffusion oracle (oracle/cd_ref.py; Sec. 3.1, Sec. 6).

* the kappa-scheme stencils against Eq. eqn42 (kappa = 0, printed) and the textbook
  second-order upwind, third-order upwind-biased and central differences
  (tests/golden/kappa_stencils.txt);
* exactness of the convective difference on polynomials: degree 2 for every kappa,
  degree 3 for kappa = 1/3 only (its truncation error is (kappa - 1/3) h^2 u''' / 4);
* the line relaxation's fixed point is the dense solution of L u = f, for both
  splittings and both line orders;
* the discrete solution converges to u = x^4 + y^4 at second order;
* the printed splittings converge with b = 0 and diverge with an upwind
  y-convection b > 0 (their line operator carries no b term).
"""
import os

import numpy as np
import pytest

from oracle import cd_ref as cd

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "kappa_stencils.txt")


def stencil(kappa, N=17, i=6):
    """a/h units of L u at interior node (i, j) for unit pulses at offsets -2..2 (b = eps = 0)."""
    pb = cd.CDProblem(N, a=1.0, b=0.0, eps=0.0, kappa=kappa)
    j = N // 2
    out = []
    for d in range(-2, 3):
        u = np.zeros((N, N))
        u[i + d, j] = 1.0
        out.append(cd.apply(pb, u)[i - 1, j - 1] * pb.h)
    return np.array(out)


def test_stencils_match_the_paper_and_the_textbook():
    rows = np.loadtxt(GOLDEN)
    for kappa, *c in rows:
        assert np.allclose(stencil(kappa), c, rtol=0, atol=1e-14), kappa


@pytest.mark.parametrize("kappa", [0.0, -1.0, 1.0 / 3.0, 0.5])
def test_convective_difference_exact_on_polynomials(kappa):
    N = 21
    pb = cd.CDProblem(N, a=1.0, b=0.0, eps=0.0, kappa=kappa)
    X = pb.x[:, None] * np.ones(N)[None, :]
    for deg in (1, 2, 3):
        u = (X - 0.3) ** deg
        du = deg * (X - 0.3) ** (deg - 1)
        err = np.max(np.abs(cd.apply(pb, u)[1:, :] - du[2:-1, 1:-1]))  # nodes i >= 2
        exact = deg <= 2 or abs(kappa - 1.0 / 3.0) < 1e-15
        if exact:
            assert err <= 1e-11, (kappa, deg, err)
        else:
            # leading term (kappa - 1/3) h^2 u''' / 4 with u''' = 6
            assert err == pytest.approx(abs(kappa - 1.0 / 3.0) * pb.h**2 * 6 / 4, rel=1e-6)
    # the first interior node (extrapolated inflow node) is exact on linear functions
    u = 2.0 * X + 1.0
    assert np.max(np.abs(cd.apply(pb, u)[0, :] - 2.0)) <= 1e-12


@pytest.mark.parametrize("splitting", ["Ls0", "Ls1"])
@pytest.mark.parametrize("order", ["lexicographic", "jacobi"])
@pytest.mark.parametrize("kappa", [0.0, 1.0 / 3.0, -1.0])
def test_relaxation_fixed_point_is_the_discrete_solution(splitting, order, kappa):
    pb = cd.CDProblem(17, kappa=kappa, eps=1e-3)
    ud = cd.solve_direct(pb)
    u, hist = cd.line_relaxation(pb, splitting, order=order, sweeps=200, tol=1e-12)
    assert hist[-1] <= 1e-12
    assert np.max(np.abs(u - ud)) <= 1e-11 * np.max(np.abs(ud))


def test_second_order_convergence_to_the_exact_solution():
    for kappa in (0.0, 1.0 / 3.0, -1.0):
        errs = []
        for N in (17, 33, 65):
            pb = cd.CDProblem(N, kappa=kappa)
            u, hist = cd.line_relaxation(pb, "Ls0", sweeps=200, tol=1e-12)
            errs.append(np.max(np.abs(u - pb.u_exact)))
        p = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
        assert np.all(p > 1.7) and np.all(p < 2.3), (kappa, errs)


def test_residual_decay_with_and_without_y_convection():
    pb = cd.CDProblem(33, kappa=0.0)
    _, hist = cd.line_relaxation(pb, "Ls0", sweeps=12)
    assert hist[-1] <= 1e-4 * hist[0]
    pb = cd.CDProblem(33, kappa=0.0, b=1.0)
    _, hist = cd.line_relaxation(pb, "Ls0", sweeps=6)
    assert hist[-1] > 1e3 * hist[0]


GOLDEN_L0 = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cd_line_operators.txt")


def _line_operator_pin_holds():
    """Every row of cd_ref.line_matrix against the printed L^0 of Eqs. eqn48 (Ls0) and eqn49 (Ls1)."""
    ok = True
    for split, kappa, cm, c0, cp, dm, d0, dp in np.loadtxt(GOLDEN_L0):
        for a, eps in ((1.0, 1e-6), (0.7, 3e-3)):
            pb = cd.CDProblem(17, a=a, eps=eps, kappa=kappa)
            A = cd.line_matrix(pb, "Ls0" if split == 0 else "Ls1")
            want = [c * a / pb.h + d * eps / pb.h**2 for c, d in ((cm, dm), (c0, d0), (cp, dp))]
            for i in range(1, A.shape[0] - 1):
                got = [A[i, i - 1], A[i, i], A[i, i + 1]]
                ok = ok and all(abs(g - w) <= 1e-12 * max(1.0, abs(w)) for g, w in zip(got, want))
            ok = ok and abs(A[0, 0] - want[1]) <= 1e-12 * abs(want[1]) and not np.any(np.triu(A, 2))
    return ok


def test_line_operator_is_the_printed_one():
    """L^0 of the x-line splittings as Sec. 3.1 prints them (Eqs. eqn48, eqn49), at four kappa and
    two (a, eps): the tridiagonal rows, and nothing beyond the first super-diagonal."""
    assert _line_operator_pin_holds()


@pytest.mark.parametrize("slip", ["ls0_as_ls1", "diffusion_diagonal_2", "kappa_sign"])
def test_line_operator_pin_catches_planted_mistakes(monkeypatch, slip):
    """Plausible slips in the splittings' coefficient, planted in the oracle, fail the pin."""
    good = cd.l0_coefficient
    if slip == "ls0_as_ls1":
        monkeypatch.setattr(cd, "l0_coefficient", lambda kappa, s: good(kappa, "Ls1"))
        assert not _line_operator_pin_holds()
    elif slip == "kappa_sign":
        monkeypatch.setattr(cd, "l0_coefficient", lambda kappa, s: good(-kappa, s))
        assert not _line_operator_pin_holds()
    else:  # a 1-D diffusion diagonal (2 eps / h^2) in place of the 5-point one
        real = cd.line_matrix

        def slipped(pb, s):
            A = real(pb, s)
            return A - 2.0 * pb.eps / pb.h**2 * np.eye(A.shape[0])

        monkeypatch.setattr(cd, "line_matrix", slipped)
        assert not _line_operator_pin_holds()
