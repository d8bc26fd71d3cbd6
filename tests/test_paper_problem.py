"""The paper's test problem (Sec. 5) as input data, pinned without a GPU: the hand
derived right-hand side against symbolic differentiation, the discrete operator's
consistency order on the analytic solution, and second-order convergence of the
discrete solution (dense solve) to it; the oracle's preconditioned s-step GMRES from
the paper's initial guess reaches the dense discrete solution."""
import numpy as np
import pytest

from oracle import dense
from oracle import sstep as osstep
from oracle import stencil as ostencil
from paper_2001_04886_gb300 import inputs


def operator(P, N):
    a0, aw, ae, as_, an = P["coef"]
    return ostencil.Stencil((N, N), a0, [aw, as_], [ae, an])


def test_right_hand_side_matches_symbolic_differentiation():
    sp = pytest.importorskip("sympy")
    x, y = sp.symbols("x y")
    gam, bet = 50.0, 1.0
    u = x * sp.exp(x * y) * sp.sin(sp.pi * x) * sp.sin(sp.pi * y)
    b, c, d, e, f = sp.exp(-x * y), sp.exp(x * y), bet * (x + y), gam * (x + y), 1 / (1 + x * y)
    L = (-sp.diff(b * sp.diff(u, x), x) - sp.diff(c * sp.diff(u, y), y) + sp.diff(d * u, x) + sp.diff(e * u, y)
         + f * u)
    gf = sp.lambdify((x, y), L, "numpy")
    N = 9
    P = inputs.paper_problem(N)
    h = 1.0 / (N + 1)
    t = (np.arange(N) + 1) * h
    X, Y = np.meshgrid(t, t)
    np.testing.assert_allclose(P["g"], h * h * gf(X, Y).reshape(-1), rtol=1e-11, atol=1e-14)
    np.testing.assert_allclose(P["u"], sp.lambdify((x, y), u, "numpy")(X, Y).reshape(-1), rtol=1e-14, atol=1e-15)


def test_discrete_operator_is_second_order_consistent():
    errs = []
    for N in (15, 31, 63):
        P = inputs.paper_problem(N)
        A = operator(P, N)
        h = 1.0 / (N + 1)
        tau = (A.apply(P["u"]) - P["g"]) / (h * h)      # truncation error of the unscaled operator
        errs.append(np.max(np.abs(tau)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.3 < r1 < 4.7 and 3.3 < r2 < 4.7, errs


def test_discrete_solution_converges_at_second_order():
    errs = []
    for N in (15, 31):
        P = inputs.paper_problem(N)
        A = operator(P, N)
        uh = np.linalg.solve(dense.dense_matrix(A), P["g"])
        errs.append(np.max(np.abs(uh - P["u"])))
    assert 3.3 < errs[0] / errs[1] < 4.7, errs


def test_preconditioned_solve_from_the_papers_initial_guess():
    N = 31
    P = inputs.paper_problem(N)
    A = operator(P, N)
    uh = np.linalg.solve(dense.dense_matrix(A), P["g"])
    M = ostencil.RedBlackILU0(A)
    r = osstep.sstep_gmres(A, P["g"], P["x0"], 2, 10, 1e-10, 1.0, 400, precond=M)
    assert r["status"] == 0
    assert np.linalg.norm(r["x"] - uh) <= 1e-7 * np.linalg.norm(uh)
    assert P["x0"][0] == 0.05 and P["x0"][48] == 0.05 * 49 and P["x0"][49] == 0.0
