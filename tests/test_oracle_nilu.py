"""ILU(0) in the natural ordering (the paper's preconditioner, Sec. 5) in the oracle,
pinned against its definition and against exact special cases:

  * the factors reproduce A on its sparsity pattern, and differ from A only by fill
    entries outside it;
  * M^-1 is the dense solve with L U;
  * on a one-row grid the operator is tridiagonal, ILU(0) drops nothing and M^-1 is A^-1;
  * with no coupling in one dimension the 2-D factorisation is the 1-D one, line by line;
  * the preconditioned solvers reach the dense solution, with fewer products than the
    red-black ILU(0) (the natural ordering is the stronger preconditioner);
  * slips planted in a copy (sign of the pivot update, the wrong row's coefficient, a
    missing pivot division) fail these pins.
"""
import copy

import numpy as np
import pytest

from oracle import dense
from oracle import sstep as osstep
from oracle import stencil as ostencil
from paper_2001_04886_gb300 import inputs


def rect(shape, beta):
    h = 1.0 / (shape[0] + 1)
    c = [b * h / 2 for b in beta]
    return ostencil.Stencil(shape, 2.0 * len(shape), [-1 - cd for cd in c], [-1 + cd for cd in c])


def random_stencil(shape, seed):
    rng = np.random.default_rng(seed)
    n = int(np.prod(shape))
    dim = len(shape)
    a0 = 2.0 * dim + rng.random(n)
    am = [-1.0 - 0.4 * rng.random(n) for _ in range(dim)]
    ap = [-1.0 + 0.4 * rng.random(n) for _ in range(dim)]
    return ostencil.Stencil(shape, a0, am, ap)


def dense_factors(A, P):
    """L (unit lower) and U from the factor arrays, entry by entry."""
    n = A.n
    L = np.eye(n)
    U = np.diag(P.d)
    for k in range(A.dim):
        st = P.stride[k]
        for p in range(n):
            if P.coord[k][p] > 0:
                L[p, p - st] = P.L[k][p]
            if P.coord[k][p] < A.shape[k] - 1:
                U[p, p + st] = P.ap[k][p]
    return L, U


CASES = [ostencil.convdiff((6, 6), (20.0, 10.0)), rect((7, 5), (20.0, -15.0)),
         ostencil.convdiff((4, 4, 4), (30.0, 20.0, 10.0)), rect((5, 4, 3), (30.0, -20.0, 10.0)),
         random_stencil((6, 5), 3), random_stencil((4, 3, 3), 4),
         ostencil.convdiff_variable(6, 40.0 * np.random.default_rng(1).random(36))]


def check_pins(A, P):
    D = dense.dense_matrix(A)
    L, U = dense_factors(A, P)
    assert np.allclose(np.tril(L, -1) != 0, np.tril(D, -1) != 0) and np.allclose(np.triu(U, 1) != 0, np.triu(D, 1) != 0)
    LU = L @ U
    pat = D != 0
    assert np.max(np.abs((LU - D)[pat])) <= 1e-14 * np.max(np.abs(D))
    v = inputs.x_true(3, A.n)
    want = np.linalg.solve(LU, v)
    got = P.apply_inv(v)
    assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))
    return LU, D


@pytest.mark.parametrize("A", CASES)
def test_factors_reproduce_a_on_its_pattern_and_apply_the_dense_inverse(A):
    P = ostencil.NaturalILU0(A)
    LU, D = check_pins(A, P)
    # a grid with more than one line in two dimensions has fill: L U differs from A there
    off = ~(D != 0)
    assert np.count_nonzero(np.abs(LU - D)[off] > 1e-12) > 0


@pytest.mark.parametrize("N", [1, 2, 9, 40])
def test_one_row_grid_is_an_exact_factorisation(N):
    A = random_stencil((N, 1), 11 + N)
    P = ostencil.NaturalILU0(A)
    x = inputs.x_true(6, A.n)
    np.testing.assert_allclose(P.apply_inv(A.apply(x)), x, rtol=0, atol=1e-13 * np.max(np.abs(x)))
    L, U = dense_factors(A, P)
    np.testing.assert_allclose(L @ U, dense.dense_matrix(A), rtol=0, atol=1e-14 * 3)


def test_uncoupled_lines_factor_as_independent_tridiagonal_systems():
    """With no y coupling the 2-D factors are those of each x line on its own."""
    rng = np.random.default_rng(5)
    nx, ny = 7, 4
    n = nx * ny
    a0, amx, apx = 3.0 + rng.random(n), -1.0 - rng.random(n) * 0.3, -1.0 + rng.random(n) * 0.3
    A = ostencil.Stencil((nx, ny), a0, [amx, np.zeros(n)], [apx, np.zeros(n)])
    P = ostencil.NaturalILU0(A)
    for j in range(ny):
        sl = slice(j * nx, (j + 1) * nx)
        A1 = ostencil.Stencil((nx, 1), a0[sl], [amx[sl], np.zeros(nx)], [apx[sl], np.zeros(nx)])
        P1 = ostencil.NaturalILU0(A1)
        np.testing.assert_array_equal(P.d[sl], P1.d)


def test_preconditioned_solvers_reach_the_dense_solution_with_fewer_products_than_red_black():
    N = 15
    Pp = inputs.paper_problem(N)
    a0, aw, ae, as_, an = Pp["coef"]
    A = ostencil.Stencil((N, N), a0, [aw, as_], [ae, an])
    xs = np.linalg.solve(dense.dense_matrix(A), Pp["g"])
    nat, rb = ostencil.NaturalILU0(A), ostencil.RedBlackILU0(A)
    for s in (1, 2):
        r_n = osstep.sstep_gmres(A, Pp["g"], Pp["x0"], s, 10, 1e-11, 1.0, 400, precond=nat)
        r_r = osstep.sstep_gmres(A, Pp["g"], Pp["x0"], s, 10, 1e-11, 1.0, 400, precond=rb)
        assert r_n["status"] == 0 and np.linalg.norm(r_n["x"] - xs) <= 1e-9 * np.linalg.norm(xs)
        assert r_n["matvecs"] < r_r["matvecs"]
    for s, k in ((1, 4), (2, 2)):
        r_n = osstep.sstep_omin(A, Pp["g"], Pp["x0"], s, k, 1e-11, 1.0, 100000, precond=nat)
        r_r = osstep.sstep_omin(A, Pp["g"], Pp["x0"], s, k, 1e-11, 1.0, 100000, precond=rb)
        assert r_n["status"] == 0 and np.linalg.norm(r_n["x"] - xs) <= 1e-9 * np.linalg.norm(xs)
        assert r_n["iters"] < r_r["iters"]


class _SignSlip(ostencil.NaturalILU0):
    """Pivot update added instead of subtracted."""

    def __init__(self, A):
        super().__init__(A)
        n = A.n
        d = np.zeros(n)
        for p in range(n):
            dp = self.a0[p]
            for k in range(A.dim):
                if self.coord[k][p] > 0:
                    q = p - self.stride[k]
                    dp += self.am[k][p] * self.ap[k][q] / d[q]
            d[p] = dp
        self.d = d
        for k in range(A.dim):
            self.L[k] = np.where(self.coord[k] > 0, self.am[k] / np.roll(d, self.stride[k]), 0.0)


class _RowSlip(ostencil.NaturalILU0):
    """A[p, p + e_d] (the row's own coefficient) in place of A[p - e_d, p] in the pivots."""

    def __init__(self, A):
        super().__init__(A)
        n = A.n
        d = np.zeros(n)
        for p in range(n):
            dp = self.a0[p]
            for k in range(A.dim):
                if self.coord[k][p] > 0:
                    q = p - self.stride[k]
                    dp -= self.am[k][p] * self.ap[k][p] / d[q]
            d[p] = dp
        self.d = d
        for k in range(A.dim):
            self.L[k] = np.where(self.coord[k] > 0, self.am[k] / np.roll(d, self.stride[k]), 0.0)


class _PivotSlip(ostencil.NaturalILU0):
    """L without the division by the pivot."""

    def __init__(self, A):
        super().__init__(A)
        for k in range(A.dim):
            self.L[k] = np.where(self.coord[k] > 0, self.am[k], 0.0)


@pytest.mark.parametrize("slip", [_SignSlip, _RowSlip, _PivotSlip])
def test_planted_slips_fail_the_pins(slip):
    A = random_stencil((6, 5), 8)
    with pytest.raises(AssertionError):
        check_pins(A, slip(A))
