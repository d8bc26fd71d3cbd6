"""Red-black ILU(0) (the right preconditioner) in the oracle, pinned against its
definition: the factors reproduce A on its sparsity pattern, M^-1 is the dense solve
with L U, a stencil without neighbours is its own factorisation, and the preconditioned
s-step GMRES reaches the dense solution with fewer products."""
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


def dense_factors(A, P):
    D = dense.dense_matrix(A)
    red = ~P.black
    perm = np.concatenate([np.where(red)[0], np.where(P.black)[0]])
    Ap = D[np.ix_(perm, perm)]
    nr = int(red.sum())
    n = A.n
    Dr = np.diag(np.diag(Ap[:nr, :nr]))
    E, F = Ap[:nr, nr:], Ap[nr:, :nr]
    # off-diagonal blocks of the same colour are empty (every neighbour has the other colour)
    assert np.count_nonzero(Ap[:nr, :nr] - Dr) == 0 and np.count_nonzero(Ap[nr:, nr:] - np.diag(np.diag(Ap[nr:, nr:]))) == 0
    L = np.block([[np.eye(nr), np.zeros((nr, n - nr))], [F @ np.linalg.inv(Dr), np.eye(n - nr)]])
    U = np.block([[Dr, E], [np.zeros((n - nr, nr)), np.diag(P.dtilde[perm[nr:]])]])
    return Ap, L, U, perm


@pytest.mark.parametrize("A", [ostencil.convdiff((4, 4, 4), (30.0, 20.0, 10.0)), rect((5, 4, 3), (30.0, -20.0, 10.0)),
                               rect((7, 6), (20.0, -15.0)),
                               ostencil.convdiff_variable(6, 40.0 * np.random.default_rng(1).random(36))])
def test_ilu0_reproduces_a_on_its_pattern_and_applies_the_dense_inverse(A):
    P = ostencil.RedBlackILU0(A)
    Ap, L, U, perm = dense_factors(A, P)
    LU = L @ U
    pat = Ap != 0
    assert np.max(np.abs((LU - Ap)[pat])) <= 1e-14 * np.max(np.abs(Ap))
    # the only change is the dropped fill between black points two steps apart
    assert np.count_nonzero(np.abs(LU - Ap) > 1e-12) > 0
    v = inputs.x_true(3, A.n)
    want = np.zeros(A.n)
    want[perm] = np.linalg.solve(LU, v[perm])
    np.testing.assert_allclose(P.apply_inv(v), want, rtol=0, atol=1e-13 * np.max(np.abs(want)))


def test_diagonal_operator_is_its_own_factorisation():
    A = ostencil.Stencil((4, 3, 3), 5.0, [0.0] * 3, [0.0] * 3)
    P = ostencil.RedBlackILU0(A)
    v = inputs.x_true(4, A.n)
    np.testing.assert_allclose(P.apply_inv(v), v / 5.0, rtol=1e-15, atol=0)


def test_preconditioned_sstep_gmres_reaches_the_dense_solution_with_fewer_products():
    A = ostencil.convdiff((6, 6, 6), (30.0, 20.0, 10.0))
    f = A.apply(inputs.x_true(5, A.n))
    xs = np.linalg.solve(dense.dense_matrix(A), f)
    P = ostencil.RedBlackILU0(A)
    for basis in ("monomial", "newton"):
        r = osstep.sstep_gmres(A, f, np.zeros(A.n), 4, 16, 1e-12, 1.0, 200, precond=P, basis=basis)
        assert r["status"] == 0
        assert np.linalg.norm(r["x"] - xs) <= 1e-9 * np.linalg.norm(xs)
    r0 = osstep.sstep_gmres(A, f, np.zeros(A.n), 4, 16, 1e-12, 1.0 / A.norm_inf(), 200)
    r1 = osstep.sstep_gmres(A, f, np.zeros(A.n), 4, 16, 1e-12, 1.0, 200, precond=P)
    assert r1["matvecs"] < r0["matvecs"]


def test_preconditioned_sstep_orthomin_reaches_the_dense_solution_with_fewer_steps():
    N = 15
    P = inputs.paper_problem(N)
    a0, aw, ae, as_, an = P["coef"]
    A = ostencil.Stencil((N, N), a0, [aw, as_], [ae, an])
    xs = np.linalg.solve(dense.dense_matrix(A), P["g"])
    M = ostencil.RedBlackILU0(A)
    for s, k in ((1, 4), (2, 2)):
        r0 = osstep.sstep_omin(A, P["g"], P["x0"], s, k, 1e-11, 1.0 / A.norm_inf(), 100000)
        r1 = osstep.sstep_omin(A, P["g"], P["x0"], s, k, 1e-11, 1.0, 100000, precond=M)
        assert r1["status"] == 0 and r1["iters"] < r0["iters"]
        assert np.linalg.norm(r1["x"] - xs) <= 1e-9 * np.linalg.norm(xs)
