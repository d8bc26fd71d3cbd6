"""Pins for the oracle's solvers: brute force, the paper's equivalences, invariants.

Each test ties the oracle to something other than itself: a direct dense solve,
a different algorithm the paper proves equivalent, or an invariant the method
guarantees. A plausible slip (a dropped projection term, a wrong window index,
a transposed Gram block, a missing 1/sigma) breaks at least one of them.
"""
import numpy as np
import pytest

from oracle import STATUS_BREAKDOWN, STATUS_OK, dense, krylov, sstep, stencil
from paper_2001_04886_gb300 import inputs


def system(shape, beta, seed=0):
    A = stencil.convdiff(shape, beta)
    xt = inputs.x_true(seed, A.n)
    return A, A.apply(xt), xt


TINY = [((4, 4), (20.0, 20.0)), ((5, 5), (20.0, 20.0)), ((3, 3, 3), (6.0, 4.0, 2.0)), ((4, 4, 4), (8.0, 6.0, 4.0))]


@pytest.mark.parametrize("shape,beta", TINY)
def test_brute_force_dense_solution(shape, beta):
    """P3: every solver reaches the dense Gaussian-elimination solution on tiny grids."""
    A, f, _ = system(shape, beta)
    xs = dense.gauss_solve(dense.dense_matrix(A), f)
    n = A.n
    z = np.zeros(n)
    sig = 1.0 / A.norm_inf()
    runs = [
        krylov.gmres(A, f, z, n, 1e-13, 5),
        krylov.gmres(A, f, z, 8, 1e-13, 200, orth="mgs"),
        krylov.omin(A, f, z, 3, 1e-13, 5000),
        sstep.sstep_gmres(A, f, z, 1, 8, 1e-13, sig, 200),
        sstep.sstep_gmres(A, f, z, 2, 8, 1e-13, sig, 200),
        sstep.sstep_gmres(A, f, z, 4, 8, 1e-13, sig, 200),
        sstep.sstep_omin(A, f, z, 2, 1, 1e-13, sig, 5000),
        sstep.sstep_omin(A, f, z, 3, 2, 1e-13, sig, 5000),
    ]
    for res in runs:
        assert res["status"] == STATUS_OK
        assert np.linalg.norm(res["x"] - xs) <= 1e-10 * np.linalg.norm(xs)


def test_full_gmres_terminates_within_n_steps():
    """GMRES(m = n) without restart is exact after at most n Arnoldi steps."""
    A, f, _ = system((4, 4), (20.0, 20.0))
    res = krylov.gmres(A, f, np.zeros(A.n), A.n, 1e-12, 1)
    assert res["status"] == STATUS_OK and res["iters"] <= A.n


def gm_steps(h, m, cycles):
    """Per-step estimates of the first `cycles` full GMRES(m) cycles (drop restart entries)."""
    out = []
    for c in range(cycles):
        out.extend(h[c * (m + 1) + 1 : (c + 1) * (m + 1)])
    return np.array(out)


@pytest.mark.parametrize("shape,beta,m", [((24, 24), (20.0, 20.0), 12), ((10, 10, 10), (30.0, 20.0, 10.0), 16)])
def test_sstep_gmres_reduces_to_gmres(shape, beta, m):
    """P4: s = 1 is GMRES (Sec. 4), and s > 1 gives the same iterates in exact arithmetic (Remark 4.1)."""
    A, f, _ = system(shape, beta)
    z = np.zeros(A.n)
    sig = 1.0 / A.norm_inf()
    ref = krylov.gmres(A, f, z, m, 1e-30, 2)
    h0 = gm_steps(ref["history"], m, 2)
    for s, tol in [(1, 1e-11), (2, 1e-9), (4, 1e-8)]:
        res = sstep.sstep_gmres(A, f, z, s, m, 1e-30, sig, 2)
        h = gm_steps(res["history"], m, 2)
        assert np.max(np.abs(h - h0) / h0) <= tol, s
        assert np.linalg.norm(res["x"] - ref["x"]) <= 1e-8 * np.linalg.norm(ref["x"])


def test_sigma_leaves_iterates_unchanged():
    """Scaling the powers by sigma does not change the Krylov space (Sec. 4 basis)."""
    A, f, _ = system((16, 16), (20.0, 20.0))
    z = np.zeros(A.n)
    a = sstep.sstep_gmres(A, f, z, 2, 8, 1e-30, 1.0, 2)
    b = sstep.sstep_gmres(A, f, z, 2, 8, 1e-30, 1.0 / 8.0, 2)
    assert np.max(np.abs(np.array(a["history"]) - b["history"]) / np.array(b["history"])) < 1e-8


@pytest.mark.parametrize("k", [1, 2, 3])
def test_sstep_omin_s1_is_omin(k):
    """P5: s = 1 in Algorithm 3.1 is Orthomin(k) of Algorithm 2.1 (Sec. 3)."""
    A, f, _ = system((20, 20), (20.0, 20.0))
    z = np.zeros(A.n)
    a = krylov.omin(A, f, z, k, 1e-8, 2000)
    b = sstep.sstep_omin(A, f, z, 1, k, 1e-8, 0.125, 2000)
    assert a["iters"] == b["iters"]
    # the last entry is the explicit residual that confirms convergence
    ha, hb = np.array(a["history"][:-1]), np.array(b["history"][:-1])
    assert np.max(np.abs(ha - hb) / ha) < 1e-10
    assert abs(a["history"][-1] - b["history"][-1]) <= 1e-6 * a["history"][-1]


@pytest.mark.parametrize("s", [2, 3, 4])
def test_sstep_omin_k0_is_restarted_gmres_s(s):
    """P5: with an empty window each s-step minimises over x_i + K_s(A, r_i): GMRES(s) restarted (s-MR, Sec. 3)."""
    A, f, _ = system((16, 16), (20.0, 20.0))
    z = np.zeros(A.n)
    om = sstep.sstep_omin(A, f, z, s, 0, 1e-30, 1.0 / 8.0, 12)
    gm = krylov.gmres(A, f, z, s, 1e-30, 12)
    restarts = np.array(gm["history"][:: s + 1][:12])
    steps = np.array(om["history"][:12])
    assert np.max(np.abs(restarts - steps) / restarts) < 1e-9


def test_gcr_equals_gmres():
    """P6: Orthomin with an unbounded window (GCR, j_i = 0) matches unrestarted GMRES step by step (Sec. 2)."""
    A, f, _ = system((14, 14), (20.0, 20.0))
    z = np.zeros(A.n)
    gcr = krylov.omin(A, f, z, 10_000, 1e-10, 60)
    gm = krylov.gmres(A, f, z, 60, 1e-10, 1)
    j = min(30, len(gcr["history"]) - 2)
    a = np.array(gcr["history"][1 : j + 1])
    b = np.array(gm["history"][1 : j + 1])
    assert np.max(np.abs(a - b) / b) < 1e-8


def test_sstep_omin1_is_sstep_gcr_for_symmetric():
    """P5: for symmetric A, s-step Omin(1) coincides with s-step GCR (Sec. 3)."""
    A, f, _ = system((16, 16), (0.0, 0.0))
    z = np.zeros(A.n)
    a = sstep.sstep_omin(A, f, z, 3, 1, 1e-9, 0.125, 200)
    b = sstep.sstep_omin(A, f, z, 3, 10_000, 1e-9, 0.125, 200)
    n = min(len(a["history"]), len(b["history"]), 25)
    ha, hb = np.array(a["history"][:n]), np.array(b["history"][:n])
    assert np.max(np.abs(ha - hb) / hb) < 1e-7


def test_invariants_sstep_gmres():
    """P7: mutually orthogonal blocks, D = U^T U block diagonal, and A V = U G (eq. 5)."""
    A, f, _ = system((20, 20), (20.0, 20.0))
    tr = {}
    s, m = 4, 16
    sig = 0.125
    sstep.sstep_gmres(A, f, np.zeros(A.n), s, m, 1e-30, sig, 1, trace=tr)
    U, G, W = tr["U"], tr["G"], tr["W"]
    K = G.shape[1]
    D = U.T @ U
    Dexp = np.zeros_like(D)
    for i, w in enumerate(W):
        Dexp[i * s : (i + 1) * s, i * s : (i + 1) * s] = w
    Dexp[K, K] = 1.0
    assert np.max(np.abs(D - Dexp)) <= 1e-10
    AV = np.column_stack([A.apply(U[:, j]) for j in range(K)])
    assert np.linalg.norm(AV - U @ G) <= 1e-10 * np.linalg.norm(AV)
    assert np.allclose(np.tril(G, -2), 0.0)            # upper Hessenberg


def test_invariants_sstep_omin():
    """P7: A P blocks in the window are A^T A-orthogonal, residuals never grow."""
    A, f, _ = system((20, 20), (20.0, 20.0))
    tr = {}
    res = sstep.sstep_omin(A, f, np.zeros(A.n), 3, 2, 1e-9, 0.125, 40, trace=tr)
    AP = tr["AP"]
    assert len(AP) == 2
    X = AP[0].T @ AP[1]
    scale = np.sqrt(np.outer(np.sum(AP[0] ** 2, 0), np.sum(AP[1] ** 2, 0)))
    assert np.max(np.abs(X) / scale) <= 1e-11
    h = np.array(res["history"][:-1])                   # updated residuals; the last is explicit
    assert np.all(np.diff(h) <= 1e-15 * h[:-1])


def test_monotone_and_final_residual():
    """P7/P8: GMRES estimates never grow within a cycle; the final explicit residual meets tol."""
    A, f, _ = system((32, 32), (20.0, 20.0))
    z = np.zeros(A.n)
    for res in [krylov.gmres(A, f, z, 10, 1e-8), sstep.sstep_gmres(A, f, z, 2, 10, 1e-8, 0.125),
                sstep.sstep_omin(A, f, z, 4, 1, 1e-8, 0.125), krylov.omin(A, f, z, 2, 1e-8)]:
        assert res["status"] == STATUS_OK
        # estimates and updated residuals never grow; explicit recomputations may
        # differ from them by rounding (relative 1e-6 allowed)
        h = np.array(res["history"])
        assert np.all(np.diff(h) <= 1e-6 * h[:-1])
        assert np.linalg.norm(f - A.apply(res["x"])) / np.linalg.norm(f) <= 1e-8


def test_breakdown_on_zero_power():
    """An all-zero power block (A r = 0 impossible for nonsingular A) is simulated with A = 0."""
    A = stencil.Stencil((3, 3), 0.0, [0.0, 0.0], [0.0, 0.0])
    f = np.ones(9)
    res = sstep.sstep_gmres(A, f, np.zeros(9), 2, 4, 1e-8, 1.0, 3)
    assert res["status"] == STATUS_BREAKDOWN
    res = sstep.sstep_omin(A, f, np.zeros(9), 2, 1, 1e-8, 1.0, 3)
    assert res["status"] == STATUS_BREAKDOWN


def test_cholesky_helpers():
    rng = np.random.default_rng(5)
    M = rng.standard_normal((6, 6))
    W = M.T @ M + 0.1 * np.eye(6)
    L = sstep.cholesky_upper(W)
    assert np.allclose(L.T @ L, W, atol=1e-13) and np.allclose(np.tril(L, -1), 0)
    b = rng.standard_normal((6, 2))
    assert np.allclose(sstep.cholesky_solve(L, b), np.linalg.solve(W, b), atol=1e-10)
    assert sstep.cholesky_upper(-np.eye(3)) is None


def test_zero_right_hand_side():
    """f = 0: A is nonsingular, so x = 0 is the solution. From x0 = 0 every solver ends
    at the first residual (one product, relres 0); from x0 != 0 the test is made on
    ||A x|| itself and the iterate goes to 0."""
    A, _, _ = system((6, 6), (20.0, 20.0))
    f, z = np.zeros(A.n), np.zeros(A.n)
    for res in (krylov.gmres(A, f, z, 10, 1e-8), krylov.omin(A, f, z, 2, 1e-8),
                sstep.sstep_gmres(A, f, z, 4, 20, 1e-8, 0.125), sstep.sstep_omin(A, f, z, 2, 1, 1e-8, 0.125)):
        assert res["status"] == STATUS_OK and res["history"] == [0.0] and res["matvecs"] == 1
        assert not np.any(res["x"]) and res["relres"] == 0.0
    x0 = inputs.x_true(3, A.n)
    r = sstep.sstep_gmres(A, f, x0, 4, 20, 1e-10, 0.125)
    assert r["status"] == STATUS_OK and np.linalg.norm(A.apply(r["x"])) <= 1e-10


def test_lucky_breakdown_and_degenerate_block():
    """A = I: the Krylov space of f has dimension 1. GMRES (and s-step GMRES with s = 1)
    meets the lucky breakdown (h_21 = 0, nu = 0) and returns x = f exactly after one
    step; a block of s = 2 monomial powers is then linearly dependent, its Gram matrix
    singular, and the method reports a breakdown (status -4) without taking a step."""
    n = 25
    A = stencil.Stencil((5, 5), np.ones(n), [np.zeros(n), np.zeros(n)], [np.zeros(n), np.zeros(n)])
    f = inputs.x_true(4, n)
    z = np.zeros(n)
    for res in (krylov.gmres(A, f, z, 10, 1e-12), sstep.sstep_gmres(A, f, z, 1, 10, 1e-12, 1.0)):
        assert res["status"] == STATUS_OK and res["iters"] == 1
        assert np.allclose(res["x"], f, rtol=0, atol=1e-15)
    bad = sstep.sstep_gmres(A, f, z, 2, 10, 1e-12, 1.0)
    assert bad["status"] == STATUS_BREAKDOWN and bad["iters"] == 0


def test_givens_least_squares_equals_lstsq():
    """eq. 2-3: the Givens QR of an upper Hessenberg H, column by column, gives after every
    column the residual norm and (at the end) the minimiser of ||g0 e1 - H y|| that a
    dense least-squares solve (LAPACK) gives; a column with a zero subdiagonal is the
    lucky breakdown (residual 0)."""
    rng = np.random.default_rng(11)
    for m in (1, 5, 20, 40):
        H = np.triu(rng.standard_normal((m + 1, m)), -1)
        H[np.arange(m), np.arange(m)] += 4.0      # well conditioned, so y is compared tightly
        g0 = 2.5
        lsq = krylov.GivensLSQ(m, g0)
        for j in range(m):
            est = lsq.add_column(H[:, j])
            rhs = np.zeros(j + 2)
            rhs[0] = g0
            y, *_ = np.linalg.lstsq(H[: j + 2, : j + 1], rhs, rcond=None)
            true = np.linalg.norm(rhs - H[: j + 2, : j + 1] @ y)
            assert abs(est - true) <= 1e-12 * g0, (m, j)
        assert np.allclose(lsq.solve(), y, rtol=1e-9, atol=1e-12)
    H = np.array([[2.0, 1.0], [0.0, 3.0], [0.0, 0.0]])
    lsq = krylov.GivensLSQ(2, 1.0)
    lsq.add_column(H[:, 0])
    assert lsq.add_column(H[:, 1]) == 0.0
