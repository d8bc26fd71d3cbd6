"""The Newton basis without a GPU: the oracle's Leja ordering and shift pins, and the
library's host-side shift computation (its own Hessenberg QR) against the oracle's
(LAPACK eigenvalues)."""
import numpy as np

import __graft_entry__ as entry
from oracle import sstep as osstep
from oracle import stencil as ostencil
from paper_2001_04886_gb300 import inputs


def test_leja_order_hand_example():
    # largest modulus first; then 0.1 is farthest from 1.7; then 0.9 (0.8 x 0.8 = 0.64 >
    # 1.2 x 0.4 = 0.48); then 0.5; then the sequence repeats
    assert osstep.leja_order([0.1, 0.5, 0.9, 1.7], 6) == [1.7, 0.1, 0.9, 0.5, 1.7, 0.1]
    # a repeated value (or one within 1e-10 max|v|, as the real parts of a complex pair) is taken once
    assert osstep.leja_order([2.0, 2.0, -1.0], 3) == [2.0, -1.0, 2.0]
    assert osstep.leja_order([2.0, 2.0 + 1e-12, -1.0], 3) == [2.0 + 1e-12, -1.0, 2.0 + 1e-12]


def test_zero_shifts_are_the_monomial_basis_and_shifted_powers_span_the_same_space():
    A = ostencil.convdiff((6, 6, 6), (30.0, 20.0, 10.0))
    v = inputs.x_true(1, A.n)
    sig = 1.0 / A.norm_inf()
    Y0 = osstep.matrix_powers(A, v, 4, sig)
    np.testing.assert_array_equal(osstep.matrix_powers(A, v, 4, sig, shifts=[0.0] * 4), Y0)
    Y1 = osstep.matrix_powers(A, v, 4, sig, shifts=[3.0, 7.5, 1.0, 9.0])
    # every shifted column lies in the span of the monomial ones (and vice versa)
    Q, _ = np.linalg.qr(Y0)
    assert np.linalg.norm(Y1 - Q @ (Q.T @ Y1)) <= 1e-10 * np.linalg.norm(Y1)


def test_newton_gmres_relation_and_solution():
    """With Newton shifts the assembly's theta terms keep A V = U G (a traced shifted
    cycle), the solve reaches the dense solution, and the shifts, real parts of Ritz
    values, lie in the real part of the field of values [lambda_min, lambda_max] of the
    symmetric part of A; for a symmetric A, inside its spectrum (interlacing)."""
    from oracle import dense

    for beta in ((30.0, 20.0, 10.0), (0.0, 0.0, 0.0)):
        A = ostencil.convdiff((5, 5, 5), beta)
        D = dense.dense_matrix(A)
        f = A.apply(inputs.x_true(2, A.n))
        xs = np.linalg.solve(D, f)
        r = osstep.sstep_gmres(A, f, np.zeros(A.n), 4, 16, 1e-12, 1.0 / A.norm_inf(), 100, basis="newton")
        assert r["status"] == 0 and r["shifts"] is not None
        assert np.linalg.norm(r["x"] - xs) <= 1e-9 * np.linalg.norm(xs)
        lam = np.linalg.eigvalsh(0.5 * (D + D.T))
        assert min(r["shifts"]) >= lam[0] - 1e-9 and max(r["shifts"]) <= lam[-1] + 1e-9
        tr = {}
        osstep.sstep_gmres(A, f, np.zeros(A.n), 4, 16, 1e-14, 1.0 / A.norm_inf(), 1, trace=tr, basis="newton",
                           shifts=r["shifts"])
        U, G = tr["U"], tr["G"]
        AV = np.column_stack([A.apply(U[:, j]) for j in range(G.shape[1])])
        assert np.linalg.norm(AV - U @ G) <= 1e-10 * np.linalg.norm(AV)
        # the same check fails if the theta terms are left out of G (the pin has teeth)
        assert np.linalg.norm(AV - U @ _without_shift_terms(G, U, r["shifts"], 4)) > 1e-6 * np.linalg.norm(AV)


def _without_shift_terms(G, U, shifts, s):
    # G minus theta_j e_{o+j} in column o+j (the block-k part of the shift term)
    G2 = G.copy()
    for c in range(G.shape[1]):
        G2[c, c] -= shifts[c % s]
    return G2


def test_library_shifts_match_the_oracle():
    entry.build()
    import paper_2001_04886_gb300 as pkg

    rng = np.random.default_rng(5)
    # a first-cycle Hessenberg from the oracle (nonsymmetric operator, real spectrum)
    A = ostencil.convdiff((8, 8, 8), (30.0, 20.0, 10.0))
    f = A.apply(inputs.x_true(0, A.n))
    tr = {}
    osstep.sstep_gmres(A, f, np.zeros(A.n), 4, 24, 1e-12, 1.0 / A.norm_inf(), 1, trace=tr)
    G = tr["G"]
    K = G.shape[1]
    want = osstep.newton_shifts(G, K, 4)
    got = pkg.sstep_newton_shifts(G, K, 4)
    np.testing.assert_allclose(got, want, rtol=1e-9, atol=1e-12)
    # random upper Hessenberg matrices, with complex eigenvalue pairs
    for n in (3, 7, 12, 20):
        H = np.triu(rng.standard_normal((n, n)), -1)
        want = osstep.leja_order(np.sort(np.linalg.eigvals(H).real), 8)
        got = pkg.sstep_newton_shifts(H, n, 8)
        np.testing.assert_allclose(got, want, rtol=1e-8, atol=1e-10)
