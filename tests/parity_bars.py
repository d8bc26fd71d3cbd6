"""The parity bar of the first block's residual history (no arithmetic of the method).

The first s least-squares estimates of an s-step GMRES cycle (Alg. 4.1, eq. 9) come from
the Cholesky factor of W_1, the Gram matrix of the first block's scaled monomial powers,
and move by about cond(W_1) times the relative error of W_1. The oracle forms W_1 with
FP64 BLAS sums, which are accurate to a few u = 2^-53; the library forms it with exact
fixed-point sums rounded once. Measured against the same oracle with an extended-precision
W_1, the oracle's own first-block estimates move by up to 1.9 u cond(W_1)
(tests/test_parity_bar.py). Two implementations that each round W_1 differently therefore
agree there to 4 u cond(W_1), and to 1e-10 wherever that is the larger bar.
"""
U53 = 2.0 ** -53
FACTOR = 4.0


def first_block_tol(cond_w1, u=U53):
    """Relative bar on the first s history entries, for a first-block Gram condition cond_w1."""
    return max(1e-10, FACTOR * u * float(cond_w1))
