"""The parity bar of the first block's residual history (no arithmetic of the method).

The first s least-squares estimates of an s-step GMRES cycle (Alg. 4.1, eq. 9) come from
the Cholesky factor of W_1, the Gram matrix of the first block's scaled monomial powers,
and move by about cond(W_1) times the relative error of W_1. The oracle forms W_1 with
FP64 BLAS sums, which are accurate to a few u = 2^-53; the library forms it with exact
fixed-point sums rounded once. Measured against the same oracle with an extended-precision
W_1, the oracle's own first-block estimates move by up to 1.9 u cond(W_1)
(tests/test_parity_bar.py). Two implementations that each round W_1 differently therefore
agree there to 4 u cond(W_1), and to 1e-10 wherever that is the larger bar.

Over the rest of the cycle the estimates fall by orders of magnitude while their rounding
error stays of the size it had in the first block, so the later entries are compared in
absolute terms, against the cycle's first entry: the oracle's own estimates move by at
most 0.045 u cond(W_1) of it when every Gram matrix and inner product of the cycle is
summed in extended precision, and the bar is 0.1 u cond(W_1) (or 1e-6 relative, where that
is larger). The iterate after the cycle moves by at most 0.37 u cond(W_1) relative in the
same experiment; the bar is max(1e-8, u cond(W_1)).
"""
U53 = 2.0 ** -53
FACTOR = 4.0


def first_block_tol(cond_w1, u=U53):
    """Relative bar on the first s history entries, for a first-block Gram condition cond_w1."""
    return max(1e-10, FACTOR * u * float(cond_w1))


def cycle_abs_tol(cond_w1, u=U53):
    """Absolute bar on every history entry of a cycle, in units of the cycle's first entry."""
    return 0.1 * u * float(cond_w1)


def cycle_x_tol(cond_w1, u=U53):
    """Relative bar on the iterate after one restart cycle."""
    return max(1e-8, u * float(cond_w1))
