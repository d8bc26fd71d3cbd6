"""Dense matrices of tiny stencil operators and a direct solve (brute-force pins only).

The dense matrix is assembled entry by entry from the row definition of the
stencil (centre, then the minus/plus neighbour of each dimension that lies
inside the grid), independently of Stencil.apply's array shifts.
"""
from __future__ import annotations

import numpy as np


def dense_matrix(St):
    n = St.n
    shape = St.shape
    dim = St.dim
    strides = [1, shape[0], shape[0] * (shape[1] if dim > 1 else 1)][:dim]
    A = np.zeros((n, n))

    def coef(c, p):
        return float(c) if np.isscalar(c) else float(np.asarray(c).reshape(-1)[p])

    for p in range(n):
        idx = []
        rem = p
        for d in range(dim):
            idx.append(rem % shape[d])
            rem //= shape[d]
        A[p, p] = coef(St.a0, p)
        for d in range(dim):
            if idx[d] > 0:
                A[p, p - strides[d]] += coef(St.am[d], p)
            if idx[d] < shape[d] - 1:
                A[p, p + strides[d]] += coef(St.ap[d], p)
    return A


def gauss_solve(A, b):
    """Gaussian elimination with partial pivoting (row swaps), then back substitution."""
    M = np.array(A, dtype=np.float64, copy=True)
    x = np.array(b, dtype=np.float64, copy=True)
    n = M.shape[0]
    for c in range(n):
        piv = c + int(np.argmax(np.abs(M[c:, c])))
        if piv != c:
            M[[c, piv]] = M[[piv, c]]
            x[[c, piv]] = x[[piv, c]]
        for r in range(c + 1, n):
            l = M[r, c] / M[c, c]
            M[r, c:] -= l * M[c, c:]
            x[r] -= l * x[c]
    for r in range(n - 1, -1, -1):
        x[r] = (x[r] - M[r, r + 1 :] @ x[r + 1 :]) / M[r, r]
    return x
