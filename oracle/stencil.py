"""The operator A: h^2-scaled centred-difference convection-diffusion stencils.

Sec. 1 motivates the block-tridiagonal matrices that come from PDEs on regular
grids; Sec. 5 (eq. 10) discretises a convection-diffusion operator with the
five-point Laplacian and centred first differences. Unknowns are the interior
nodes of an N_1 x ... x N_d grid with spacing h = 1/(N+1), ordered
lexicographically with x fastest, and neighbours outside the grid are zero
(homogeneous Dirichlet).

Row p of the h^2-scaled operator for -Lap u + sum_d beta_d du/dx_d is
    2d u_p + sum_d [ (-1 - c_d) u_{p - e_d} + (-1 + c_d) u_{p + e_d} ],
with c_d = beta_d h / 2 (the centred first difference times h^2).

A general stencil is held as a centre coefficient a0 and, per dimension d, the
coefficients am[d] of u_{p-e_d} and ap[d] of u_{p+e_d}. Each is either a scalar
(constant coefficients) or an array of n values (variable coefficients).
"""
from __future__ import annotations

import numpy as np


class Stencil:
    """A (2d+1)-point stencil on a grid of `shape` = (N_x, N_y[, N_z]), x fastest."""

    def __init__(self, shape, a0, am, ap):
        self.shape = tuple(int(v) for v in shape)
        self.dim = len(self.shape)
        assert self.dim in (2, 3) and len(am) == self.dim and len(ap) == self.dim
        self.n = int(np.prod(self.shape))
        self.a0 = a0
        self.am = list(am)
        self.ap = list(ap)

    # numpy array axis of grid dimension d (x is the last, fastest axis)
    def _axis(self, d):
        return self.dim - 1 - d

    def _grid(self, v):
        return np.asarray(v, dtype=np.float64).reshape(self.shape[::-1])

    def _coef(self, c):
        return c if np.isscalar(c) else self._grid(c)

    def apply(self, x):
        """y = A x, by the row definition, summing centre, then (minus, plus) per dimension."""
        X = self._grid(x)
        Y = self._coef(self.a0) * X
        for d in range(self.dim):
            ax = self._axis(d)
            lo = [slice(None)] * self.dim
            hi = [slice(None)] * self.dim
            # x_minus[p] = x[p - e_d] (zero at the low boundary)
            xm = np.zeros_like(X)
            lo[ax] = slice(1, None)
            hi[ax] = slice(None, -1)
            xm[tuple(lo)] = X[tuple(hi)]
            # x_plus[p] = x[p + e_d] (zero at the high boundary)
            xp = np.zeros_like(X)
            xp[tuple(hi)] = X[tuple(lo)]
            Y = Y + self._coef(self.am[d]) * xm
            Y = Y + self._coef(self.ap[d]) * xp
        return Y.reshape(-1)

    def norm_inf(self):
        """max_p sum_q |A_pq| (boundary rows drop their missing neighbours)."""
        tot = np.abs(np.broadcast_to(self._coef(self.a0), self.shape[::-1])).copy()
        for d in range(self.dim):
            ax = self._axis(d)
            m = np.abs(np.broadcast_to(self._coef(self.am[d]), self.shape[::-1])).copy()
            p = np.abs(np.broadcast_to(self._coef(self.ap[d]), self.shape[::-1])).copy()
            lo = [slice(None)] * self.dim
            lo[ax] = 0
            m[tuple(lo)] = 0.0  # no neighbour below the first plane
            hi = [slice(None)] * self.dim
            hi[ax] = -1
            p[tuple(hi)] = 0.0  # no neighbour above the last plane
            tot += m + p
        return float(tot.max())


def convdiff(shape, beta):
    """Constant-coefficient operator of -Lap u + beta . grad u on the unit square/cube.

    All sides must be equal (one h). c_d = beta_d h / 2, h = 1/(N+1).
    """
    shape = tuple(int(v) for v in shape)
    N = shape[0]
    assert all(v == N for v in shape), "convdiff needs a square/cubic grid"
    dim = len(shape)
    h = 1.0 / (N + 1)
    c = [beta[d] * h / 2.0 for d in range(dim)]
    return Stencil(shape, 2.0 * dim, [-1.0 - cd for cd in c], [-1.0 + cd for cd in c])


def convdiff_variable(N, beta_field):
    """2-D operator of -Lap u + beta(x, y) (u_x + u_y) with beta sampled at the nodes.

    Non-conservative form: c(p) = beta(x_p, y_p) h / 2 multiplies both first
    differences of row p.
    """
    h = 1.0 / (N + 1)
    c = np.asarray(beta_field, dtype=np.float64) * (h / 2.0)
    return Stencil((N, N), 4.0, [-1.0 - c, -1.0 - c], [-1.0 + c, -1.0 + c])


def jacobi(A, f, x, sweeps, omega):
    """Damped Jacobi relaxation: `sweeps` times x <- x + omega D^{-1} (f - A x), D = diag(A) = a0.

    A textbook smoother (Saad, Iterative Methods for Sparse Linear Systems, Sec. 4.1),
    not one of the paper's methods: it post-smooths the learned initial guess.
    """
    d = np.broadcast_to(A._coef(A.a0), A.shape[::-1]).reshape(-1)
    x = np.array(x, dtype=np.float64)
    f = np.asarray(f, dtype=np.float64)
    for _ in range(sweeps):
        x = x + omega * (f - A.apply(x)) / d
    return x
