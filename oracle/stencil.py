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


class NaturalILU0:
    """ILU(0) of a stencil operator in the natural (lexicographic, x fastest) ordering: the
    preconditioner of the paper's tables (Sec. 5: right preconditioning with ILU(0)).

    ILU(0) keeps the sparsity of A, so L U equals A on that sparsity. For a (2d+1)-point
    stencil this fixes the factors row by row in the natural order:
      * U has A's upper part off the diagonal (U[p, p + e_d] = A[p, p + e_d]) and the
        pivots d[p] on it;
      * L is unit lower triangular with L[p, p - e_d] = A[p, p - e_d] / d[p - e_d];
      * d[p] = A[p, p] - sum_d A[p, p - e_d] A[p - e_d, p] / d[p - e_d], the diagonal of
        (L U)[p, p] matched to A[p, p]. The other products L[p, p - e_d] U[p - e_d, q] land
        at q = p - e_d + e_d' (d != d'), outside the sparsity: that is the dropped fill.
    M^-1 v = U^-1 (L^-1 v): a forward substitution y[p] = v[p] - sum_d L[p, p - e_d] y[p - e_d]
    in the natural order, then a backward one z[p] = (y[p] - sum_d A[p, p + e_d] z[p + e_d]) / d[p]
    in the reverse order. The sums run over the dimensions x, y, z in turn; every loop here
    is the definition, one point at a time (the library sweeps the same arithmetic along
    hyperplanes, where the points are independent).
    """

    def __init__(self, A):
        self.A = A
        n, dim = A.n, A.dim
        sh = A.shape[::-1]
        self.a0 = np.broadcast_to(A._coef(A.a0), sh).reshape(-1).astype(np.float64)
        self.am = [np.broadcast_to(A._coef(A.am[d]), sh).reshape(-1).astype(np.float64) for d in range(dim)]
        self.ap = [np.broadcast_to(A._coef(A.ap[d]), sh).reshape(-1).astype(np.float64) for d in range(dim)]
        self.stride = [1, A.shape[0], A.shape[0] * A.shape[1]][:dim]
        self.coord = np.indices(sh).reshape(dim, -1)[::-1]     # coord[d][p]: index of p along dimension d
        d = np.zeros(n)
        L = [np.zeros(n) for _ in range(dim)]
        a0, am, ap = self.a0.tolist(), [v.tolist() for v in self.am], [v.tolist() for v in self.ap]
        coord = [c.tolist() for c in self.coord]
        for p in range(n):
            dp = a0[p]
            for k in range(dim):
                if coord[k][p] > 0:
                    q = p - self.stride[k]
                    dp -= am[k][p] * ap[k][q] / d[q]
            d[p] = dp
            for k in range(dim):
                if coord[k][p] > 0:
                    L[k][p] = am[k][p] / d[p - self.stride[k]]
        self.d, self.L = d, L

    def apply_inv(self, v):
        """z = M^-1 v = U^-1 L^-1 v."""
        A = self.A
        n, dim = A.n, A.dim
        v = np.asarray(v, dtype=np.float64).tolist()
        L = [x.tolist() for x in self.L]
        ap = [x.tolist() for x in self.ap]
        d = self.d.tolist()
        coord = [c.tolist() for c in self.coord]
        y = [0.0] * n
        for p in range(n):
            t = v[p]
            for k in range(dim):
                if coord[k][p] > 0:
                    t -= L[k][p] * y[p - self.stride[k]]
            y[p] = t
        z = [0.0] * n
        for p in range(n - 1, -1, -1):
            t = y[p]
            for k in range(dim):
                if coord[k][p] < A.shape[k] - 1:
                    t -= ap[k][p] * z[p + self.stride[k]]
            z[p] = t / d[p]
        return np.array(z)


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


class RedBlackILU0:
    """ILU(0) of a stencil operator in red-black ordering (red: x + y + z even).

    Every neighbour of a point has the other colour, so with the red points first
    A = [[D_r, E], [F, D_b]] with diagonal D_r, D_b. ILU(0) keeps the sparsity of A:
    L = [[I, 0], [F D_r^-1, I]], U = [[D_r, E], [0, D~_b]], and the black diagonal
    D~_b = D_b - diag(F D_r^-1 E) is the only entry that changes (the off-diagonal part of
    F D_r^-1 E, between black points two steps apart, is the dropped fill). Applying
    M^-1 = (L U)^-1: w_b = (v_b - sum_r A[b, r] v_r / a0_r) / d~_b for black points, then
    w_r = (v_r - sum_b A[r, b] w_b) / a0_r for red points. (The paper's tables use ILU(0)
    in the natural ordering; this ordering has the same sparsity and two parallel
    half-sweeps instead of 3N - 2 sequential hyperplanes per triangular solve.)
    """

    def __init__(self, A):
        self.A = A
        sh = A.shape[::-1]                         # numpy axes (z, y, x) / (y, x)
        grids = np.indices(sh)
        self.black = (grids.sum(axis=0) % 2 == 1).reshape(-1)
        a0 = np.broadcast_to(A._coef(A.a0), sh).reshape(-1).astype(np.float64)
        self.a0 = a0.copy()
        # d~_b = a0_b - sum over neighbours r of A[b, r] A[r, b] / a0_r
        dt = a0.copy()
        for (ax, coef_b, coef_r, step) in self._couplings():
            dt -= coef_b * self._shift(coef_r / a0.reshape(sh), ax, step).reshape(-1)
        self.dtilde = np.where(self.black, dt, a0)

    def _couplings(self):
        # (axis, A[b, b + step e_d] as an array over b, A[r, r - step e_d] over r, step)
        A = self.A
        sh = A.shape[::-1]
        out = []
        for d in range(A.dim):
            ax = A._axis(d)
            am = np.broadcast_to(A._coef(A.am[d]), sh)
            ap = np.broadcast_to(A._coef(A.ap[d]), sh)
            # neighbour r = b - e_d: A[b, r] = am_d(b); A[r, b] = ap_d(r)
            out.append((ax, self._mask(am, ax, -1).reshape(-1), ap, -1))
            # neighbour r = b + e_d: A[b, r] = ap_d(b); A[r, b] = am_d(r)
            out.append((ax, self._mask(ap, ax, +1).reshape(-1), am, +1))
        return out

    @staticmethod
    def _shift(X, ax, step):
        """Y[p] = X[p + step e_ax] (zero outside the grid)."""
        Y = np.zeros_like(X, dtype=np.float64)
        src = [slice(None)] * X.ndim
        dst = [slice(None)] * X.ndim
        if step > 0:
            src[ax], dst[ax] = slice(1, None), slice(None, -1)
        else:
            src[ax], dst[ax] = slice(None, -1), slice(1, None)
        Y[tuple(dst)] = X[tuple(src)]
        return Y

    @staticmethod
    def _mask(C, ax, step):
        """C where the neighbour p + step e_ax exists, else 0."""
        M = np.array(C, dtype=np.float64, copy=True)
        idx = [slice(None)] * M.ndim
        idx[ax] = -1 if step > 0 else 0
        M[tuple(idx)] = 0.0
        return M

    def apply_inv(self, v):
        """w = M^-1 v."""
        A = self.A
        sh = A.shape[::-1]
        v = np.asarray(v, dtype=np.float64)
        red_v = np.where(self.black, 0.0, v)
        # black: w_b = (v_b - sum_r A[b, r] v_r / a0_r) / d~_b
        t = np.zeros(A.n)
        for (ax, coef_b, coef_r, step) in self._couplings():
            t += coef_b * self._shift((red_v / self.a0).reshape(sh), ax, step).reshape(-1)
        w = np.where(self.black, (v - t) / self.dtilde, 0.0)
        # red: w_r = (v_r - sum_b A[r, b] w_b) / a0_r, with A[r, b] the row-r coefficient of b
        s = np.zeros(A.n)
        for d in range(A.dim):
            ax = A._axis(d)
            am = self._mask(np.broadcast_to(A._coef(A.am[d]), sh), ax, -1)
            ap = self._mask(np.broadcast_to(A._coef(A.ap[d]), sh), ax, +1)
            W = w.reshape(sh)
            s += (am * self._shift(W, ax, -1) + ap * self._shift(W, ax, +1)).reshape(-1)
        return np.where(self.black, w, (v - s) / self.a0)
