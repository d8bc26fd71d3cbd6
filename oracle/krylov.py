"""Algorithm 2.1 (Orthomin(k)) and Algorithm 2.2 (GMRES(m)), plain FP64.

Conventions shared by every solver in this package (they are readings of the
paper, which states the stopping test only as a garbled "||r_i||^{1/2} < 1e-6"
in Sec. 6):
  * relres = ||f - A x||_2 / ||f||_2; a solve succeeds when relres <= tol.
  * GMRES-type methods (restarted) recompute r = f - A x explicitly at every
    restart (Algorithm 4.2 step 5) and append its relres to the history; after
    each Krylov step they append the least-squares residual estimate
    |g_{j+1}| / ||f|| of eq. 2 (standard Givens QR), and a cycle stops early
    once that estimate is <= tol. The explicit residual of the next restart
    decides convergence.
  * Orthomin-type methods append ||r_i|| / ||f|| of the updated residual after
    each step; when it drops to tol the residual is recomputed explicitly, and
    if that is still above tol the method restarts from the explicit residual.
"""
from __future__ import annotations

import numpy as np

from . import STATUS_BREAKDOWN, STATUS_NOT_CONVERGED, STATUS_OK


def norm(v):
    return float(np.sqrt(np.dot(v, v)))


def residual_scale(f):
    """||f||, the denominator of the relative residual test ||f - A x|| / ||f|| <= tol;
    1 when f = 0 (A is nonsingular, so x = 0 is the solution and the test is made on
    ||f - A x|| itself: from x0 = 0 the solve ends at once)."""
    nf = norm(f)
    return nf if nf > 0.0 else 1.0


class GivensLSQ:
    """min_y || g0 e_1 - H y || for an upper Hessenberg H given column by column (eq. 2).

    Each new column (length j+2 for column j) is hit by the previous rotations,
    then a rotation zeroing its subdiagonal entry is formed as
    c = a/d, s = b/d, d = sqrt(a^2 + b^2), and applied to the right-hand side.
    |g[j+1]| is the residual norm of the least-squares problem after j+1 columns.
    """

    def __init__(self, mmax, g0):
        self.R = np.zeros((mmax + 1, mmax))
        self.g = np.zeros(mmax + 1)
        self.g[0] = g0
        self.c = np.zeros(mmax)
        self.s = np.zeros(mmax)
        self.j = 0

    def add_column(self, col):
        j = self.j
        h = np.array(col[: j + 2], dtype=np.float64)
        for i in range(j):
            t = self.c[i] * h[i] + self.s[i] * h[i + 1]
            h[i + 1] = -self.s[i] * h[i] + self.c[i] * h[i + 1]
            h[i] = t
        a, b = h[j], h[j + 1]
        d = np.sqrt(a * a + b * b)
        self.c[j] = a / d
        self.s[j] = b / d
        h[j] = d
        h[j + 1] = 0.0
        self.R[: j + 2, j] = h
        self.g[j + 1] = -self.s[j] * self.g[j]
        self.g[j] = self.c[j] * self.g[j]
        self.j = j + 1
        return abs(self.g[j + 1])

    def solve(self):
        """y solving the leading j x j triangle R y = g (back substitution)."""
        j = self.j
        y = np.zeros(j)
        for i in range(j - 1, -1, -1):
            y[i] = (self.g[i] - np.dot(self.R[i, i + 1 : j], y[i + 1 : j])) / self.R[i, i]
        return y


def gmres(A, f, x0, m, tol, max_cycles=1000, orth="cgs"):
    """Restarted GMRES(m), Algorithm 2.2 and eq. 2-3.

    Per cycle: r0 = f - A x0, q_1 = r0/||r0||; for j = 1..m (m Arnoldi steps,
    m+1 basis vectors; the listing's upper limit m-1 is read as m):
      h_ij = q_i^T A q_j for i <= j (classical Gram-Schmidt, all i at once),
      q^_{j+1} = A q_j - sum_i h_ij q_i, h_{j+1,j} = ||q^_{j+1}||,
      q_{j+1} = q^_{j+1} / h_{j+1,j};
    then x_m = x0 + Q_m y_m with y_m minimising ||beta e_1 - G_m y|| (eq. 2).
    orth="mgs" is the modified Gram-Schmidt cross-check (one inner product at
    a time, each against the partially orthogonalised vector).

    Returns dict(x, status, cycles, iters, matvecs, history, relres).
    """
    n = f.shape[0]
    nf = residual_scale(f)
    x = np.array(x0, dtype=np.float64, copy=True)
    hist = []
    cycles = iters = mv = 0
    status = STATUS_NOT_CONVERGED
    while True:
        r = f - A.apply(x)
        mv += 1
        beta = norm(r)
        relres = beta / nf
        hist.append(relres)
        if relres <= tol:
            status = STATUS_OK
            break
        if cycles >= max_cycles:
            break
        cycles += 1
        Q = np.zeros((n, m + 1))
        Q[:, 0] = r / beta
        lsq = GivensLSQ(m, beta)
        for j in range(m):
            w = A.apply(Q[:, j])
            mv += 1
            if orth == "cgs":
                h = Q[:, : j + 1].T @ w
                w = w - Q[:, : j + 1] @ h
            else:
                h = np.zeros(j + 1)
                for i in range(j + 1):
                    h[i] = np.dot(Q[:, i], w)
                    w = w - h[i] * Q[:, i]
            hn = norm(w)
            est = lsq.add_column(np.concatenate([h, [hn]]))
            iters += 1
            hist.append(est / nf)
            if est <= tol * nf or hn == 0.0:
                break
            Q[:, j + 1] = w / hn
        y = lsq.solve()
        x = x + Q[:, : lsq.j] @ y
    return dict(x=x, status=status, cycles=cycles, iters=iters, matvecs=mv, history=hist, relres=relres)


def omin(A, f, x0, k, tol, max_iters=100000):
    """Orthomin(k), Algorithm 2.1.

    a_i = r_i^T A p_i / (A p_i)^T A p_i; x += a_i p_i; r -= a_i A p_i;
    b_j = (A r_{i+1})^T A p_j / (A p_j)^T A p_j for j_i <= j <= i;
    p_{i+1} = r_{i+1} - sum_j b_j p_j; A p_{i+1} = A r_{i+1} - sum_j b_j A p_j.
    The window index is read as j_i = max(0, i-k+1) (the k most recent
    directions; the printed min(0, i-k+1) would always give GCR). k = 0 keeps
    no previous direction (the minimal-residual steepest descent of Sec. 3).
    """
    nf = residual_scale(f)
    x = np.array(x0, dtype=np.float64, copy=True)
    mv = 0
    hist = []
    status = STATUS_NOT_CONVERGED
    it = 0
    P = AP = APn2 = None
    while True:
        if P is None:
            # (re)start: r = f - A x, p_0 = r, A p_0 = A r
            r = f - A.apply(x)
            mv += 1
            relres = norm(r) / nf
            hist.append(relres)
            if relres <= tol:
                status = STATUS_OK
                break
            if it >= max_iters:
                break
            P, AP = [r.copy()], [A.apply(r)]
            mv += 1
            APn2 = [np.dot(AP[0], AP[0])]
        a = np.dot(r, AP[-1]) / APn2[-1]                  # step 1
        x = x + a * P[-1]                                  # step 2
        r = r - a * AP[-1]                                 # step 3
        it += 1
        rr = norm(r) / nf
        hist.append(rr)
        if rr <= tol or it >= max_iters:
            P = None                                       # confirm with the explicit residual
            if it >= max_iters:
                relres = norm(f - A.apply(x)) / nf
                mv += 1
                hist.append(relres)
                if relres <= tol:
                    status = STATUS_OK
                break
            continue
        Ar = A.apply(r)
        mv += 1
        p = r.copy()
        ap = Ar.copy()
        lo = len(P) - min(k, len(P))                      # window j_i .. i
        for j in range(lo, len(P)):
            b = np.dot(Ar, AP[j]) / APn2[j]                # step 4
            p = p - b * P[j]                               # step 5
            ap = ap - b * AP[j]                            # step 6
        P.append(p)
        AP.append(ap)
        APn2.append(np.dot(ap, ap))
        keep = max(k, 1)
        P, AP, APn2 = P[-keep:], AP[-keep:], APn2[-keep:]
    return dict(x=x, status=status, iters=it, matvecs=mv, history=hist, relres=relres)
