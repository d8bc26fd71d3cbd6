"""Algorithm 3.1 (s-step Orthomin(k)) and Algorithms 4.1/4.2 (s-step GMRES), plain FP64.

Readings of passages the paper leaves garbled or open (each applies to both
solvers where relevant):
  * The monomial powers are scaled, y^{j+1} = sigma A y^j, with sigma given by
    the caller (1/||A||_inf by default in the library). Scaling leaves every
    Krylov space unchanged; sigma = 1 is the paper's literal form.
  * s-step GMRES(m): m is the Krylov dimension of one cycle, built as m/s
    blocks of s vectors (Sec. 6 chooses "m = m_bar s"), compared with GMRES(m).
  * Algorithm 4.1: block k's raw powers are Y = [y^1, ..., y^{s+1}] with
    y^1 = v_k^1. Steps 4-5 take the inner products of y^2..y^{s+1} with the
    earlier blocks; Scalar2 solves W_i t = c per earlier block, and step 7
    subtracts sum_i V_i t (the first column gets coefficient 0, as printed).
    Scalar1's W_k = V_k^T V_k is then computed from the projected block (the
    paper's "compute and decompose W_i"); deriving it from the raw-power Gram
    instead loses positive definiteness at s = 8. The next start vector is the
    projection of y^{s+1} (equal, up to span(V_1..V_k), to A v_k^s of step 2):
    u = z - V_k S with S = W_k^{-1} V_k^T z, normalised, v_{k+1}^1 = u/||u||.
  * eq. 4-5: the relation is read as A V_k = U_k G_k with U_k = [V_k, v_{k+1}^1];
    the subdiagonal entry of the last column of block k is ||u|| / sigma.
  * eq. 6-9: D = U^T U = diag(W_1, ..., W_k, 1) = L^T L with L upper
    triangular, and the least-squares functional is ||L (beta e_1 - G y)||
    (eq. 9 then follows because L e_1 = ||v_1^1|| e_1). It is minimised by
    Givens QR of the upper Hessenberg L G, one column at a time; the row of
    the newest start vector is scaled by 1 (its norm).
  * A non-positive Cholesky pivot in W_k ends the cycle with the blocks built
    so far; in the first block of a cycle it is a breakdown (status -4).
  * Algorithm 3.1: step 2 solves W_i a = m_i (the printed right-hand side b_i
    is read as m_i); c_j^l is read as C_j = (A P_j)^T A R_{i+1} with
    A R = [A r, A R_2, ..., A R_s] and R = [r, sigma A r, ..., sigma A R_{s-1}];
    step 5 computes R_{i+1}; the window is j_i = max(0, i-k+1).
  * Sec. 3's remedy for large s (not implemented in the paper): each new direction
    block is made A^T A-orthogonal by modified Gram-Schmidt once it is formed, so
    that W_i is diagonal and Scalar1/Scalar2 are diagonal solves. It is read as
    applying to P_{i+1} after the projection against the window (steps 8-9), and to
    P_0 = R_0, so that every W_j of the window is diagonal; the columns are also
    normalised (A p_j^l of unit length), the diagonal then being the identity up to
    rounding, and the diagonal solves divide by the computed diagonal of W.
"""
from __future__ import annotations

import numpy as np

from . import STATUS_BREAKDOWN, STATUS_NOT_CONVERGED, STATUS_OK
from .krylov import GivensLSQ, norm, residual_scale


# ---------------------------------------------------------------- small dense algebra
def cholesky_upper(W):
    """W = L^T L with L upper triangular; returns None on a non-positive pivot."""
    s = W.shape[0]
    L = np.zeros_like(W)
    for i in range(s):
        d = W[i, i] - np.dot(L[:i, i], L[:i, i])
        if not d > 0.0:
            return None
        L[i, i] = np.sqrt(d)
        for j in range(i + 1, s):
            L[i, j] = (W[i, j] - np.dot(L[:i, i], L[:i, j])) / L[i, i]
    return L


def cholesky_solve(L, B):
    """Solve (L^T L) X = B by forward (L^T) then backward (L) substitution."""
    B = np.array(B, dtype=np.float64, copy=True)
    vec = B.ndim == 1
    if vec:
        B = B[:, None]
    s = L.shape[0]
    Z = np.zeros_like(B)
    for i in range(s):
        Z[i] = (B[i] - L[:i, i] @ Z[:i]) / L[i, i]
    X = np.zeros_like(B)
    for i in range(s - 1, -1, -1):
        X[i] = (Z[i] - L[i, i + 1 :] @ X[i + 1 :]) / L[i, i]
    return X[:, 0] if vec else X


# ---------------------------------------------------------------- block primitives
def matrix_powers(A, v, s, sigma, scale=1.0, shifts=None):
    """Y = [y^1, ..., y^{s+1}], y^1 = scale v, y^{j+1} = sigma A y^j (s products).

    The directions R_i = [r, Ar, ..., A^{s-1} r] of Sec. 3 and the raw block of
    Algorithm 4.1 step 3 are both such power blocks. With `shifts` (theta_1..theta_s)
    the block is the Newton basis y^{j+1} = sigma (A - theta_j I) y^j, which spans the
    same Krylov space (Sec. 3 points to better-conditioned bases for large s).
    """
    Y = np.zeros((v.shape[0], s + 1))
    Y[:, 0] = scale * v
    for j in range(s):
        Y[:, j + 1] = sigma * A.apply(Y[:, j])
        if shifts is not None:
            Y[:, j + 1] -= sigma * shifts[j] * Y[:, j]
    return Y


def leja_order(values, count):
    """The first `count` points of the Leja ordering of real `values`: the largest in
    modulus first, then each next point maximises the product of its distances to the
    points already taken (sums of logarithms; ties go to the earlier value). Points within
    1e-10 max|value| of a taken one (the two real parts of a complex pair) are skipped;
    when the distinct values run out, the sequence repeats from its start."""
    vals = [float(v) for v in values]
    if not vals:
        return [0.0] * count
    tiny = 1e-10 * max(abs(v) for v in vals)
    first = max(range(len(vals)), key=lambda i: (abs(vals[i]), -i))
    order = [first]
    while len(order) < len(vals):
        best, best_score = None, None
        for i, v in enumerate(vals):
            if i in order:
                continue
            d = [abs(v - vals[j]) for j in order]
            if min(d) <= tiny:
                continue
            score = sum(np.log(x) for x in d)
            if best_score is None or score > best_score:
                best, best_score = i, score
        if best is None:
            break
        order.append(best)
    seq = [vals[i] for i in order]
    return [seq[j % len(seq)] for j in range(count)]


def newton_shifts(G, K, s):
    """Shifts for the Newton basis: the real parts of the Ritz values of A on the first
    cycle's Krylov space, i.e. the eigenvalues of the leading K x K block of G (the basis
    U is orthogonal between blocks and its next start vector is orthogonal to V, so this
    is the Galerkin projection), sorted ascending, then in Leja order."""
    ev = np.linalg.eigvals(G[:K, :K])
    return leja_order(np.sort(np.real(ev)), s)


def inner_products(V, Y):
    """C = V^T Y: the simultaneous inner products of one s-step (Sec. 1, Alg. 4.1 steps 4-5)."""
    return V.T @ Y


def block_update(Y, V, T):
    """Y_hat = Y - V T and its Gram matrix Y_hat^T Y_hat (Alg. 4.1 step 7 and Scalar1)."""
    Yh = Y - V @ T
    return Yh, Yh.T @ Yh


# ---------------------------------------------------------------- s-step GMRES
class _RightPreconditioned:
    """The operator A M^-1 (right preconditioning): apply(v) = A (M^-1 v)."""

    def __init__(self, A, M):
        self.A, self.M = A, M

    def apply(self, v):
        return self.A.apply(self.M.apply_inv(v))


def sstep_gmres(A, f, x0, s, m, tol, sigma, max_cycles=1000, trace=None, basis="monomial", shifts=None,
                shift_rule=None, precond=None):
    """Restarted s-step GMRES, Algorithm 4.2 over the s-step Arnoldi of Algorithm 4.1.

    Returns dict(x, status, cycles, iters, matvecs, history, relres, shifts); the
    history holds the explicit relres at each restart and the least-squares
    estimate after each of the s steps of every block. If `trace` is a dict,
    the first cycle's basis U, Hessenberg G and Gram blocks W are stored in it.
    basis = "newton": the first cycle uses the monomial powers; every later cycle the
    Newton basis with the Leja-ordered real parts of the first cycle's Ritz values.
    `shifts` (test use): Newton shifts to apply from the first cycle on. `shift_rule`
    (test use): replaces newton_shifts(G, K, s) after the first cycle.
    precond: an object with apply_inv(v) = M^-1 v (e.g. stencil.RedBlackILU0(A)): right
    preconditioning, the s-step Arnoldi of A M^-1 and x = x0 + M^-1 V y; the restart
    residual stays the true f - A x.
    """
    assert m % s == 0 and s >= 1
    n = f.shape[0]
    nb = m // s
    nf = residual_scale(f)
    x = np.array(x0, dtype=np.float64, copy=True)
    hist = []
    cycles = iters = mv = 0
    status = STATUS_NOT_CONVERGED
    shifts = None if shifts is None else list(shifts)
    op = A if precond is None else _RightPreconditioned(A, precond)
    while True:
        r = f - A.apply(x)                                   # step 1 / step 5 (restart)
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
        U = np.zeros((n, m + 1))
        U[:, 0] = r / beta
        G = np.zeros((m + 1, m))
        Ls, Ws = [], []
        lsq = None
        K = 0
        for k in range(nb):                                  # Algorithm 4.1, block k+1
            o = k * s
            Y = matrix_powers(op, U[:, o], s, sigma, shifts=shifts)   # step 3: s products
            mv += s
            T = np.zeros((o, s + 1))
            if o > 0:
                C = inner_products(U[:, :o], Y[:, 1:])      # step 4: earlier blocks vs new powers
                for i in range(k):                           # Scalar2: W_i t = c
                    T[i * s : (i + 1) * s, 1:] = cholesky_solve(Ls[i], C[i * s : (i + 1) * s])
            Yh, G2 = block_update(Y, U[:, :o], T)            # step 7, and V_k^T V_k for Scalar1
            Lk = cholesky_upper(G2[:s, :s])                  # Scalar1: decompose W_k
            if Lk is None:
                if k == 0:
                    status = STATUS_BREAKDOWN
                break
            S = cholesky_solve(Lk, G2[:s, s])
            u = Yh[:, s] - Yh[:, :s] @ S                     # projection of A v_k^s (step 2)
            nu = norm(u)
            U[:, o : o + s] = Yh[:, :s]
            if nu > 0.0:
                U[:, o + s] = u / nu
            Ls.append(Lk)
            Ws.append(G2[:s, :s])
            # eq. 4-5: column o+j of G holds A v_k^{j+1} in the coordinates of U
            for j in range(s):
                col = np.zeros(m + 1)
                col[:o] = T[:, j + 1]
                if j + 1 < s:
                    col[o + j + 1] = 1.0
                else:
                    col[o : o + s] = S
                    col[o + s] = nu
                col = col / sigma
                if shifts is not None:   # A y^{j+1} = y^{j+2} / sigma + theta_j y^{j+1}
                    col[:o] += shifts[j] * T[:, j]
                    col[o + j] += shifts[j]
                if o > 0:
                    col = col - G[:, :o] @ T[:, j]
                G[:, o + j] = col
            # eq. 9: Givens on L G, L = diag(L_1..L_k) and 1 on the newest start row
            if lsq is None:
                lsq = GivensLSQ(m, beta * Ls[0][0, 0])
            stop = False
            for j in range(s):
                c = o + j
                lg = np.zeros(m + 1)
                for i in range(k + 1):
                    rows = slice(i * s, (i + 1) * s)
                    lg[rows] = Ls[i] @ G[rows, c]
                lg[o + s] = G[o + s, c]
                est = lsq.add_column(lg)
                iters += 1
                hist.append(est / nf)
            K = o + s
            if est <= tol * nf or nu == 0.0:
                stop = True
            if stop:
                break
        if trace is not None and "U" not in trace:
            trace.update(U=U[:, : K + 1].copy(), G=G[: K + 1, :K].copy(), W=[w.copy() for w in Ws], s=s)
        if basis == "newton" and shifts is None and K > 0:
            shifts = (shift_rule or newton_shifts)(G, K, s)
        if K > 0:
            y = lsq.solve()[:K] if lsq.j == K else lsq.solve()
            dx = U[:, : lsq.j] @ y                           # step 3: x_m = x_0 + V y
            x = x + (dx if precond is None else precond.apply_inv(dx))
        if status == STATUS_BREAKDOWN:
            relres = norm(f - A.apply(x)) / nf
            break
    return dict(x=x, status=status, cycles=cycles, iters=iters, matvecs=mv, history=hist, relres=relres,
                shifts=shifts)


# ---------------------------------------------------------------- s-step Orthomin
def _omin_factor(AP, ortho):
    """What Scalar1/Scalar2 need of W = (A P)^T A P: its Cholesky factor, or (ortho)
    its diagonal (None on a non-positive pivot or diagonal entry)."""
    if ortho:
        d = np.einsum("ij,ij->j", AP, AP)
        return d if np.all(d > 0.0) else None
    return cholesky_upper(AP.T @ AP)


def _omin_solve(Lw, rhs, ortho):
    """W x = rhs with W given by _omin_factor (rhs a vector or an s-row matrix)."""
    if ortho:
        return rhs / (Lw if np.ndim(rhs) == 1 else Lw[:, None])
    return cholesky_solve(Lw, rhs)


def omin_powers(A, r, s, sigma):
    """R = [r, sigma A r, ..., sigma A R_{s-1}] and A R, with s products."""
    R = np.zeros((r.shape[0], s))
    AR = np.zeros((r.shape[0], s))
    R[:, 0] = r
    for j in range(s):
        AR[:, j] = A.apply(R[:, j])
        if j + 1 < s:
            R[:, j + 1] = sigma * AR[:, j]
    return R, AR


def ata_mgs(P, AP):
    """Modified Gram-Schmidt of the block P in the A^T A inner product (Sec. 3).

    Works on the columns of A P and applies every operation to P as well: for
    l = 1..s, A p^l is normalised, then its component is removed from the later
    columns. Returns (P Q, A P Q) with Q upper triangular and (A P Q)^T (A P Q) = I
    up to rounding, or None when a column has no component left (breakdown).
    """
    P = np.array(P, dtype=np.float64, copy=True)
    AP = np.array(AP, dtype=np.float64, copy=True)
    s = P.shape[1]
    for l in range(s):
        nrm = norm(AP[:, l])
        if not nrm > 0.0:
            return None
        AP[:, l] /= nrm
        P[:, l] /= nrm
        for j in range(l + 1, s):
            d = np.dot(AP[:, l], AP[:, j])
            AP[:, j] -= d * AP[:, l]
            P[:, j] -= d * P[:, l]
    return P, AP


def sstep_omin(A, f, x0, s, k, tol, sigma, max_iters=100000, trace=None, precond=None, basis="monomial"):
    """s-step Orthomin(k), Algorithm 3.1.

    Per step i: m_i = (A P_i)^T r_i and W_i = (A P_i)^T A P_i; a = W_i^{-1} m_i
    (Scalar1); x += P_i a; r -= A P_i a; R_{i+1}, A R_{i+1} from r;
    C_j = (A P_j)^T A R_{i+1} and B_j = -W_j^{-1} C_j (Scalar2) for the window
    j = max(0, i-k+1)..i; P_{i+1} = R_{i+1} + sum_j P_j B_j and
    A P_{i+1} = A R_{i+1} + sum_j A P_j B_j. s = 1 is Orthomin(k) (Alg. 2.1).
    If `trace` is a dict it receives the A P blocks of the last window.
    precond (apply_inv(v) = M^-1 v): right preconditioning, the method on A M^-1 (the
    residual is the true f - A x); the steps P a accumulate in du and x += M^-1 du before
    every explicit residual.
    basis="ortho": every direction block is A^T A-orthonormalised by ata_mgs once
    formed (P_0 and each P_{i+1}); W_j is then diagonal and Scalar1 (a = m / diag W)
    and Scalar2 (B_j = -C_j / diag W_j, row-wise) are diagonal solves (Sec. 3).
    """
    if basis not in ("monomial", "ortho"):
        raise ValueError(basis)
    ortho = basis == "ortho"
    nf = residual_scale(f)
    x = np.array(x0, dtype=np.float64, copy=True)
    mv = 0
    hist = []
    status = STATUS_NOT_CONVERGED
    it = 0
    P = None
    op = A if precond is None else _RightPreconditioned(A, precond)
    du = np.zeros_like(x)

    def fold(x, du):
        if precond is None:
            return x, du
        return x + precond.apply_inv(du), np.zeros_like(du)

    while True:
        if P is None:
            x, du = fold(x, du)
            r = f - A.apply(x)
            mv += 1
            relres = norm(r) / nf
            hist.append(relres)
            if relres <= tol:
                status = STATUS_OK
                break
            if it >= max_iters:
                break
            R, AR = omin_powers(op, r, s, sigma)            # R_0, P_0 = R_0
            mv += s
            if ortho:
                Q = ata_mgs(R, AR)
                if Q is None:
                    status = STATUS_BREAKDOWN
                    break
                R, AR = Q
            L0 = _omin_factor(AR, ortho)
            if L0 is None:
                status = STATUS_BREAKDOWN
                break
            P, AP, Ls = [R], [AR], [L0]
        mvec = AP[-1].T @ r                                  # step 1
        a = _omin_solve(Ls[-1], mvec, ortho)                 # step 2 (Scalar1)
        if precond is None:
            x = x + P[-1] @ a                                # step 3
        else:
            du = du + P[-1] @ a
        r = r - AP[-1] @ a                                   # step 4
        it += 1
        rr = norm(r) / nf
        hist.append(rr)
        if rr <= tol or it >= max_iters:
            P = None
            if it >= max_iters:
                x, du = fold(x, du)
                relres = norm(f - A.apply(x)) / nf
                mv += 1
                hist.append(relres)
                if relres <= tol:
                    status = STATUS_OK
                break
            continue
        R, AR = omin_powers(op, r, s, sigma)                 # step 5
        mv += s
        Pn = R.copy()
        APn = AR.copy()
        lo = len(P) - min(k, len(P))
        for j in range(lo, len(P)):
            C = AP[j].T @ AR                                 # step 6
            B = -_omin_solve(Ls[j], C, ortho)                # step 7 (Scalar2)
            Pn = Pn + P[j] @ B                               # step 8
            APn = APn + AP[j] @ B                            # step 9
        Q = ata_mgs(Pn, APn) if ortho else (Pn, APn)
        Ln = None if Q is None else _omin_factor(Q[1], ortho)
        if Ln is None:
            status = STATUS_BREAKDOWN
            x, du = fold(x, du)
            relres = norm(f - A.apply(x)) / nf
            break
        Pn, APn = Q
        P.append(Pn)
        AP.append(APn)
        Ls.append(Ln)
        keep = max(k, 1)
        P, AP, Ls = P[-keep:], AP[-keep:], Ls[-keep:]
        if trace is not None:
            trace["AP"] = [b.copy() for b in AP]
    return dict(x=x, status=status, iters=it, matvecs=mv, history=hist, relres=relres)
