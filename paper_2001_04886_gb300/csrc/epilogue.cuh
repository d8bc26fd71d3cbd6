// Scalar work of the s-step methods on the device: small FP64 algebra (Cholesky,
// triangular solves, Givens) and the epilogues that run in the last CTA of a
// reduction (Scalar1 / Scalar2 of Alg. 3.1 and 4.1, the Hessenberg columns of
// eq. 4-5, the least squares of eq. 6-9, restart decisions). Included by every
// translation unit that launches reductions; each gets its own copy.
#pragma once

#include <math.h>

#include "kernels.cuh"

namespace sstep {
namespace {   // internal linkage: each translation unit keeps its own copy

// ================================================================== small FP64 algebra
// Plain roundings (no contraction) so the scalar work follows the written formulas.
__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }

// W = L^T L, L upper triangular (col-major, ld s). false on a non-positive pivot.
__device__ bool chol_upper(const double* W, int ldw, int s, double* L) {
    for (int i = 0; i < s; ++i)
        for (int j = 0; j < s; ++j) L[i + j * s] = 0.0;
    for (int i = 0; i < s; ++i) {
        double t = 0.0;
        for (int q = 0; q < i; ++q) t = add(t, mul(L[q + i * s], L[q + i * s]));
        double d = sub(W[i + i * ldw], t);
        if (!(d > 0.0)) return false;
        double lii = sqrt(d);
        L[i + i * s] = lii;
        for (int j = i + 1; j < s; ++j) {
            double u = 0.0;
            for (int q = 0; q < i; ++q) u = add(u, mul(L[q + i * s], L[q + j * s]));
            L[i + j * s] = sub(W[i + j * ldw], u) / lii;
        }
    }
    return true;
}

// x = (L^T L)^{-1} b (forward with L^T, then backward with L); b and x may alias; s <= kMaxS.
__device__ void chol_solve(const double* L, int s, const double* b, double* x) {
    double z[kMaxS];
    for (int i = 0; i < s; ++i) {
        double t = 0.0;
        for (int q = 0; q < i; ++q) t = add(t, mul(L[q + i * s], z[q]));
        z[i] = sub(b[i], t) / L[i + i * s];
    }
    for (int i = s - 1; i >= 0; --i) {
        double t = 0.0;
        for (int q = i + 1; q < s; ++q) t = add(t, mul(L[i + q * s], x[q]));
        x[i] = sub(z[i], t) / L[i + i * s];
    }
}

// The same solves spread over lanes, with the divisions taken off the dependent chain.
// An FP64 division or square root is a long dependent sequence of FP64 operations, which
// GB300 issues slowly (about 1.5k cycles each, measured in these epilogues); one thread
// doing an s x s factorization and its two substitutions one operation after another
// waits for each in turn, in the last CTA of a reduction, while the rest of the GPU is
// idle. So the factorization divides a whole row of L at once (one lane per entry, the
// same quotients as chol_upper: a singular block still gives a zero or negative pivot
// exactly where the sequential factorization does), and the substitutions multiply by
// reciprocals of the diagonal formed off their dependent chain (each product differs
// from the quotient by at most an ulp; the solves stay backward stable).
//
// Forward substitution z = L^{-T} b for an aligned group of G lanes (G a power of two,
// s <= G; lane r of the group brings b_r and gets z_r; rd[q] = 1 / L_qq): column by
// column, z_q by lane q and then every lane r > q adds L[q, r] z_q to its sum, so each sum
// runs over q in ascending order, as in chol_solve. Every lane of the warp calls it.
__device__ double tri_fwd_group(const double* L, const double* rd, int s, double b_r, int r, int G) {
    double t = 0.0, z = 0.0;
    for (int q = 0; q < s; ++q) {
        if (r == q) z = mul(sub(b_r, t), rd[q]);
        const double zq = __shfl_sync(0xffffffffu, z, q, G);
        if (r > q && r < s) t = add(t, mul(L[q + r * s], zq));
    }
    return z;
}

// Backward substitution x = L^{-1} z for the same lanes: x_q from q = s - 1 down; lane r < q
// adds L[r, q] x_q to its sum (so in descending q; chol_solve sums in ascending q).
__device__ double tri_bwd_group(const double* L, const double* rd, int s, double z_r, int r, int G) {
    double t = 0.0, x = 0.0;
    for (int q = s - 1; q >= 0; --q) {
        if (r == q) x = mul(sub(z_r, t), rd[q]);
        const double xq = __shfl_sync(0xffffffffu, x, q, G);
        if (r < q) t = add(t, mul(L[r + q * s], xq));
    }
    return x;
}

// One warp (every lane calls it): W = L^T L (L upper, col-major ld s, into shared Ls) with
// z = L^{-T} b formed in the same sweep as column s of the factor of [W b] (row i of L,
// columns i + 1 .. s, one lane each, after its pivot: chol_upper's and chol_solve's
// forward pass, operation for operation), then x = L^{-1} z; lane r < s gets x_r. false
// (warp-uniform: every lane computes the pivots) on a non-positive pivot, with Ls as
// chol_upper leaves it. zs, rs: s doubles of shared scratch each (z, 1 / L_ii).
__device__ bool chol_solve_warp(const double* W, int ldw, const double* b, int s, double* Ls, double* zs, double* rs,
                                double& x) {
    const int lane = threadIdx.x & 31;
    for (int t = lane; t < s * s; t += 32) Ls[t] = 0.0;
    __syncwarp();
    bool ok = true;
    for (int i = 0; i < s; ++i) {
        double t = 0.0;
        for (int q = 0; q < i; ++q) t = add(t, mul(Ls[q + i * s], Ls[q + i * s]));
        const double d = sub(W[i + i * ldw], t);
        if (!(d > 0.0)) {
            ok = false;
            break;
        }
        const double lii = sqrt(d);
        // one division by every lane at once: lanes 0 .. s-1-i the entries of row i (the last
        // of them z_i), lane 31 the reciprocal 1 / L_ii
        const int j = i + 1 + lane;
        double num = 1.0;
        if (j <= s) {
            const double* cj = j < s ? Ls + j * s : zs;   // column j of L, or z
            double u = 0.0;
            for (int q = 0; q < i; ++q) u = add(u, mul(Ls[q + i * s], cj[q]));
            num = sub(j < s ? W[i + j * ldw] : b[i], u);
        }
        const double qv = num / lii;
        if (j < s) Ls[i + j * s] = qv;
        else if (j == s) zs[i] = qv;
        if (lane == 31) rs[i] = qv;
        if (lane == 0) Ls[i + i * s] = lii;
        __syncwarp();
    }
    x = 0.0;
    if (!ok) return false;
    x = tri_bwd_group(Ls, rs, s, lane < s ? zs[lane] : 0.0, lane, 32);
    return true;
}

__device__ void hist_push(SolverState* st, double v) {
    if (st->hist_len < st->hist_cap) st->hist[st->hist_len] = v;
    st->hist_len += 1;
}

// Adds column j (h[0..j+1]) of an upper Hessenberg matrix to the running Givens QR
// (eq. 2): previous rotations, a new rotation c = a/d, s = b/d, d = sqrt(a^2+b^2),
// and the update of g. Returns |g[j+1]|, the least-squares residual norm.
__device__ double givens_add(SolverState* st, int j, double* h) {
    const int ld = st->m + 1;
    for (int i = 0; i < j; ++i) {
        double c = st->gc[i], s = st->gs[i];
        double t = add(mul(c, h[i]), mul(s, h[i + 1]));
        h[i + 1] = add(mul(-s, h[i]), mul(c, h[i + 1]));
        h[i] = t;
    }
    double a = h[j], b = h[j + 1];
    double d = sqrt(add(mul(a, a), mul(b, b)));
    double c = a / d, s = b / d;
    st->gc[j] = c;
    st->gs[j] = s;
    h[j] = d;
    h[j + 1] = 0.0;
    for (int i = 0; i <= j + 1; ++i) st->R[i + j * ld] = h[i];
    double gj = st->g[j];
    st->g[j + 1] = mul(-s, gj);
    st->g[j] = mul(c, gj);
    return fabs(st->g[j + 1]);
}

// ================================================================== epilogues
// GMRES-type restart: the explicit residual decides (Alg. 4.2 step 5).
__device__ void epi_restart(SolverState* st, double rr) {
    st->matvecs += 1;
    double beta = sqrt(rr);
    double rel = beta / st->nf;
    st->relres = rel;
    st->beta = beta;
    hist_push(st, rel);
    if (!isfinite(rel)) {
        st->status = SSTEP_ERR_NAN;
        st->active = 0;
        st->building = 0;
    } else if (rel <= st->tol) {
        st->status = SSTEP_OK;
        st->active = 0;
        st->building = 0;
    } else if (st->cycles >= st->max_cycles) {
        st->status = SSTEP_NOT_CONVERGED;
        st->active = 0;
        st->building = 0;
    } else {
        st->cycles += 1;
        st->building = 1;
        st->K = 0;
        st->vscale = 1.0 / beta;
    }
}

// Scalar2 of Alg. 4.1: T[b*s..b*s+s-1, j+1] = W_b^{-1} C[b*s.., j] for earlier blocks b.
__device__ void epi_gm_T(const Epi& e, const double* C) {
    SolverState* st = e.st;
    const int s = st->s, m = st->m, o = e.o, nblk = o / s;
    __shared__ double sL[kMaxCols * kMaxS], sR[kMaxCols];   // the factors, the reciprocals of their diagonals
    for (int t = threadIdx.x; t < nblk * s * s; t += blockDim.x) sL[t] = st->L[t];
    for (int t = threadIdx.x; t < nblk * s; t += blockDim.x) {
        const int b = t / s, i = t % s;
        sR[t] = 1.0 / st->L[b * s * s + i + i * s];
    }
    __syncthreads();
    // one solve per group of 8 lanes (s <= 8): lane r holds row r; whole warps take part
    const int nsol = nblk * s, nwarp = (int)(blockDim.x >> 5);
    for (int w0 = (int)(threadIdx.x >> 5) * 4; w0 < nsol; w0 += nwarp * 4) {
        const int sol = w0 + (int)((threadIdx.x & 31) >> 3), r = threadIdx.x & 7;
        const bool act = sol < nsol && r < s;
        const int b = sol < nsol ? sol / s : 0, j = sol < nsol ? sol % s : 0;
        const double* Lb = sL + b * s * s;
        const double z = tri_fwd_group(Lb, sR + b * s, s, act ? C[(b * s + r) + j * o] : 0.0, r, 8);
        const double x = tri_bwd_group(Lb, sR + b * s, s, z, r, 8);
        if (act) st->T[(b * s + r) + (j + 1) * m] = x;
    }
    for (int i = threadIdx.x; i < o; i += blockDim.x) st->T[i] = 0.0;   // first column: 0 (step 7)
}

// Scalar1 of Alg. 4.1 on the projected block: W_k = V_k^T V_k, S = W_k^{-1} V_k^T z.
// The factor and the solution are formed in shared memory and then stored: formed in
// place in global memory, every read of an entry just written would wait for L2.
__device__ void epi_gm_W(const Epi& e, const double* G2) {
    SolverState* st = e.st;
    __shared__ double sLk[kMaxS * kMaxS], sz[kMaxS], sr[kMaxS];
    if (threadIdx.x >= 32) return;   // one warp
    const int s = st->s, o = e.o, ld = s + 1, lane = threadIdx.x;
    double* Lk = st->L + (o / s) * s * s;
    double x;
    const bool ok = chol_solve_warp(G2, ld, G2 + s * ld, s, sLk, sz, sr, x);
    for (int t = lane; t < s * s; t += 32) Lk[t] = sLk[t];
    if (lane == 0) {
        st->matvecs += s;
        if (!ok) {
            st->building = 0;
            if (o == 0) {
                st->status = SSTEP_ERR_BREAKDOWN;
                st->active = 0;
            }
        }
    }
    if (ok && lane < s) st->S[lane] = x;
}

// u = z - V_k S has been formed; nu = ||u||. Columns o..o+s-1 of G hold A v_k^j in
// the coordinates of U = [V_1..V_k, v_{k+1}^1] (eq. 4-5), then enter the Givens QR
// of L G (eq. 9). The products L G and the sweep of the earlier rotations over the
// s new columns run in parallel from shared memory; only the s new rotations among
// the new columns are sequential.
__device__ void epi_gm_nu(const Epi& e, const double* red) {
    SolverState* st = e.st;
    const int s = st->s, m = st->m, o = e.o, ldg = m + 1, kb = o / s;
    __shared__ double nu_s;
    __shared__ double sLG[(kMaxM + 1) * kMaxS];   // column jj of L G at sLG[jj*(m+1) + r]
    __shared__ double sc_[kMaxM], ss_[kMaxM];
    if (threadIdx.x == 0) {
        double nu = sqrt(red[0]);
        nu_s = nu;
        st->nu = nu;
        st->vscale = nu > 0.0 ? 1.0 / nu : 0.0;
    }
    for (int i = threadIdx.x; i < o; i += blockDim.x) {
        sc_[i] = st->gc[i];
        ss_[i] = st->gs[i];
    }
    __syncthreads();
    const double nu = nu_s, sigma = st->sigma;
    // columns of G (eq. 4-5)
    for (int t = threadIdx.x; t < ldg * s; t += blockDim.x) {
        const int r = t % ldg, j = t / ldg;
        double raw;
        if (r < o) raw = st->T[r + (j + 1) * m];
        else if (j + 1 < s) raw = (r == o + j + 1) ? 1.0 : 0.0;
        else if (r < o + s) raw = st->S[r - o];
        else raw = (r == o + s) ? nu : 0.0;
        double val = raw / sigma;
        {   // Newton basis: A y^{j+1} = y^{j+2} / sigma + theta_j y^{j+1} (theta_j = 0: monomial);
            // y^1 is the start vector itself, y^{j+1} has coordinates T[:, j] and e_{o+j}
            double rj = (r == o + j) ? 1.0 : 0.0;
            if (j > 0 && r < o) rj = st->T[r + j * m];
            val = fma(st->theta[j], rj, val);
        }
        if (o > 0) {   // the same multiply-adds in order; the loads of 8 terms issued together
            double acc = 0.0;
            for (int i0 = 0; i0 < o; i0 += 8) {
                double gv[8], tv[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const bool in = i0 + u < o;
                    gv[u] = in ? st->G[r + (i0 + u) * ldg] : 0.0;
                    tv[u] = in ? st->T[(i0 + u) + j * m] : 0.0;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (i0 + u < o) acc = fma(gv[u], tv[u], acc);
            }
            val = sub(val, acc);
        }
        st->G[r + (o + j) * ldg] = val;
    }
    __syncthreads();
    // L G for the new columns: block b rows use the upper factor L_b; the newest start row is scaled by 1
    const int rows = o + s + 1;
    for (int t = threadIdx.x; t < rows * s; t += blockDim.x) {
        const int r = t % rows, jj = t / rows, c = o + jj;
        double v;
        if (r < o + s) {
            const int b = r / s, rl = r % s;
            const double* Lb = st->L + b * s * s;
            double lv[kMaxS], gv[kMaxS];   // the loads first, then the multiply-adds in order
#pragma unroll
            for (int q = 0; q < kMaxS; ++q) {
                lv[q] = q < s ? Lb[rl + q * s] : 0.0;
                gv[q] = q < s ? st->G[(b * s + q) + c * ldg] : 0.0;
            }
            double acc = 0.0;
#pragma unroll
            for (int q = 0; q < kMaxS; ++q)
                if (q < s) acc = fma(lv[q], gv[q], acc);
            v = acc;
        } else {
            v = st->G[r + c * ldg];
        }
        sLG[jj * ldg + r] = v;
    }
    __syncthreads();
    (void)kb;
    // the earlier rotations 0..o-1, one thread per new column
    if (threadIdx.x < s) {
        double* h = sLG + threadIdx.x * ldg;
        for (int i = 0; i < o; ++i) {
            const double c = sc_[i], sn = ss_[i];
            const double t = add(mul(c, h[i]), mul(sn, h[i + 1]));
            h[i + 1] = add(mul(-sn, h[i]), mul(c, h[i + 1]));
            h[i] = t;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (o == 0) {
            for (int i = 0; i <= m; ++i) st->g[i] = 0.0;
            st->g[0] = mul(st->beta, st->L[0]);
        }
        double gj = st->g[o];
        double est = 0.0;
        const double nf = st->nf, tol = st->tol;
        int hl = st->hist_len;
        const int hc = st->hist_cap;
        double* hist = st->hist;
        for (int jj = 0; jj < s; ++jj) {
            double* h = sLG + jj * ldg;
            const int c = o + jj;
            for (int i = o; i < c; ++i) {       // rotations of this block's earlier columns
                const double cc = sc_[i], sn = ss_[i];
                const double t = add(mul(cc, h[i]), mul(sn, h[i + 1]));
                h[i + 1] = add(mul(-sn, h[i]), mul(cc, h[i + 1]));
                h[i] = t;
            }
            const double a = h[c], b = h[c + 1];
            const double h2 = add(mul(a, a), mul(b, b)), rh = rsqrt(h2);   // one reciprocal square root
            const double d = mul(h2, rh), cc = mul(a, rh), sn = mul(b, rh);
            sc_[c] = cc;
            ss_[c] = sn;
            h[c] = d;
            h[c + 1] = 0.0;
            const double gn = mul(-sn, gj);
            st->g[c] = mul(cc, gj);
            gj = gn;
            est = fabs(gn);
            if (hl < hc) hist[hl] = est / nf;
            ++hl;
        }
        st->hist_len = hl;
        st->iters += s;
        st->g[o + s] = gj;
        st->K = o + s;
        st->est = est / nf;
        if (est <= tol * nf || !(nu > 0.0) || !isfinite(nu) || e.lastblock) st->building = 0;
    }
    __syncthreads();
    // write back the reduced columns and the new rotations
    for (int t = threadIdx.x; t < rows * s; t += blockDim.x) {
        const int r = t % rows, jj = t / rows;
        st->R[r + (o + jj) * ldg] = sLG[jj * ldg + r];
    }
    for (int i = threadIdx.x; i < s; i += blockDim.x) {
        st->gc[o + i] = sc_[o + i];
        st->gs[o + i] = ss_[o + i];
    }
}

// Standard GMRES, Alg. 2.2 step 1: h_{i,j} = q_i^T A q_j.
__device__ void epi_st_h(const Epi& e, const double* h) {
    SolverState* st = e.st;
    const int j = e.o, ldg = st->m + 1;
    for (int i = threadIdx.x; i <= j; i += blockDim.x) st->G[i + j * ldg] = h[i];
}

// Standard GMRES, steps 3-4 and eq. 2: h_{j+1,j} = ||q^_{j+1}||, Givens, estimate.
// The column and the earlier rotations are staged in shared memory first.
__device__ void epi_st_norm(const Epi& e, double ww) {
    SolverState* st = e.st;
    const int j = e.o, m = st->m, ldg = m + 1;
    __shared__ double h[kMaxM + 1], sc_[kMaxM], ss_[kMaxM];
    for (int i = threadIdx.x; i <= j; i += blockDim.x) h[i] = st->G[i + j * ldg];
    for (int i = threadIdx.x; i < j; i += blockDim.x) {
        sc_[i] = st->gc[i];
        ss_[i] = st->gs[i];
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const double hn = sqrt(ww);
    st->G[(j + 1) + j * ldg] = hn;
    h[j + 1] = hn;
    st->matvecs += 1;
    if (j == 0) {
        for (int i = 0; i <= m; ++i) st->g[i] = 0.0;
        st->g[0] = st->beta;
    }
    for (int i = 0; i < j; ++i) {
        const double c = sc_[i], sn = ss_[i];
        const double t = add(mul(c, h[i]), mul(sn, h[i + 1]));
        h[i + 1] = add(mul(-sn, h[i]), mul(c, h[i + 1]));
        h[i] = t;
    }
    const double a = h[j], b = h[j + 1];
    const double d = sqrt(add(mul(a, a), mul(b, b)));
    const double c = a / d, sn = b / d;
    st->gc[j] = c;
    st->gs[j] = sn;
    h[j] = d;
    h[j + 1] = 0.0;
    for (int i = 0; i <= j + 1; ++i) st->R[i + j * ldg] = h[i];
    const double gj = st->g[j];
    const double est = fabs(mul(-sn, gj));
    st->g[j + 1] = mul(-sn, gj);
    st->g[j] = mul(c, gj);
    hist_push(st, est / st->nf);
    st->iters += 1;
    st->K = j + 1;
    st->nu = hn;
    st->vscale = hn > 0.0 ? 1.0 / hn : 0.0;
    st->est = est / st->nf;
    if (est <= st->tol * st->nf || !(hn > 0.0) || !isfinite(hn) || e.lastblock) st->building = 0;
}

// Orthomin (re)start from the explicit residual.
__device__ void epi_om_restart(SolverState* st, double rr) {
    st->matvecs += 1;
    double rel = sqrt(rr) / st->nf;
    st->relres = rel;
    hist_push(st, rel);
    st->confirm = 0;
    if (!isfinite(rel)) {
        st->status = SSTEP_ERR_NAN;
        st->active = 0;
        st->building = 0;
    } else if (rel <= st->tol) {
        st->status = SSTEP_OK;
        st->active = 0;
        st->building = 0;
    } else if (st->iters >= st->max_iters) {
        st->status = SSTEP_NOT_CONVERGED;
        st->active = 0;
        st->building = 0;
    } else {
        st->cycles += 1;
        st->building = 1;
    }
}

// Orthomin, updated residual after Alg. 3.1 step 4.
__device__ void epi_om_r(SolverState* st, double rr) {
    st->iters += 1;
    double rel = sqrt(rr) / st->nf;
    st->est = rel;
    hist_push(st, rel);
    if (rel <= st->tol || st->iters >= st->max_iters || !isfinite(rel)) {
        st->confirm = 1;
        st->building = 0;
    }
}

// Orthomin Scalar2 (Alg. 3.1 step 7): B_w = -W_w^{-1} C_w for each window block w.
// B is stored in st->T as (nwin*s) x s, col-major, ld kMaxCols.
// e.ortho: C has a last block A R^T A R. The Gram matrix of the projected block
// A R + sum_w A P_w B_w is then W = A R^T A R + sum_w C_w^T B_w (exact arithmetic);
// with W = L^T L, F = L^{-1} makes (A R + sum_w A P_w B_w) F A^T A-orthonormal. F is
// folded into the coefficients (B_w <- B_w F) and stored below them in T (rows
// nwin*s..), so the block update forms the orthonormal block directly. F = I where the
// predicted W is not positive definite.
__device__ void epi_om_B(const Epi& e, const double* C) {
    SolverState* st = e.st;
    const int s = st->s, rows = (e.nwin + e.ortho) * s;
    for (int t = threadIdx.x; t < e.nwin * s; t += blockDim.x) {
        const int w = t / s, j = t % s;
        double rhs[kMaxS], x[kMaxS];
        for (int q = 0; q < s; ++q) rhs[q] = C[(w * s + q) + j * rows];
        chol_solve(st->L + e.win[w] * s * s, s, rhs, x);
        for (int q = 0; q < s; ++q) st->T[(w * s + q) + j * kMaxCols] = -x[q];
    }
    if (!e.ortho) return;
    __syncthreads();
    if (threadIdx.x != 0) return;
    const int o = e.nwin * s;
    double W[kMaxS * kMaxS], L[kMaxS * kMaxS], F[kMaxS * kMaxS];
    for (int j = 0; j < s; ++j)
        for (int q = 0; q <= j; ++q) {
            double t = C[(o + q) + j * rows];
            for (int i = 0; i < o; ++i) t = add(t, mul(C[i + q * rows], st->T[i + j * kMaxCols]));
            W[q + j * s] = t;
        }
    for (int i = 0; i < s * s; ++i) F[i] = 0.0;
    if (chol_upper(W, s, s, L)) {
        for (int c = 0; c < s; ++c) {   // column c of L^{-1}: back substitution, upper triangular
            F[c + c * s] = 1.0 / L[c + c * s];
            for (int i = c - 1; i >= 0; --i) {
                double t = 0.0;
                for (int q = i + 1; q <= c; ++q) t = add(t, mul(L[i + q * s], F[q + c * s]));
                F[i + c * s] = -t / L[i + i * s];
            }
        }
    } else {
        for (int c = 0; c < s; ++c) F[c + c * s] = 1.0;
    }
    for (int i = 0; i < o; ++i) {
        double b[kMaxS];
        for (int q = 0; q < s; ++q) b[q] = st->T[i + q * kMaxCols];
        for (int j = 0; j < s; ++j) {
            double t = 0.0;
            for (int q = 0; q <= j; ++q) t = add(t, mul(b[q], F[q + j * s]));
            st->T[i + j * kMaxCols] = t;
        }
    }
    for (int j = 0; j < s; ++j)
        for (int q = 0; q < s; ++q) st->T[(o + q) + j * kMaxCols] = F[q + j * s];
}

// Orthomin Scalar1 (Alg. 3.1 steps 1-2): W = L^T L, a = W^{-1} m for the new block.
__device__ void epi_om_W(const Epi& e, const double* red) {
    SolverState* st = e.st;
    __shared__ double sW[kMaxS * kMaxS], sLn[kMaxS * kMaxS], sz[kMaxS], sr[kMaxS];   // the factor: formed here, then stored
    if (threadIdx.x >= 32) return;   // one warp
    const int s = st->s, lane = threadIdx.x;
    // W from the packed upper triangle (column q: rows 0..q), then the right-hand side
    for (int t = lane; t < s * s; t += 32) {
        const int p = t % s, q = t / s, lo = p < q ? p : q, hi = p < q ? q : p;
        sW[t] = red[hi * (hi + 1) / 2 + lo];
    }
    __syncwarp();
    const int idx = s * (s + 1) / 2;
    double* Ln = st->L + e.slot * s * s;
    double x;
    const bool ok = chol_solve_warp(sW, s, red + idx, s, sLn, sz, sr, x);
    for (int t = lane; t < s * s; t += 32) Ln[t] = sLn[t];
    if (lane == 0) {
        st->matvecs += s;
        if (!ok) {
            st->status = SSTEP_ERR_BREAKDOWN;
            st->active = 0;
            st->building = 0;
        }
    }
    if (ok && lane < s) st->a[lane] = x;
}

__device__ __noinline__ void run_epilogue(const Epi& e, const double* red, int ka, int kb) {
    switch (e.mode) {
        case EPI_NONE:
            for (int t = threadIdx.x; t < ka * kb; t += blockDim.x) e.out[(t % ka) + (t / ka) * e.ldo] = red[t];
            break;
        case EPI_NF:   // the denominator of every relative residual below
            if (threadIdx.x == 0) {   // f = 0: x = 0 is the solution; test ||f - A x|| itself
                const double nf = sqrt(red[0]);
                e.st->nf = nf > 0.0 ? nf : 1.0;
            }
            break;
        case EPI_FINAL:
            if (threadIdx.x == 0) e.st->relres = sqrt(red[0]) / e.st->nf;
            break;
        case EPI_RESTART:
            if (threadIdx.x == 0) epi_restart(e.st, red[0]);
            break;
        case EPI_GM_T: epi_gm_T(e, red); break;
        case EPI_GM_W: epi_gm_W(e, red); break;
        case EPI_GM_NU: epi_gm_nu(e, red); break;
        case EPI_ST_H: epi_st_h(e, red); break;
        case EPI_ST_NORM: epi_st_norm(e, red[0]); break;
        case EPI_OM_RESTART:
            if (threadIdx.x == 0) epi_om_restart(e.st, red[0]);
            break;
        case EPI_OM_R:
            if (threadIdx.x == 0) epi_om_r(e.st, red[0]);
            break;
        case EPI_OM_B: epi_om_B(e, red); break;
        case EPI_OM_W: epi_om_W(e, red); break;
        default: break;
    }
}

// Second stage of a grid reduction in the last CTA: res[v] = sum over CTAs of
// partials[cta*nv + v]. Each value is summed by a group of G lanes (a power of two,
// as many as the CTA allows): lane l adds CTAs l, l+G, l+2G, ... in order, then the
// group combines its lanes by a fixed shuffle tree, so the order is fixed and the
// result bitwise reproducible. Then the arrival counter is re-armed.
__device__ void finish_reduction(double* res, int nv, int nctas, Scratch sc) {
    int G = 32;
    while (G > 1 && G * nv > (int)blockDim.x) G >>= 1;
    const int ngroups = blockDim.x / G;
    const int g = threadIdx.x / G, l = threadIdx.x % G;
    for (int v0 = 0; v0 < nv; v0 += ngroups) {
        const int v = v0 + g;
        double t = 0.0;
        if (v < nv)
            for (int c = l; c < nctas; c += G) t += ld_cg(sc.partials + (int64_t)c * nv + v);
        for (int off = G / 2; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off, G);
        if (v < nv && l == 0) res[v] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) *sc.counter = 0u;
}

}  // namespace
}  // namespace sstep
