// Streaming kernels of the FP64 path: stencil sweep, residual, tall-skinny Gram,
// block update, Orthomin updates, and the small FP64 work of Scalar1 / Scalar2 /
// the Hessenberg least squares, which runs in the last CTA of each reduction.
#include <math.h>

#include "kernels.cuh"

namespace sstep {

constexpr int kMaxCtas = 152 * 8;      // 8 CTAs of 256 threads per SM at most
constexpr int kGramKA = 8;             // V columns per Gram CTA (grid.y splits ka)
constexpr int kMaxNV = kGramKA * (kMaxS + 1);   // largest per-CTA partial vector

int max_partials_doubles() { return kMaxCtas * kMaxNV; }

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

// x = (L^T L)^{-1} b (forward with L^T, then backward with L); b and x may alias.
__device__ void chol_solve(const double* L, int s, const double* b, double* x) {
    double z[kMaxCols];
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
    for (int t = threadIdx.x; t < nblk * s; t += blockDim.x) {
        const int b = t / s, j = t % s;
        double rhs[kMaxS], x[kMaxS];
        for (int q = 0; q < s; ++q) rhs[q] = C[(b * s + q) + j * o];
        chol_solve(st->L + b * s * s, s, rhs, x);
        for (int q = 0; q < s; ++q) st->T[(b * s + q) + (j + 1) * m] = x[q];
    }
    for (int i = threadIdx.x; i < o; i += blockDim.x) st->T[i] = 0.0;   // first column: 0 (step 7)
}

// Scalar1 of Alg. 4.1 on the projected block: W_k = V_k^T V_k, S = W_k^{-1} V_k^T z.
__device__ void epi_gm_W(const Epi& e, const double* G2) {
    SolverState* st = e.st;
    if (threadIdx.x != 0) return;
    const int s = st->s, o = e.o, ld = s + 1;
    st->matvecs += s;
    double* Lk = st->L + (o / s) * s * s;
    if (!chol_upper(G2, ld, s, Lk)) {
        st->building = 0;
        if (o == 0) {
            st->status = SSTEP_ERR_BREAKDOWN;
            st->active = 0;
        }
        return;
    }
    chol_solve(Lk, s, G2 + s * ld, st->S);
}

// u = z - V_k S has been formed; nu = ||u||. Columns o..o+s-1 of G hold A v_k^j in
// the coordinates of U = [V_1..V_k, v_{k+1}^1] (eq. 4-5), then enter the Givens QR
// of L G (eq. 9) one by one.
__device__ void epi_gm_nu(const Epi& e, const double* red) {
    SolverState* st = e.st;
    const int s = st->s, m = st->m, o = e.o, ldg = m + 1;
    __shared__ double nu_s;
    if (threadIdx.x == 0) {
        double nu = sqrt(red[0]);
        nu_s = nu;
        st->nu = nu;
        st->vscale = nu > 0.0 ? 1.0 / nu : 0.0;
    }
    __syncthreads();
    const double nu = nu_s, sigma = st->sigma;
    for (int r = threadIdx.x; r < ldg; r += blockDim.x) {
        for (int j = 0; j < s; ++j) {
            double raw;
            if (r < o) raw = st->T[r + (j + 1) * m];
            else if (j + 1 < s) raw = (r == o + j + 1) ? 1.0 : 0.0;
            else if (r < o + s) raw = st->S[r - o];
            else raw = (r == o + s) ? nu : 0.0;
            double val = raw / sigma;
            if (o > 0) {
                double acc = 0.0;
                for (int i = 0; i < o; ++i) acc = fma(st->G[r + i * ldg], st->T[i + j * m], acc);
                val = sub(val, acc);
            }
            st->G[r + (o + j) * ldg] = val;
        }
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const int kb = o / s;
    if (o == 0) {
        for (int i = 0; i <= m; ++i) st->g[i] = 0.0;
        st->g[0] = mul(st->beta, st->L[0]);
    }
    double est = 0.0;
    double lg[kMaxM + 1];
    for (int jj = 0; jj < s; ++jj) {
        const int c = o + jj;
        for (int b = 0; b <= kb; ++b) {
            const double* Lb = st->L + b * s * s;
            for (int rl = 0; rl < s; ++rl) {
                double acc = 0.0;
                for (int q = 0; q < s; ++q) acc = fma(Lb[rl + q * s], st->G[(b * s + q) + c * ldg], acc);
                lg[b * s + rl] = acc;
            }
        }
        lg[o + s] = st->G[(o + s) + c * ldg];
        est = givens_add(st, c, lg);
        hist_push(st, est / st->nf);
        st->iters += 1;
    }
    st->K = o + s;
    st->est = est / st->nf;
    if (est <= st->tol * st->nf || !(nu > 0.0) || !isfinite(nu) || e.lastblock) st->building = 0;
}

// Standard GMRES, Alg. 2.2 step 1: h_{i,j} = q_i^T A q_j.
__device__ void epi_st_h(const Epi& e, const double* h) {
    SolverState* st = e.st;
    const int j = e.o, ldg = st->m + 1;
    for (int i = threadIdx.x; i <= j; i += blockDim.x) st->G[i + j * ldg] = h[i];
}

// Standard GMRES, steps 3-4 and eq. 2: h_{j+1,j} = ||q^_{j+1}||, Givens, estimate.
__device__ void epi_st_norm(const Epi& e, double ww) {
    SolverState* st = e.st;
    if (threadIdx.x != 0) return;
    const int j = e.o, m = st->m, ldg = m + 1;
    double hn = sqrt(ww);
    st->G[(j + 1) + j * ldg] = hn;
    st->matvecs += 1;
    if (j == 0) {
        for (int i = 0; i <= m; ++i) st->g[i] = 0.0;
        st->g[0] = st->beta;
    }
    double h[kMaxM + 1];
    for (int i = 0; i <= j + 1; ++i) h[i] = st->G[i + j * ldg];
    double est = givens_add(st, j, h);
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
__device__ void epi_om_B(const Epi& e, const double* C) {
    SolverState* st = e.st;
    const int s = st->s, rows = e.nwin * s;
    for (int t = threadIdx.x; t < e.nwin * s; t += blockDim.x) {
        const int w = t / s, j = t % s;
        double rhs[kMaxS], x[kMaxS];
        for (int q = 0; q < s; ++q) rhs[q] = C[(w * s + q) + j * rows];
        chol_solve(st->L + e.win[w] * s * s, s, rhs, x);
        for (int q = 0; q < s; ++q) st->T[(w * s + q) + j * kMaxCols] = -x[q];
    }
}

// Orthomin Scalar1 (Alg. 3.1 steps 1-2): W = L^T L, a = W^{-1} m for the new block.
__device__ void epi_om_W(const Epi& e, const double* red) {
    SolverState* st = e.st;
    if (threadIdx.x != 0) return;
    const int s = st->s;
    st->matvecs += s;
    double W[kMaxS * kMaxS];
    int idx = 0;
    for (int q = 0; q < s; ++q)
        for (int p = 0; p <= q; ++p) {
            W[p + q * s] = red[idx];
            W[q + p * s] = red[idx];
            ++idx;
        }
    double* Ln = st->L + e.slot * s * s;
    if (!chol_upper(W, s, s, Ln)) {
        st->status = SSTEP_ERR_BREAKDOWN;
        st->active = 0;
        st->building = 0;
        return;
    }
    chol_solve(Ln, s, red + idx, st->a);
}

__device__ __noinline__ void run_epilogue(const Epi& e, const double* red, int ka, int kb) {
    switch (e.mode) {
        case EPI_NONE:
            for (int t = threadIdx.x; t < ka * kb; t += blockDim.x) e.out[(t % ka) + (t / ka) * e.ldo] = red[t];
            break;
        case EPI_NF:
            if (threadIdx.x == 0) e.st->nf = sqrt(red[0]);
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

// Second stage of a grid reduction in the last CTA: out[v] = sum over CTAs (in CTA
// order) of partials[cta*nv + v], for v < nv; then the counter is re-armed.
__device__ void finish_reduction(double* res, int nv, int nctas, Scratch sc) {
    for (int v = threadIdx.x; v < nv; v += blockDim.x) {
        double t = 0.0;
        for (int c = 0; c < nctas; ++c) t += ld_cg(sc.partials + (int64_t)c * nv + v);
        res[v] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) *sc.counter = 0u;
}

// ================================================================== stencil sweep
__device__ __forceinline__ void grid_xyz(const StencilDesc& A, int64_t p, int& x, int& y, int& z) {
    const unsigned up = (unsigned)p;
    const unsigned t = up / (unsigned)A.nx;
    x = (int)(up - t * (unsigned)A.nx);
    const unsigned zz = t / (unsigned)A.ny;
    y = (int)(t - zz * (unsigned)A.ny);
    z = (int)zz;
}

__global__ void __launch_bounds__(kThreads) stencil_kernel(StencilDesc A, const double* __restrict__ v,
                                                           double fy, double* __restrict__ y, double fw,
                                                           double* __restrict__ w, const double* dscale,
                                                           const SolverState* st, int gate) {
    if (!gate_open(st, gate)) return;
    if (dscale) {
        const double d = *dscale;
        fy *= d;
        fw *= d;
    }
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < A.n; p += stride) {
        int x, yy, z;
        grid_xyz(A, p, x, yy, z);
        y[p] = fy * stencil_row(A, v, p, x, yy, z);
        if (w) w[p] = fw * v[p];
    }
}

void launch_stencil(const StencilDesc& A, const double* v, double fy, double* y, double fw, double* w,
                    const double* dscale, const SolverState* st, int gate, cudaStream_t stream) {
    int grid = grid_for(A.n, kMaxCtas);
    stencil_kernel<<<grid, kThreads, 0, stream>>>(A, v, fy, y, fw, w, dscale, st, gate);
}

// ================================================================== residual
__global__ void __launch_bounds__(kThreads) residual_kernel(StencilDesc A, const double* __restrict__ f,
                                                            const double* __restrict__ xv,
                                                            double* __restrict__ out, Scratch sc, Epi epi,
                                                            int gate) {
    __shared__ double red[(kWarps + 1) * 1];
    if (!gate_open(epi.st, gate)) return;
    double acc[1] = {0.0};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < A.n; p += stride) {
        double r = f[p];
        if (xv) {
            int x, yy, z;
            grid_xyz(A, p, x, yy, z);
            r = r - stencil_row(A, xv, p, x, yy, z);
        }
        if (out) out[p] = r;
        acc[0] = fma(r, r, acc[0]);
    }
    block_reduce<1>(acc, red);
    if (!publish_partial(red + kWarps, 1, sc.partials, sc.counter)) return;
    __shared__ double res[1];
    finish_reduction(res, 1, gridDim.x * gridDim.y, sc);
    run_epilogue(epi, res, 1, 1);
}

void launch_residual(const StencilDesc& A, const double* f, const double* x, double* out, Scratch sc,
                     const Epi& epi, int gate, cudaStream_t stream) {
    int grid = grid_for(A.n, kMaxCtas / 2);
    residual_kernel<<<grid, kThreads, 0, stream>>>(A, f, x, out, sc, epi, gate);
}

// ================================================================== Gram pass
// CTA (bx, by) accumulates C[by*KA + i, j] = sum_rows V[row, by*KA+i] Y[row, j] over
// its rows; the last CTA sums the partials of every CTA in CTA order.
template <int KB>
__global__ void __launch_bounds__(kThreads) gram_kernel(int64_t n, const double* __restrict__ V, int64_t ldv,
                                                        int ka, const double* __restrict__ Y, int64_t ldy,
                                                        int win_s, Scratch sc, Epi epi, int gate) {
    constexpr int NV = kGramKA * KB;
    __shared__ double red[(kWarps + 1) * NV];
    __shared__ double res[kMaxCols * (kMaxS + 1)];
    if (!gate_open(epi.st, gate)) return;
    const int a0 = blockIdx.y * kGramKA;
    const int na = min(kGramKA, ka - a0);
    // column offsets of V: contiguous, or (win_s > 0) blocks of win_s columns at the
    // panel slots listed in epi.win (an Orthomin window held in a ring of slots)
    int64_t voff[kGramKA];
#pragma unroll
    for (int i = 0; i < kGramKA; ++i) {
        const int c = min(a0 + i, ka - 1);
        voff[i] = win_s ? ((int64_t)epi.win[c / win_s] * win_s + c % win_s) * ldv : (int64_t)c * ldv;
    }
    double acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
        double yv[KB];
#pragma unroll
        for (int j = 0; j < KB; ++j) yv[j] = __ldg(Y + p + j * ldy);
#pragma unroll
        for (int i = 0; i < kGramKA; ++i) {
            if (i < na) {
                const double a = __ldg(V + p + voff[i]);
#pragma unroll
                for (int j = 0; j < KB; ++j) acc[i * KB + j] = fma(a, yv[j], acc[i * KB + j]);
            }
        }
    }
    block_reduce<NV>(acc, red);
    if (!publish_partial(red + kWarps * NV, NV, sc.partials, sc.counter)) return;
    // second stage: entry (i, j) of C, column-major ka x KB
    const int nctas = gridDim.x * gridDim.y, gx = gridDim.x;
    for (int t = threadIdx.x; t < ka * KB; t += blockDim.x) {
        const int i = t % ka, j = t / ka, by = i / kGramKA, ii = i % kGramKA;
        double s = 0.0;
        for (int bx = 0; bx < gx; ++bx) s += ld_cg(sc.partials + (int64_t)(by * gx + bx) * NV + ii * KB + j);
        res[t] = s;
    }
    (void)nctas;
    __syncthreads();
    if (threadIdx.x == 0) *sc.counter = 0u;
    run_epilogue(epi, res, ka, KB);
}

void launch_gram(int64_t n, const double* V, int64_t ldv, int ka, const double* Y, int64_t ldy, int kb,
                 int win_s, Scratch sc, const Epi& epi, int gate, cudaStream_t stream) {
    const int gy = (ka + kGramKA - 1) / kGramKA;
    int gx = grid_for(n, kMaxCtas / gy > 0 ? kMaxCtas / gy : 1);
    dim3 grid(gx, gy);
    switch (kb) {
#define SSTEP_GRAM_CASE(KB) \
    case KB: gram_kernel<KB><<<grid, kThreads, 0, stream>>>(n, V, ldv, ka, Y, ldy, win_s, sc, epi, gate); break;
        SSTEP_GRAM_CASE(1)
        SSTEP_GRAM_CASE(2)
        SSTEP_GRAM_CASE(3)
        SSTEP_GRAM_CASE(4)
        SSTEP_GRAM_CASE(5)
        SSTEP_GRAM_CASE(6)
        SSTEP_GRAM_CASE(7)
        SSTEP_GRAM_CASE(8)
        SSTEP_GRAM_CASE(9)
#undef SSTEP_GRAM_CASE
        default: break;
    }
}

// ================================================================== block update
template <int KB, bool GRAM>
__global__ void __launch_bounds__(kThreads) update_kernel(int64_t n, const double* __restrict__ V, int64_t ldv,
                                                          int ka, const double* Yin, int64_t ldy, double* Yout,
                                                          int64_t ldo, int j0, const double* __restrict__ T,
                                                          int ldt, double sgn, Scratch sc, Epi epi, int gate) {
    constexpr int NV = GRAM ? KB * (KB + 1) / 2 : 1;
    __shared__ double Ts[kMaxCols * KB];
    __shared__ double red[(kWarps + 1) * NV];
    __shared__ double res[(kMaxS + 1) * (kMaxS + 1)];
    if (!gate_open(epi.st, gate)) return;
    if (ka < 0) {                       // x += U y over the current cycle's K columns
        ka = epi.st->K;
        T = epi.st->y;
        ldt = kMaxCols;
    }
    for (int t = threadIdx.x; t < ka * KB; t += blockDim.x) {
        const int i = t % ka, j = t / ka;
        Ts[i * KB + j] = sgn * T[i + (int64_t)j * ldt];
    }
    __syncthreads();
    double acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = 0.0;
    const bool inplace = (Yin == Yout) && (ldy == ldo);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
        double yv[KB];
#pragma unroll
        for (int j = 0; j < KB; ++j) yv[j] = Yin[p + j * ldy];
        double sum[KB];
#pragma unroll
        for (int j = 0; j < KB; ++j) sum[j] = 0.0;
        for (int i = 0; i < ka; ++i) {
            const double a = __ldg(V + p + (int64_t)i * ldv);
#pragma unroll
            for (int j = 0; j < KB; ++j)
                if (j >= j0) sum[j] = fma(a, Ts[i * KB + j], sum[j]);
        }
#pragma unroll
        for (int j = 0; j < KB; ++j) {
            if (j >= j0 && ka > 0) yv[j] = yv[j] + sum[j];
            if (!inplace || (j >= j0 && ka > 0)) Yout[p + j * ldo] = yv[j];
        }
        if (GRAM) {
            int idx = 0;
#pragma unroll
            for (int q = 0; q < KB; ++q)
#pragma unroll
                for (int pp = 0; pp <= q; ++pp) {
                    acc[idx] = fma(yv[pp], yv[q], acc[idx]);
                    ++idx;
                }
        }
    }
    if (!GRAM) return;
    block_reduce<NV>(acc, red);
    if (!publish_partial(red + kWarps * NV, NV, sc.partials, sc.counter)) return;
    __shared__ double packed[NV];
    finish_reduction(packed, NV, gridDim.x * gridDim.y, sc);
    // expand the packed upper triangle to a full symmetric KB x KB matrix
    for (int t = threadIdx.x; t < KB * KB; t += blockDim.x) {
        int pp = t % KB, q = t / KB;
        if (pp > q) {
            int tmp = pp;
            pp = q;
            q = tmp;
        }
        res[t] = packed[q * (q + 1) / 2 + pp];
    }
    __syncthreads();
    run_epilogue(epi, res, KB, KB);
}

void launch_update(int64_t n, const double* V, int64_t ldv, int ka, const double* Yin, int64_t ldy,
                   double* Yout, int64_t ldo, int kb, int j0, const double* T, int ldt, double sgn,
                   bool gram, Scratch sc, const Epi& epi, int gate, cudaStream_t stream) {
    int grid = grid_for(n, kMaxCtas / 2);
    switch (kb) {
#define SSTEP_UPD_CASE(KB)                                                                                \
    case KB:                                                                                              \
        if (gram)                                                                                         \
            update_kernel<KB, true><<<grid, kThreads, 0, stream>>>(n, V, ldv, ka, Yin, ldy, Yout, ldo, j0, \
                                                                   T, ldt, sgn, sc, epi, gate);          \
        else                                                                                              \
            update_kernel<KB, false><<<grid, kThreads, 0, stream>>>(n, V, ldv, ka, Yin, ldy, Yout, ldo,    \
                                                                    j0, T, ldt, sgn, sc, epi, gate);     \
        break;
        SSTEP_UPD_CASE(1)
        SSTEP_UPD_CASE(2)
        SSTEP_UPD_CASE(3)
        SSTEP_UPD_CASE(4)
        SSTEP_UPD_CASE(5)
        SSTEP_UPD_CASE(6)
        SSTEP_UPD_CASE(7)
        SSTEP_UPD_CASE(8)
        SSTEP_UPD_CASE(9)
#undef SSTEP_UPD_CASE
        default: break;
    }
}

// ================================================================== Orthomin updates
template <int S>
__global__ void __launch_bounds__(kThreads) omin_xr_kernel(int64_t n, const double* __restrict__ P,
                                                           const double* __restrict__ AP, int64_t ld,
                                                           double* __restrict__ x, double* __restrict__ r,
                                                           Scratch sc, Epi epi, int gate) {
    __shared__ double red[(kWarps + 1)];
    __shared__ double as[S];
    if (!gate_open(epi.st, gate)) return;
    if (threadIdx.x < S) as[threadIdx.x] = epi.st->a[threadIdx.x];
    __syncthreads();
    double acc[1] = {0.0};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
        double dx = 0.0, dr = 0.0;
#pragma unroll
        for (int j = 0; j < S; ++j) {
            dx = fma(__ldg(P + p + j * ld), as[j], dx);
            dr = fma(__ldg(AP + p + j * ld), as[j], dr);
        }
        x[p] = x[p] + dx;
        const double rn = r[p] - dr;
        r[p] = rn;
        acc[0] = fma(rn, rn, acc[0]);
    }
    block_reduce<1>(acc, red);
    if (!publish_partial(red + kWarps, 1, sc.partials, sc.counter)) return;
    __shared__ double res[1];
    finish_reduction(res, 1, gridDim.x * gridDim.y, sc);
    run_epilogue(epi, res, 1, 1);
}

void launch_omin_xr(int64_t n, const double* P, const double* AP, int64_t ld, int s, double* x, double* r,
                    Scratch sc, const Epi& epi, int gate, cudaStream_t stream) {
    int grid = grid_for(n, kMaxCtas / 2);
    switch (s) {
#define SSTEP_XR_CASE(S) \
    case S: omin_xr_kernel<S><<<grid, kThreads, 0, stream>>>(n, P, AP, ld, x, r, sc, epi, gate); break;
        SSTEP_XR_CASE(1)
        SSTEP_XR_CASE(2)
        SSTEP_XR_CASE(3)
        SSTEP_XR_CASE(4)
        SSTEP_XR_CASE(5)
        SSTEP_XR_CASE(6)
        SSTEP_XR_CASE(7)
        SSTEP_XR_CASE(8)
#undef SSTEP_XR_CASE
        default: break;
    }
}

// P_new[:, j] = R_j + sum_w sum_q P_w[:, q] B_w[q, j] (same for AP with AR), R_0 = r,
// R_j = sigma AR_{j-1}; reduces W = AP_new^T AP_new (packed) and m = AP_new^T r.
template <int S>
__global__ void __launch_bounds__(kThreads) omin_pupdate_kernel(int64_t n, const double* __restrict__ r,
                                                                const double* __restrict__ AR,
                                                                const double* Ppanel, const double* APpanel,
                                                                int64_t ld, double sigma, Scratch sc, Epi epi,
                                                                int gate) {
    constexpr int NV = S * (S + 1) / 2 + S;
    __shared__ double Bs[kMaxCols * S];
    __shared__ double red[(kWarps + 1) * NV];
    if (!gate_open(epi.st, gate)) return;
    const int nwin = epi.nwin, rows = nwin * S;
    for (int t = threadIdx.x; t < rows * S; t += blockDim.x) {
        const int i = t % rows, j = t / rows;
        Bs[i * S + j] = epi.st->T[i + j * kMaxCols];
    }
    __syncthreads();
    double* Pn = (double*)Ppanel + (int64_t)epi.slot * S * ld;
    double* APn = (double*)APpanel + (int64_t)epi.slot * S * ld;
    double acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
        const double rv = __ldg(r + p);
        double pv[S], apv[S];
#pragma unroll
        for (int j = 0; j < S; ++j) {
            apv[j] = __ldg(AR + p + j * ld);
            pv[j] = (j == 0) ? rv : sigma * __ldg(AR + p + (j - 1) * ld);
        }
        for (int w = 0; w < nwin; ++w) {
            const double* Pw = Ppanel + (int64_t)epi.win[w] * S * ld;
            const double* APw = APpanel + (int64_t)epi.win[w] * S * ld;
            double sp[S], sap[S];
#pragma unroll
            for (int j = 0; j < S; ++j) sp[j] = sap[j] = 0.0;
#pragma unroll
            for (int q = 0; q < S; ++q) {
                const double a = __ldg(Pw + p + q * ld), b = __ldg(APw + p + q * ld);
#pragma unroll
                for (int j = 0; j < S; ++j) {
                    sp[j] = fma(a, Bs[(w * S + q) * S + j], sp[j]);
                    sap[j] = fma(b, Bs[(w * S + q) * S + j], sap[j]);
                }
            }
#pragma unroll
            for (int j = 0; j < S; ++j) {
                pv[j] = pv[j] + sp[j];
                apv[j] = apv[j] + sap[j];
            }
        }
        int idx = 0;
#pragma unroll
        for (int q = 0; q < S; ++q) {
            Pn[p + q * ld] = pv[q];
            APn[p + q * ld] = apv[q];
#pragma unroll
            for (int pp = 0; pp <= q; ++pp) {
                acc[idx] = fma(apv[pp], apv[q], acc[idx]);
                ++idx;
            }
        }
#pragma unroll
        for (int q = 0; q < S; ++q) acc[idx + q] = fma(apv[q], rv, acc[idx + q]);
    }
    block_reduce<NV>(acc, red);
    if (!publish_partial(red + kWarps * NV, NV, sc.partials, sc.counter)) return;
    __shared__ double res[NV];
    finish_reduction(res, NV, gridDim.x * gridDim.y, sc);
    run_epilogue(epi, res, NV, 1);
}

void launch_omin_pupdate(int64_t n, const double* r, const double* AR, const double* Ppanel,
                         const double* APpanel, int64_t ld, int s, double sigma, Scratch sc, const Epi& epi,
                         int gate, cudaStream_t stream) {
    int grid = grid_for(n, kMaxCtas / 2);
    switch (s) {
#define SSTEP_PU_CASE(S)                                                                                 \
    case S:                                                                                              \
        omin_pupdate_kernel<S><<<grid, kThreads, 0, stream>>>(n, r, AR, Ppanel, APpanel, ld, sigma, sc, \
                                                              epi, gate);                               \
        break;
        SSTEP_PU_CASE(1)
        SSTEP_PU_CASE(2)
        SSTEP_PU_CASE(3)
        SSTEP_PU_CASE(4)
        SSTEP_PU_CASE(5)
        SSTEP_PU_CASE(6)
        SSTEP_PU_CASE(7)
        SSTEP_PU_CASE(8)
#undef SSTEP_PU_CASE
        default: break;
    }
}

// ================================================================== least squares solve
__global__ void lsq_solve_kernel(SolverState* st, int gate) {
    if (!gate_open(st, gate)) return;
    if (threadIdx.x != 0) return;
    const int K = st->K, ld = st->m + 1;
    for (int i = K - 1; i >= 0; --i) {
        double t = 0.0;
        for (int q = i + 1; q < K; ++q) t = add(t, mul(st->R[i + q * ld], st->y[q]));
        st->y[i] = sub(st->g[i], t) / st->R[i + i * ld];
    }
}

void launch_lsq_solve(SolverState* st, int gate, cudaStream_t stream) {
    lsq_solve_kernel<<<1, 32, 0, stream>>>(st, gate);
}

}  // namespace sstep
