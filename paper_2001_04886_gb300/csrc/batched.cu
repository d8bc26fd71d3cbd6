// Batched s-step GMRES: many independent small systems in one persistent launch.
//
// Each CTA takes the next system from an atomic work queue and runs the whole
// solve of Alg. 4.1/4.2 on it: matrix powers, the inner-product pass, the block
// update, Scalar1/Scalar2, the Hessenberg columns and the Givens least squares,
// restarts and the x update. Reductions are CTA-wide (shuffles and shared
// memory, fixed order), so no grid-wide synchronisation and no waiting on other
// CTAs is needed: CTAs only ever wait at __syncthreads. The scalar work reuses
// the epilogues of the multi-kernel path, which are CTA-level functions.
//
// The queue hands out systems in the order of `order` (largest first by
// default), which balances uneven sizes across the SMs. Block size and CTAs per
// SM are launch parameters chosen by the autotuner in capi.cu.
#include "epilogue.cuh"

namespace sstep {

constexpr int kBatchMaxS = 8;
constexpr int kBatchMaxM = 40;

// CTA-level helpers ---------------------------------------------------------------

__device__ __forceinline__ void cta_grid_xyz(const StencilDesc& A, int64_t p, int& x, int& y, int& z) {
    const unsigned up = (unsigned)p;
    const unsigned t = up / (unsigned)A.nx;
    x = (int)(up - t * (unsigned)A.nx);
    const unsigned zz = t / (unsigned)A.ny;
    y = (int)(t - zz * (unsigned)A.ny);
    z = (int)zz;
}

// y = fy (A v); w = fw v when w is set (the scaled start vector of a block)
__device__ void cta_stencil(const StencilDesc& A, const double* v, double fy, double* y, double fw, double* w) {
    for (int64_t p = threadIdx.x; p < A.n; p += blockDim.x) {
        int x, yy, z;
        cta_grid_xyz(A, p, x, yy, z);
        y[p] = fy * stencil_row(A, v, p, x, yy, z);
        if (w) w[p] = fw * v[p];
    }
    __syncthreads();
}

// sum over the CTA of NV per-thread values into out[0..NV) (shared), fixed order
template <int NV>
__device__ __forceinline__ void cta_reduce(double (&acc)[NV], double* scratch, double* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        double t = warp_sum(acc[v]);
        if (lane == 0) scratch[warp * NV + v] = t;
    }
    __syncthreads();
    for (int v = threadIdx.x; v < NV; v += blockDim.x) {
        double t = 0.0;
        for (int w = 0; w < nw; ++w) t += scratch[w * NV + v];
        out[v] = t;
    }
    __syncthreads();
}

// r = f - A x into out, returns ||r||^2 in res[0]
__device__ void cta_residual(const StencilDesc& A, const double* f, const double* xv, double* out, double* scratch,
                             double* res) {
    double acc[1] = {0.0};
    for (int64_t p = threadIdx.x; p < A.n; p += blockDim.x) {
        double r = f[p];
        if (xv) {
            int x, yy, z;
            cta_grid_xyz(A, p, x, yy, z);
            r = r - stencil_row(A, xv, p, x, yy, z);
        }
        if (out) out[p] = r;
        acc[0] = fma(r, r, acc[0]);
    }
    cta_reduce<1>(acc, scratch, res);
}

// C = V^T Y, V: ka columns (ka <= kBatchMaxM), Y: S columns; C column-major ka x S in res
template <int S>
__device__ void cta_gram(int64_t n, const double* V, int64_t ld, int ka, const double* Y, double* scratch,
                         double* res) {
    constexpr int KA = 4;
    for (int a0 = 0; a0 < ka; a0 += KA) {
        const int na = min(KA, ka - a0);
        double acc[KA * S];
#pragma unroll
        for (int v = 0; v < KA * S; ++v) acc[v] = 0.0;
        for (int64_t p = threadIdx.x; p < n; p += blockDim.x) {
            double yv[S];
#pragma unroll
            for (int j = 0; j < S; ++j) yv[j] = Y[p + j * ld];
#pragma unroll
            for (int i = 0; i < KA; ++i)
                if (i < na) {
                    const double a = V[p + (int64_t)(a0 + i) * ld];
#pragma unroll
                    for (int j = 0; j < S; ++j) acc[i * S + j] = fma(a, yv[j], acc[i * S + j]);
                }
        }
        __shared__ double part[KA * S];
        cta_reduce<KA * S>(acc, scratch, part);
        for (int t = threadIdx.x; t < na * S; t += blockDim.x) {
            const int i = t / S, j = t % S;
            res[(a0 + i) + j * ka] = part[i * S + j];
        }
        __syncthreads();
    }
}

// Y[:, j] -= V T[:, j] for j >= j0 (in place, or into Yout), then the Gram of the
// KB output columns (full KB x KB in res)
template <int KB>
__device__ void cta_update(int64_t n, const double* V, int64_t ld, int ka, double* Yin, double* Yout, int j0,
                           const double* T, int ldt, double* scratch, double* res) {
    constexpr int NV = KB * (KB + 1) / 2;
    __shared__ double Ts[kBatchMaxM * KB];
    for (int t = threadIdx.x; t < ka * KB; t += blockDim.x) Ts[(t % ka) * KB + t / ka] = -T[(t % ka) + (t / ka) * ldt];
    __syncthreads();
    double acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = 0.0;
    for (int64_t p = threadIdx.x; p < n; p += blockDim.x) {
        double yv[KB], sum[KB];
#pragma unroll
        for (int j = 0; j < KB; ++j) {
            yv[j] = Yin[p + j * ld];
            sum[j] = 0.0;
        }
        for (int i = 0; i < ka; ++i) {
            const double a = V[p + (int64_t)i * ld];
#pragma unroll
            for (int j = 0; j < KB; ++j)
                if (j >= j0) sum[j] = fma(a, Ts[i * KB + j], sum[j]);
        }
#pragma unroll
        for (int j = 0; j < KB; ++j) {
            if (j >= j0 && ka > 0) yv[j] = yv[j] + sum[j];
            if (Yout != Yin || (j >= j0 && ka > 0)) Yout[p + j * ld] = yv[j];
        }
        int idx = 0;
#pragma unroll
        for (int q = 0; q < KB; ++q)
#pragma unroll
            for (int pp = 0; pp <= q; ++pp) {
                acc[idx] = fma(yv[pp], yv[q], acc[idx]);
                ++idx;
            }
    }
    __shared__ double packed[NV];
    cta_reduce<NV>(acc, scratch, packed);
    for (int t = threadIdx.x; t < KB * KB; t += blockDim.x) {
        int pp = t % KB, q = t / KB;
        if (pp > q) {
            const int tmp = pp;
            pp = q;
            q = tmp;
        }
        res[t] = packed[q * (q + 1) / 2 + pp];
    }
    __syncthreads();
}

// back substitution y = R^{-1} g by one warp (the dot products as warp reductions)
__device__ void cta_lsq(SolverState* st) {
    if (threadIdx.x >= 32) return;
    const int K = st->K, ld = st->m + 1, lane = threadIdx.x;
    for (int i = K - 1; i >= 0; --i) {
        double t = 0.0;
        for (int q = i + 1 + lane; q < K; q += 32) t = fma(st->R[i + q * ld], st->y[q], t);
        t = warp_sum(t);
        if (lane == 0) st->y[i] = sub(st->g[i], t) / st->R[i + i * ld];
        __syncwarp();
    }
}

__device__ __forceinline__ int flag(const SolverState* st, int which) { return ((volatile const int*)st)[which]; }

// One whole s-step GMRES solve of one system by one CTA.
template <int S>
__device__ void cta_solve(const BatchSys& b, double* scratch) {
    const StencilDesc& A = b.A;
    SolverState* st = b.st;
    const int64_t n = A.n, ld = b.ld;
    const int m = st->m, nb = m / S;
    double* U = b.U;
    double* uraw = U + (int64_t)(m + 1) * ld;
    __shared__ double res[kBatchMaxM * (kBatchMaxS + 1)];
    Epi e;
    e.st = st;
    cta_residual(A, b.f, nullptr, nullptr, scratch, res);
    e.mode = EPI_NF;
    run_epilogue(e, res, 1, 1);
    __syncthreads();
    if (st->pad_) {   // x0 guard: restart from zero when ||f - A x0|| > ||f||
        cta_residual(A, b.f, b.x, nullptr, scratch, res);
        const bool bad = !(res[0] <= st->nf * st->nf);
        __syncthreads();
        if (bad)
            for (int64_t p = threadIdx.x; p < n; p += blockDim.x) b.x[p] = 0.0;
        __syncthreads();
    }
    for (;;) {
        cta_residual(A, b.f, b.x, uraw, scratch, res);
        e.mode = EPI_RESTART;
        run_epilogue(e, res, 1, 1);
        __syncthreads();
        if (!flag(st, 0)) break;
        for (int k = 0; k < nb; ++k) {
            if (!flag(st, 1)) break;
            const int o = k * S;
            const double vs = st->vscale, sigma = st->sigma;
            cta_stencil(A, uraw, sigma * vs, U + (o + 1) * ld, vs, U + o * ld);
            for (int j = 2; j <= S; ++j) cta_stencil(A, U + (o + j - 1) * ld, sigma, U + (o + j) * ld, 0.0, nullptr);
            if (k > 0) {
                cta_gram<S>(n, U, ld, o, U + (o + 1) * ld, scratch, res);
                e.mode = EPI_GM_T;
                e.o = o;
                run_epilogue(e, res, o, S);
                __syncthreads();
            }
            cta_update<S + 1>(n, U, ld, o, U + o * ld, U + o * ld, 1, st->T, m, scratch, res);
            e.mode = EPI_GM_W;
            e.o = o;
            run_epilogue(e, res, S + 1, S + 1);
            __syncthreads();
            if (!flag(st, 1)) break;
            cta_update<1>(n, U + o * ld, ld, S, U + (o + S) * ld, uraw, 0, st->S, S, scratch, res);
            e.mode = EPI_GM_NU;
            e.o = o;
            e.lastblock = (k == nb - 1);
            run_epilogue(e, res, 1, 1);
            __syncthreads();
        }
        cta_lsq(st);
        __syncthreads();
        // x += U y
        const int K = st->K;
        for (int64_t p = threadIdx.x; p < n; p += blockDim.x) {
            double acc = 0.0;
            for (int i = 0; i < K; ++i) acc = fma(U[p + (int64_t)i * ld], st->y[i], acc);
            b.x[p] = b.x[p] + acc;
        }
        __syncthreads();
    }
    cta_residual(A, b.f, b.x, nullptr, scratch, res);
    e.mode = EPI_FINAL;
    run_epilogue(e, res, 1, 1);
    __syncthreads();
}

template <int S>
__global__ void __launch_bounds__(256) batched_sstep_gmres_kernel(const BatchSys* __restrict__ sys, const int* __restrict__ order, int nsys,
                                           unsigned* queue) {
    extern __shared__ double scratch[];   // (blockDim/32) x 45 doubles for the CTA reductions
    __shared__ int next;
    for (;;) {
        if (threadIdx.x == 0) next = (int)atomicAdd(queue, 1u);
        __syncthreads();
        const int i = next;
        __syncthreads();
        if (i >= nsys) break;
        cta_solve<S>(sys[order ? order[i] : i], scratch);
    }
}

size_t batched_scratch_bytes(int threads) { return sizeof(double) * (threads / 32) * 45; }

int launch_batched(const BatchSys* sys, const int* order, int nsys, unsigned* queue, int s, int threads, int ctas,
                   cudaStream_t stream) {
    const size_t smem = batched_scratch_bytes(threads);
    switch (s) {
#define SSTEP_BAT(S)                                                                                         \
    case S:                                                                                                  \
        batched_sstep_gmres_kernel<S><<<ctas, threads, smem, stream>>>(sys, order, nsys, queue);            \
        break;
        SSTEP_BAT(1)
        SSTEP_BAT(2)
        SSTEP_BAT(4)
        SSTEP_BAT(8)
#undef SSTEP_BAT
        default: return -1;
    }
    return 0;
}

}  // namespace sstep
