// Batched s-step GMRES: many independent small systems in one persistent launch.
//
// A CTA, or a thread-block cluster of G CTAs for the largest systems, takes the next
// system from an atomic work queue and runs the whole solve of Alg. 4.1/4.2 on it:
// matrix powers, the inner-product pass, the block update, Scalar1/Scalar2, the
// Hessenberg columns and the Givens least squares, restarts and the x update.
// Reductions are CTA-wide (shuffles and shared memory, fixed order) and, in a
// cooperative solve, cluster-wide through distributed shared memory. No CTA ever
// waits on a CTA outside its own cluster, and inside a cluster only at hardware
// cluster barriers. The scalar work reuses the epilogues of the multi-kernel path,
// which are CTA-level functions.
//
// The queue hands out systems in the order of `order` (largest first by default),
// which balances uneven sizes across the SMs. Block size, CTAs per SM, the cluster
// size and the size from which a system gets a whole cluster are launch parameters
// chosen by the autotuner in capi.cu. A single CTA solves one system at the FP64
// rate of its SM, so without clusters the largest system alone sets the batch time.
#include <cooperative_groups.h>

#include <type_traits>

#include "df64.cuh"
#include "epilogue.cuh"

namespace sstep {

constexpr int kBatchMaxS = 8;
constexpr int kBatchMaxM = 40;

// Rows of one system handled by one CTA: [r0, r1). A system is solved either by one
// CTA (r0 = 0, r1 = n) or cooperatively by the G CTAs of a thread-block cluster, each
// owning a contiguous slice of rows (CO = true). In the cooperative form every CTA
// keeps its own copy of the solver state and runs the scalar epilogues itself on
// bitwise identical inputs (the cluster-wide sums are formed in rank order by every
// CTA), so all copies, and every control decision taken from them, agree; vectors
// are shared through global memory, and data written by another CTA of the cluster
// is read through L2 (__ldcg) after a cluster barrier.
struct Rows {
    int64_t r0, r1;
};

namespace cg = cooperative_groups;

template <bool CO>
__device__ __forceinline__ void step_sync() {
    if constexpr (CO) cg::this_cluster().sync();
    else __syncthreads();
}

// a vector entry that this kernel may have written: from L2 when another CTA of the
// cluster wrote it (after a cluster barrier), else a plain (coherent) load
template <bool CO>
__device__ __forceinline__ double ldv(const double* p) {
    if constexpr (CO) return __ldcg(p);
    else return *p;
}

__device__ __forceinline__ void cta_grid_xyz(const StencilDesc& A, int64_t p, int& x, int& y, int& z) {
    const unsigned up = (unsigned)p;
    const unsigned t = up / (unsigned)A.nx;
    x = (int)(up - t * (unsigned)A.nx);
    const unsigned zz = t / (unsigned)A.ny;
    y = (int)(t - zz * (unsigned)A.ny);
    z = (int)zz;
}

// (A v)_p as stencil_row, with the vector loads through ldv<CO>
template <bool CO>
__device__ __forceinline__ double row_at(const StencilDesc& A, const double* v, int64_t p, int x, int y, int z) {
    double acc = coef(A, 0, p) * ldv<CO>(v + p);
    if (x > 0) acc = fma(coef(A, 1, p), ldv<CO>(v + p - 1), acc);
    if (x < A.nx - 1) acc = fma(coef(A, 2, p), ldv<CO>(v + p + 1), acc);
    if (y > 0) acc = fma(coef(A, 3, p), ldv<CO>(v + p - A.nx), acc);
    if (y < A.ny - 1) acc = fma(coef(A, 4, p), ldv<CO>(v + p + A.nx), acc);
    if (A.dim == 3) {
        const int64_t pl = (int64_t)A.nx * A.ny;
        if (z > 0) acc = fma(coef(A, 5, p), ldv<CO>(v + p - pl), acc);
        if (z < A.nz - 1) acc = fma(coef(A, 6, p), ldv<CO>(v + p + pl), acc);
    }
    return acc;
}

// y = fy (A v); w = fw v when w is set (the scaled start vector of a block); then a
// barrier (cluster-wide when cooperative: the next sweep reads halo rows of y)
template <bool CO>
__device__ void cta_stencil(const StencilDesc& A, Rows R, const double* v, double fy, double* y, double fw, double* w) {
    for (int64_t p = R.r0 + threadIdx.x; p < R.r1; p += blockDim.x) {
        int x, yy, z;
        cta_grid_xyz(A, p, x, yy, z);
        y[p] = fy * row_at<CO>(A, v, p, x, yy, z);
        if (w) w[p] = fw * ldv<CO>(v + p);
    }
    step_sync<CO>();
}

// sum over the CTA of NV per-thread values into out[0..NV) (shared), fixed order; when
// cooperative, then over the cluster's CTAs in rank order (every CTA forms the same sums)
template <int NV, bool CO>
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
    if constexpr (CO) {
        static_assert(NV <= 64, "two entries per thread at 32 threads or more");
        cg::cluster_group cl = cg::this_cluster();
        cl.sync();                                   // every CTA's partial is in its out[]
        double t[2] = {0.0, 0.0};
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int v = threadIdx.x + k * blockDim.x;
            if (v < NV)
                for (unsigned g = 0; g < cl.num_blocks(); ++g) t[k] += cl.map_shared_rank(out, g)[v];
        }
        cl.sync();                                   // all remote reads done before out[] changes
#pragma unroll
        for (int k = 0; k < 2; ++k)
            if (threadIdx.x + k * blockDim.x < NV) out[threadIdx.x + k * blockDim.x] = t[k];
    }
    __syncthreads();
}

// r = f - A x into out, returns ||r||^2 in res[0]
template <bool CO>
__device__ void cta_residual(const StencilDesc& A, Rows R, const double* f, const double* xv, double* out,
                             double* scratch, double* res) {
    double acc[1] = {0.0};
    for (int64_t p = R.r0 + threadIdx.x; p < R.r1; p += blockDim.x) {
        double r = f[p];
        if (xv) {
            int x, yy, z;
            cta_grid_xyz(A, p, x, yy, z);
            r = r - row_at<CO>(A, xv, p, x, yy, z);
        }
        if (out) out[p] = r;
        acc[0] = fma(r, r, acc[0]);
    }
    cta_reduce<1, CO>(acc, scratch, res);
}

// C = V^T Y, V: ka columns (ka <= kBatchMaxM), Y: S columns; C column-major ka x S in res
template <int S, bool CO>
__device__ void cta_gram(Rows R, const double* V, int64_t ld, int ka, const double* Y, double* scratch, double* res) {
    constexpr int KA = 4;
    for (int a0 = 0; a0 < ka; a0 += KA) {
        const int na = min(KA, ka - a0);
        double acc[KA * S];
#pragma unroll
        for (int v = 0; v < KA * S; ++v) acc[v] = 0.0;
        for (int64_t p = R.r0 + threadIdx.x; p < R.r1; p += blockDim.x) {
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
        cta_reduce<KA * S, CO>(acc, scratch, part);
        for (int t = threadIdx.x; t < na * S; t += blockDim.x) {
            const int i = t / S, j = t % S;
            res[(a0 + i) + j * ka] = part[i * S + j];
        }
        __syncthreads();
    }
}

// Y[:, j] -= V T[:, j] for j >= j0 (in place, or into Yout), then the Gram of the
// KB output columns (full KB x KB in res)
template <int KB, bool CO>
__device__ void cta_update(Rows R, const double* V, int64_t ld, int ka, double* Yin, double* Yout, int j0,
                           const double* T, int ldt, double* scratch, double* res) {
    constexpr int NV = KB * (KB + 1) / 2;
    __shared__ double Ts[kBatchMaxM * KB];
    for (int t = threadIdx.x; t < ka * KB; t += blockDim.x) Ts[(t % ka) * KB + t / ka] = -T[(t % ka) + (t / ka) * ldt];
    __syncthreads();
    double acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = 0.0;
    for (int64_t p = R.r0 + threadIdx.x; p < R.r1; p += blockDim.x) {
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
    cta_reduce<NV, CO>(acc, scratch, packed);
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

// back substitution y = R^{-1} g by one warp, column by column from the last (as
// lsq_solve_kernel): lane l owns rows l and l + 32; the reciprocals of the diagonal are
// formed first, off the dependent chain
__device__ void cta_lsq(SolverState* st) {
    if (threadIdx.x >= 32) return;
    static_assert(kBatchMaxM <= 64, "two rows per lane");
    const int K = st->K, ld = st->m + 1, lane = threadIdx.x, i0 = lane, i1 = lane + 32;
    const double* R = st->R;
    const double r0 = i0 < K ? 1.0 / R[i0 + i0 * ld] : 0.0, r1 = i1 < K ? 1.0 / R[i1 + i1 * ld] : 0.0;
    const double g0 = i0 < K ? st->g[i0] : 0.0, g1 = i1 < K ? st->g[i1] : 0.0;
    double t0 = 0.0, t1 = 0.0, y0 = 0.0, y1 = 0.0;
    for (int q = K - 1; q >= 0; --q) {
        const double a0 = i0 < q ? R[i0 + q * ld] : 0.0, a1 = i1 < q ? R[i1 + q * ld] : 0.0;
        if (q == i0) y0 = mul(sub(g0, t0), r0);
        if (q == i1) y1 = mul(sub(g1, t1), r1);
        const double yq = __shfl_sync(0xffffffffu, q < 32 ? y0 : y1, q & 31);
        if (i0 < q) t0 = fma(a0, yq, t0);
        if (i1 < q) t1 = fma(a1, yq, t1);
    }
    if (i0 < K) st->y[i0] = y0;
    if (i1 < K) st->y[i1] = y1;
}

__device__ __forceinline__ int flag(const SolverState* st, int which) { return ((volatile const int*)st)[which]; }

// ================================================================== FP32 basis
// The precision form of the batched solver (precision SSTEP_PREC_FP32): the basis and its
// powers are FP32 columns; every inner product and every projection Y - V T adds exact
// FP32 products in double-float (df64.cuh) and is rounded once; the restart residual, x
// and all scalar work stay FP64. Each restart is then a step of FP32 iterative refinement
// with an FP64 stopping test, as in the single-system FP32 mode. The FP64 pipe, which a
// CTA of the FP64 form keeps busy, is left with the residual and the x update.

template <bool CO>
__device__ __forceinline__ float ldf(const float* p) {
    if constexpr (CO) return __ldcg(p);
    else return *p;
}

__device__ __forceinline__ float coef32(const StencilDesc& A, int q, int64_t p) {
    return A.variable ? __ldg(A.fdf[q] + p).x : A.ch[q];
}

// (A v)_p in FP32 (the coefficients' high parts), the same order as row_at
template <bool CO>
__device__ __forceinline__ float row32(const StencilDesc& A, const float* v, int64_t p, int x, int y, int z) {
    float acc = __fmul_rn(coef32(A, 0, p), ldf<CO>(v + p));
    if (x > 0) acc = __fmaf_rn(coef32(A, 1, p), ldf<CO>(v + p - 1), acc);
    if (x < A.nx - 1) acc = __fmaf_rn(coef32(A, 2, p), ldf<CO>(v + p + 1), acc);
    if (y > 0) acc = __fmaf_rn(coef32(A, 3, p), ldf<CO>(v + p - A.nx), acc);
    if (y < A.ny - 1) acc = __fmaf_rn(coef32(A, 4, p), ldf<CO>(v + p + A.nx), acc);
    if (A.dim == 3) {
        const int64_t pl = (int64_t)A.nx * A.ny;
        if (z > 0) acc = __fmaf_rn(coef32(A, 5, p), ldf<CO>(v + p - pl), acc);
        if (z < A.nz - 1) acc = __fmaf_rn(coef32(A, 6, p), ldf<CO>(v + p + pl), acc);
    }
    return acc;
}

// y = fy (A v); w = fw v when w is set; then a barrier (as cta_stencil)
template <bool CO>
__device__ void cta_stencil32(const StencilDesc& A, Rows R, const float* v, float fy, float* y, float fw, float* w) {
    for (int64_t p = R.r0 + threadIdx.x; p < R.r1; p += blockDim.x) {
        int x, yy, z;
        cta_grid_xyz(A, p, x, yy, z);
        y[p] = __fmul_rn(fy, row32<CO>(A, v, p, x, yy, z));
        if (w) w[p] = __fmul_rn(fw, ldf<CO>(v + p));
    }
    step_sync<CO>();
}

// r = f - A x in FP64, stored rounded to FP32 into out; ||r||^2 (FP64) in res[0]
template <bool CO>
__device__ void cta_residual32(const StencilDesc& A, Rows R, const double* f, const double* xv, float* out,
                               double* scratch, double* res) {
    double acc[1] = {0.0};
    for (int64_t p = R.r0 + threadIdx.x; p < R.r1; p += blockDim.x) {
        int x, yy, z;
        cta_grid_xyz(A, p, x, yy, z);
        const double r = f[p] - row_at<CO>(A, xv, p, x, yy, z);
        out[p] = __double2float_rn(r);
        acc[0] = fma(r, r, acc[0]);
    }
    cta_reduce<1, CO>(acc, scratch, res);
}

// s += a b (a FP32, b a float pair): the product's two parts exactly, then TwoSum into s
__device__ __forceinline__ void acc_fd(DfAcc& s, float a, df64 b) {
    const float p = __fmul_rn(a, b.hi);
    float e = __fmaf_rn(a, b.hi, -p);
    e = __fmaf_rn(a, b.lo, e);
    float h, t;
    two_sum(s.hi, p, h, t);
    s.hi = h;
    s.lo = __fadd_rn(s.lo, __fadd_rn(t, e));
}

// C = V^T Y (FP32 columns, double-float sums, FP64 across threads); as cta_gram
template <int S, bool CO>
__device__ void cta_gram32(Rows R, const float* V, int64_t ld, int ka, const float* Y, double* scratch, double* res) {
    constexpr int KA = 4;
    for (int a0 = 0; a0 < ka; a0 += KA) {
        const int na = min(KA, ka - a0);
        DfAcc acc[KA * S];
        int cnt = 0;
        for (int64_t p = R.r0 + threadIdx.x; p < R.r1; p += blockDim.x) {
            float yv[S];
#pragma unroll
            for (int j = 0; j < S; ++j) yv[j] = Y[p + j * ld];
#pragma unroll
            for (int i = 0; i < KA; ++i)
                if (i < na) {
                    const float a = V[p + (int64_t)(a0 + i) * ld];
#pragma unroll
                    for (int j = 0; j < S; ++j) acc[i * S + j].add_prod(a, yv[j]);
                }
            if (++cnt == 32) {   // keep each error term within a few ulps of its sum
                cnt = 0;
#pragma unroll
                for (int v = 0; v < KA * S; ++v) acc[v].normalize();
            }
        }
        double accd[KA * S];
#pragma unroll
        for (int v = 0; v < KA * S; ++v) accd[v] = acc[v].value();
        __shared__ double part[KA * S];
        cta_reduce<KA * S, CO>(accd, scratch, part);
        for (int t = threadIdx.x; t < na * S; t += blockDim.x) {
            const int i = t / S, j = t % S;
            res[(a0 + i) + j * ka] = part[i * S + j];
        }
        __syncthreads();
    }
}

// Y[:, j] -= V T[:, j] for j >= j0 (in place, or into Yout): y + sum_a V_a (-T_aj) in
// double-float, rounded once to FP32; then the Gram of the KB output columns as stored
template <int KB, bool CO>
__device__ void cta_update32(Rows R, const float* V, int64_t ld, int ka, float* Yin, float* Yout, int j0,
                             const double* T, int ldt, double* scratch, double* res) {
    constexpr int NV = KB * (KB + 1) / 2;
    __shared__ df64 Ts[kBatchMaxM * KB];
    for (int t = threadIdx.x; t < ka * KB; t += blockDim.x)
        Ts[(t % ka) * KB + t / ka] = df_from_double(-T[(t % ka) + (t / ka) * ldt]);
    __syncthreads();
    DfAcc acc[NV];
    int cnt = 0;
    for (int64_t p = R.r0 + threadIdx.x; p < R.r1; p += blockDim.x) {
        float yv[KB];
        DfAcc sum[KB];
#pragma unroll
        for (int j = 0; j < KB; ++j) {
            yv[j] = Yin[p + j * ld];
            sum[j].hi = yv[j];
        }
        for (int i = 0; i < ka; ++i) {
            const float a = V[p + (int64_t)i * ld];
#pragma unroll
            for (int j = 0; j < KB; ++j)
                if (j >= j0) acc_fd(sum[j], a, Ts[i * KB + j]);
        }
#pragma unroll
        for (int j = 0; j < KB; ++j) {
            if (j >= j0 && ka > 0) yv[j] = __fadd_rn(sum[j].hi, sum[j].lo);
            if (Yout != Yin || (j >= j0 && ka > 0)) Yout[p + j * ld] = yv[j];
        }
        int idx = 0;
#pragma unroll
        for (int q = 0; q < KB; ++q)
#pragma unroll
            for (int pp = 0; pp <= q; ++pp) {
                acc[idx].add_prod(yv[pp], yv[q]);
                ++idx;
            }
        if (++cnt == 32) {
            cnt = 0;
#pragma unroll
            for (int v = 0; v < NV; ++v) acc[v].normalize();
        }
    }
    double accd[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) accd[v] = acc[v].value();
    __shared__ double packed[NV];
    cta_reduce<NV, CO>(accd, scratch, packed);
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

// One whole s-step GMRES solve of one system, by one CTA (CO = false) or by the CTAs
// of a cluster (CO = true; st is this CTA's own copy of the state).
template <int S, bool CO, bool F32>
__device__ void cta_solve(const BatchSys& b, SolverState* st, Rows R, double* scratch) {
    using T = typename std::conditional<F32, float, double>::type;   // the basis type
    const StencilDesc& A = b.A;
    const int64_t ld = b.ld;
    const int m = st->m, nb = m / S;
    T* U = reinterpret_cast<T*>(b.U);
    T* uraw = U + (int64_t)(m + 1) * ld;
    __shared__ double res[kBatchMaxM * (kBatchMaxS + 1)];
    Epi e;
    e.st = st;
    cta_residual<CO>(A, R, b.f, nullptr, nullptr, scratch, res);
    e.mode = EPI_NF;
    run_epilogue(e, res, 1, 1);
    __syncthreads();
    if (st->pad_) {   // x0 guard: restart from zero when ||f - A x0|| > ||f||
        cta_residual<CO>(A, R, b.f, b.x, nullptr, scratch, res);
        const bool bad = !(res[0] <= st->nf * st->nf);
        __syncthreads();
        if (bad)
            for (int64_t p = R.r0 + threadIdx.x; p < R.r1; p += blockDim.x) b.x[p] = 0.0;
        step_sync<CO>();
    }
    for (;;) {
        if constexpr (F32) cta_residual32<CO>(A, R, b.f, b.x, uraw, scratch, res);
        else cta_residual<CO>(A, R, b.f, b.x, uraw, scratch, res);
        e.mode = EPI_RESTART;
        run_epilogue(e, res, 1, 1);
        __syncthreads();
        if (!flag(st, 0)) break;
        for (int k = 0; k < nb; ++k) {
            if (!flag(st, 1)) break;
            const int o = k * S;
            const double vs = st->vscale, sigma = st->sigma;
            if constexpr (F32) {
                cta_stencil32<CO>(A, R, uraw, __double2float_rn(sigma * vs), U + (o + 1) * ld, __double2float_rn(vs),
                                  U + o * ld);
                for (int j = 2; j <= S; ++j)
                    cta_stencil32<CO>(A, R, U + (o + j - 1) * ld, __double2float_rn(sigma), U + (o + j) * ld, 0.f,
                                      nullptr);
            } else {
                cta_stencil<CO>(A, R, uraw, sigma * vs, U + (o + 1) * ld, vs, U + o * ld);
                for (int j = 2; j <= S; ++j)
                    cta_stencil<CO>(A, R, U + (o + j - 1) * ld, sigma, U + (o + j) * ld, 0.0, nullptr);
            }
            if (k > 0) {
                if constexpr (F32) cta_gram32<S, CO>(R, U, ld, o, U + (o + 1) * ld, scratch, res);
                else cta_gram<S, CO>(R, U, ld, o, U + (o + 1) * ld, scratch, res);
                e.mode = EPI_GM_T;
                e.o = o;
                run_epilogue(e, res, o, S);
                __syncthreads();
            }
            if constexpr (F32) cta_update32<S + 1, CO>(R, U, ld, o, U + o * ld, U + o * ld, 1, st->T, m, scratch, res);
            else cta_update<S + 1, CO>(R, U, ld, o, U + o * ld, U + o * ld, 1, st->T, m, scratch, res);
            e.mode = EPI_GM_W;
            e.o = o;
            run_epilogue(e, res, S + 1, S + 1);
            __syncthreads();
            if (!flag(st, 1)) break;
            if constexpr (F32) cta_update32<1, CO>(R, U + o * ld, ld, S, U + (o + S) * ld, uraw, 0, st->S, S, scratch, res);
            else cta_update<1, CO>(R, U + o * ld, ld, S, U + (o + S) * ld, uraw, 0, st->S, S, scratch, res);
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
        if constexpr (F32) {   // y as float pairs; the sum in double-float, added to x in FP64
            __shared__ df64 ys[kBatchMaxM];
            for (int i = threadIdx.x; i < K; i += blockDim.x) ys[i] = df_from_double(st->y[i]);
            __syncthreads();
            for (int64_t p = R.r0 + threadIdx.x; p < R.r1; p += blockDim.x) {
                DfAcc acc;
                for (int i = 0; i < K; ++i) acc_fd(acc, U[p + (int64_t)i * ld], ys[i]);
                b.x[p] = b.x[p] + acc.value();
            }
        } else {
            for (int64_t p = R.r0 + threadIdx.x; p < R.r1; p += blockDim.x) {
                double acc = 0.0;
                for (int i = 0; i < K; ++i) acc = fma(U[p + (int64_t)i * ld], st->y[i], acc);
                b.x[p] = b.x[p] + acc;
            }
        }
        step_sync<CO>();   // the next residual reads halo rows of x
    }
    cta_residual<CO>(A, R, b.f, b.x, nullptr, scratch, res);
    e.mode = EPI_FINAL;
    run_epilogue(e, res, 1, 1);
    __syncthreads();
}

// Persistent loop. Rank 0 of each cluster takes the next system from the queue; a
// system with at least nbig unknowns is solved by all G CTAs of the cluster together,
// otherwise rank 0 takes G - 1 more and every CTA solves one alone. The queue order
// is largest first, so the cooperative systems come first and the G systems of an
// independent round have similar sizes. Every cluster barrier below is reached by all
// CTAs of the cluster: the round's items are read from rank 0, and the cooperative
// solve's branches come from identical state copies.
template <int S, bool F32>
__global__ void __launch_bounds__(256) batched_sstep_gmres_kernel(const BatchSys* __restrict__ sys,
                                                                  const int* __restrict__ order, int nsys,
                                                                  unsigned* queue, int64_t nbig) {
    extern __shared__ double scratch[];   // (blockDim/32) x 45 doubles for the CTA reductions
    __shared__ int items[8];
    __shared__ int round_coop;
    __shared__ int mine[2];
    cg::cluster_group cl = cg::this_cluster();
    const int G = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    for (;;) {
        if (rank == 0 && threadIdx.x == 0) {
            const int i = (int)atomicAdd(queue, 1u);
            const int coop = G > 1 && i < nsys && sys[order ? order[i] : i].A.n >= nbig;
            items[0] = i;
            if (!coop && G > 1) {
                const int j = (int)atomicAdd(queue, (unsigned)(G - 1));
                for (int g = 1; g < G; ++g) items[g] = j + g - 1;
            }
            round_coop = coop;
        }
        cl.sync();
        if (threadIdx.x == 0) {
            const int* it = cl.map_shared_rank(items, 0);
            const int co = *cl.map_shared_rank(&round_coop, 0);
            mine[0] = co ? it[0] : it[rank];
            mine[1] = co | (it[0] >= nsys ? 2 : 0);
        }
        cl.sync();   // rank 0's items are read before they can change
        const int item = mine[0], mode = mine[1];
        if (mode & 2) break;                 // the queue is empty (the same in every CTA)
        if (mode & 1) {
            const BatchSys& b = sys[order ? order[item] : item];
            const int64_t n = b.A.n;
            const Rows R{n * rank / G, n * (rank + 1) / G};
            SolverState* st = (SolverState*)((char*)b.st + (int64_t)rank * b.st_stride);
            cta_solve<S, true, F32>(b, st, R, scratch);
        } else if (item < nsys) {
            const BatchSys& b = sys[order ? order[item] : item];
            cta_solve<S, false, F32>(b, b.st, Rows{0, b.A.n}, scratch);
        }
        cl.sync();   // the round is over in every CTA before rank 0 takes the next items
    }
}

size_t batched_scratch_bytes(int threads) { return sizeof(double) * (threads / 32) * 45; }

__global__ void batch_init_kernel(const SolverState* __restrict__ src, const BatchSys* __restrict__ sys, int nsys) {
    const int c = blockIdx.x, i = c / kBatchCopies, g = c % kBatchCopies;
    if (i >= nsys) return;
    const unsigned* s = (const unsigned*)(src + c);
    unsigned* d = (unsigned*)((char*)sys[i].st + (int64_t)g * sys[i].st_stride);
    for (int w = threadIdx.x; w < (int)(sizeof(SolverState) / sizeof(unsigned)); w += blockDim.x) d[w] = s[w];
}

void launch_batch_init(const SolverState* src, const BatchSys* sys, int nsys, cudaStream_t stream) {
    static_assert(sizeof(SolverState) % sizeof(unsigned) == 0, "state is copied in 32-bit words");
    batch_init_kernel<<<nsys * kBatchCopies, 64, 0, stream>>>(src, sys, nsys);
}

template <int S>
cudaLaunchConfig_t batched_config(int threads, int grid, int cluster, cudaLaunchAttribute* at, cudaStream_t stream) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = batched_scratch_bytes(threads);
    cfg.stream = stream;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cfg;
}

template <int S, bool F32>
int batched_grid_s(int threads, int ctas, int cluster) {
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = batched_config<S>(threads, (ctas / cluster) * cluster, cluster, at, nullptr);
    int maxc = 0;
    if (cfg.gridDim.x < 1 ||
        cudaOccupancyMaxActiveClusters(&maxc, batched_sstep_gmres_kernel<S, F32>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    int nclu = ctas / cluster;              // a persistent grid: no more clusters than fit at once
    if (nclu > maxc) nclu = maxc;
    return nclu >= 1 ? nclu * cluster : -1;
}

int batched_grid(int s, int threads, int ctas, int cluster, bool f32) {
    if (cluster < 1 || cluster > kBatchCopies || threads > 256 || threads % 32) return -1;
    switch (s) {
#define SSTEP_BG(S_) \
    case S_: return f32 ? batched_grid_s<S_, true>(threads, ctas, cluster) : batched_grid_s<S_, false>(threads, ctas, cluster);
        SSTEP_BG(1)
        SSTEP_BG(2)
        SSTEP_BG(4)
        SSTEP_BG(8)
#undef SSTEP_BG
        default: return -1;
    }
}

template <int S, bool F32>
int launch_batched_s(const BatchSys* sys, const int* order, int nsys, unsigned* queue, int threads, int grid,
                     int cluster, int64_t nbig, cudaStream_t stream) {
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = batched_config<S>(threads, grid, cluster, at, stream);
    return cudaLaunchKernelEx(&cfg, batched_sstep_gmres_kernel<S, F32>, sys, order, nsys, queue, nbig) == cudaSuccess
               ? 0
               : -1;
}

int launch_batched(const BatchSys* sys, const int* order, int nsys, unsigned* queue, int s, int threads, int grid,
                   int cluster, int64_t nbig, bool f32, cudaStream_t stream) {
    if (cluster < 1 || cluster > kBatchCopies || threads > 256 || threads % 32 || grid < cluster || grid % cluster)
        return -1;
    switch (s) {
#define SSTEP_LB(S_)                                                                                           \
    case S_:                                                                                                   \
        return f32 ? launch_batched_s<S_, true>(sys, order, nsys, queue, threads, grid, cluster, nbig, stream)  \
                   : launch_batched_s<S_, false>(sys, order, nsys, queue, threads, grid, cluster, nbig, stream);
        SSTEP_LB(1)
        SSTEP_LB(2)
        SSTEP_LB(4)
        SSTEP_LB(8)
#undef SSTEP_LB
        default: return -1;
    }
}

}  // namespace sstep
