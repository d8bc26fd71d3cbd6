// Mixed-precision basis kernels: the s-step block with its Krylov basis stored in
// double-float pairs (PREC_DF64) or in FP32 (PREC_FP32).
//
// GB300 runs FP64 FMAs at 1/64 of its FP32 rate, so the FP64 kernels of this
// path are FP64-pipe bound. These variants keep every byte-heavy vector operation
// on the FP32 pipe: double-float arithmetic (48-bit significand) for PREC_DF64,
// FP32 storage with double-float accumulation for PREC_FP32. Every projection
// Y - V T is summed in double-float and rounded once (FP32 arithmetic there
// loses the cancellation and doubles the cycles of FP32 refinement at s = 8).
// The right-hand side, the iterate, the explicit residuals and all scalar work
// (Cholesky, least squares) stay FP64.
//
// The row loops are software-pipelined: the loads of the next row (or of the
// next group of basis columns) are issued before the current one is computed,
// so a warp keeps loads in flight while it spends its FP32 instructions.
#include "df64.cuh"
#include "epilogue.cuh"

namespace sstep {

constexpr int kMpRedCtas = 152 * 2;    // reductions with many accumulators: many rows per thread
constexpr int kMpCtas = 152 * 4;       // light kernels
constexpr int kRenorm = 8;             // rows between accumulator renormalisations
constexpr int kChunk = 8;              // basis columns loaded together in the projection

// ------------------------------------------------------------------ storage / arithmetic traits
template <int P>
struct Mode;

template <>
struct Mode<PREC_DF64> {
    using T = float2;
    using V = df64;
    static __device__ __forceinline__ V load(const T* p) {
        const float2 t = __ldg(p);
        return df64{t.x, t.y};
    }
    static __device__ __forceinline__ V load_rw(const T* p) {
        const float2 t = *p;
        return df64{t.x, t.y};
    }
    static __device__ __forceinline__ void store(T* p, V v) { *p = make_float2(v.hi, v.lo); }
    static __device__ __forceinline__ df64 wide(V v) { return v; }
    static __device__ __forceinline__ V narrow(df64 v) { return v; }
    static __device__ __forceinline__ V zero() { return df64{0.f, 0.f}; }
};

template <>
struct Mode<PREC_FP32> {
    using T = float;
    using V = float;
    static __device__ __forceinline__ V load(const T* p) { return __ldg(p); }
    static __device__ __forceinline__ V load_rw(const T* p) { return *p; }
    static __device__ __forceinline__ void store(T* p, V v) { *p = v; }
    static __device__ __forceinline__ df64 wide(V v) { return df64{v, 0.f}; }
    static __device__ __forceinline__ V narrow(df64 v) { return __fadd_rn(v.hi, v.lo); }
    static __device__ __forceinline__ V zero() { return 0.f; }
};

// exact-ish product a*b added into a double-float accumulator, for a of either mode
__device__ __forceinline__ void acc_add(DfAcc& acc, float a, df64 b) {
    const float p = __fmul_rn(a, b.hi);
    float e = __fmaf_rn(a, b.hi, -p);
    e = __fmaf_rn(a, b.lo, e);
    float s, t;
    two_sum(acc.hi, p, s, t);
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(t, e));
}
__device__ __forceinline__ void acc_add(DfAcc& acc, df64 a, df64 b) { acc.add_prod(a, b); }
__device__ __forceinline__ void acc_add(DfAcc& acc, float a, float b) { acc.add_prod(a, b); }

// Reduce NV double-float accumulators over the CTA in FP32 arithmetic (shuffles and
// double-float additions in a fixed order), leaving the NV sums as doubles in
// red[kWarps*NV .. kWarps*NV+NV) like block_reduce of the FP64 path.
template <int NV>
__device__ __forceinline__ void block_reduce_df(DfAcc (&acc)[NV], double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ float2 wsum[kWarps * NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        acc[v].normalize();
        df64 a{acc[v].hi, acc[v].lo};
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            df64 b{__shfl_down_sync(0xffffffffu, a.hi, off), __shfl_down_sync(0xffffffffu, a.lo, off)};
            a = df_add(a, b);
        }
        if (lane == 0) wsum[warp * NV + v] = make_float2(a.hi, a.lo);
    }
    __syncthreads();
    for (int v = threadIdx.x; v < NV; v += blockDim.x) {
        df64 t{0.f, 0.f};
        for (int w = 0; w < kWarps; ++w) t = df_add(t, df64{wsum[w * NV + v].x, wsum[w * NV + v].y});
        red[kWarps * NV + v] = df_to_double(t);
    }
    __syncthreads();
}

// Per-CTA df64 copies of launch-time FP64 scalars: computed by one thread (the FP64
// pipe is slow) and broadcast through shared memory.
__device__ __forceinline__ void broadcast_factors(double fy, double fw, const double* dscale, df64* out2) {
    if (threadIdx.x == 0) {
        if (dscale) {
            const double d = *dscale;
            fy *= d;
            fw *= d;
        }
        out2[0] = df_from_double(fy);
        out2[1] = df_from_double(fw);
    }
    __syncthreads();
}

// ================================================================== stencil sweep
template <int P>
__device__ __forceinline__ df64 mp_coef(const StencilDesc& A, int q, int64_t p) {
    if (A.variable) {
        const float2 t = __ldg(A.fdf[q] + p);
        return df64{t.x, t.y};
    }
    return df64{A.ch[q], P == PREC_DF64 ? A.cl[q] : 0.f};
}

template <int P>
__device__ __forceinline__ typename Mode<P>::V mp_row(const StencilDesc& A, const typename Mode<P>::T* v,
                                                      int64_t p) {
    using M = Mode<P>;
    const unsigned up = (unsigned)p;
    const unsigned t = up / (unsigned)A.nx;
    const int x = (int)(up - t * (unsigned)A.nx);
    const unsigned zz = t / (unsigned)A.ny;
    const int y = (int)(t - zz * (unsigned)A.ny), z = (int)zz;
    const int64_t pl = (int64_t)A.nx * A.ny;
    // gather the neighbours first (independent loads), then combine
    typename M::V nb[7];
    nb[0] = M::load(v + p);
    nb[1] = x > 0 ? M::load(v + p - 1) : M::zero();
    nb[2] = x < A.nx - 1 ? M::load(v + p + 1) : M::zero();
    nb[3] = y > 0 ? M::load(v + p - A.nx) : M::zero();
    nb[4] = y < A.ny - 1 ? M::load(v + p + A.nx) : M::zero();
    nb[5] = (A.dim == 3 && z > 0) ? M::load(v + p - pl) : M::zero();
    nb[6] = (A.dim == 3 && z < A.nz - 1) ? M::load(v + p + pl) : M::zero();
    if constexpr (P == PREC_DF64) {
        df64 acc = df_mul(mp_coef<P>(A, 0, p), nb[0]);
#pragma unroll
        for (int q = 1; q < 7; ++q)
            if (q < 2 * A.dim + 1) acc = df_fma(mp_coef<P>(A, q, p), nb[q], acc);
        return acc;
    } else {
        float acc = __fmul_rn(mp_coef<P>(A, 0, p).hi, nb[0]);
#pragma unroll
        for (int q = 1; q < 7; ++q)
            if (q < 2 * A.dim + 1) acc = __fmaf_rn(mp_coef<P>(A, q, p).hi, nb[q], acc);
        return acc;
    }
}

template <int P>
__global__ void __launch_bounds__(kThreads) mp_stencil_kernel(StencilDesc A, const typename Mode<P>::T* __restrict__ v,
                                                              double fy, typename Mode<P>::T* __restrict__ y, double fw,
                                                              typename Mode<P>::T* __restrict__ w,
                                                              const double* dscale, const SolverState* st, int gate) {
    using M = Mode<P>;
    __shared__ df64 fac[2];
    if (!gate_open(st, gate)) return;
    broadcast_factors(fy, fw, dscale, fac);
    const df64 vfy = fac[0], vfw = fac[1];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // two rows per iteration: their neighbour loads are all in flight together
    for (; p + stride < A.n; p += 2 * stride) {
        const auto r0 = mp_row<P>(A, v, p);
        const auto r1 = mp_row<P>(A, v, p + stride);
        if constexpr (P == PREC_DF64) {
            M::store(y + p, df_mul(vfy, r0));
            M::store(y + p + stride, df_mul(vfy, r1));
            if (w) {
                M::store(w + p, df_mul(vfw, M::load(v + p)));
                M::store(w + p + stride, df_mul(vfw, M::load(v + p + stride)));
            }
        } else {
            M::store(y + p, __fmul_rn(vfy.hi, r0));
            M::store(y + p + stride, __fmul_rn(vfy.hi, r1));
            if (w) {
                M::store(w + p, __fmul_rn(vfw.hi, M::load(v + p)));
                M::store(w + p + stride, __fmul_rn(vfw.hi, M::load(v + p + stride)));
            }
        }
    }
    if (p < A.n) {
        const auto r0 = mp_row<P>(A, v, p);
        if constexpr (P == PREC_DF64) {
            M::store(y + p, df_mul(vfy, r0));
            if (w) M::store(w + p, df_mul(vfw, M::load(v + p)));
        } else {
            M::store(y + p, __fmul_rn(vfy.hi, r0));
            if (w) M::store(w + p, __fmul_rn(vfw.hi, M::load(v + p)));
        }
    }
}

template <int P>
void mp_launch_stencil(const StencilDesc& A, const void* v, double fy, void* y, double fw, void* w,
                       const double* dscale, const SolverState* st, int gate, cudaStream_t stream) {
    using T = typename Mode<P>::T;
    int grid = grid_for(A.n, 152 * 8);
    mp_stencil_kernel<P><<<grid, kThreads, 0, stream>>>(A, (const T*)v, fy, (T*)y, fw, (T*)w, dscale, st, gate);
}

// ================================================================== residual (FP64) into the basis type
template <int P>
__global__ void __launch_bounds__(kThreads) mp_residual_kernel(StencilDesc A, const double* __restrict__ f,
                                                               const double* __restrict__ xv,
                                                               typename Mode<P>::T* __restrict__ out, Scratch sc,
                                                               Epi epi, int gate) {
    using M = Mode<P>;
    __shared__ double red[(kWarps + 1) * 1];
    if (!gate_open(epi.st, gate)) return;
    double acc[1] = {0.0};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < A.n; p += stride) {
        const unsigned up = (unsigned)p;
        const unsigned t = up / (unsigned)A.nx;
        const int x = (int)(up - t * (unsigned)A.nx);
        const unsigned zz = t / (unsigned)A.ny;
        const int yy = (int)(t - zz * (unsigned)A.ny);
        const double r = f[p] - stencil_row(A, xv, p, x, yy, (int)zz);
        if (out) {
            if constexpr (P == PREC_FP32) M::store(out + p, __double2float_rn(r));
            else M::store(out + p, df_from_double(r));
        }
        acc[0] = fma(r, r, acc[0]);
    }
    block_reduce<1>(acc, red);
    if (!publish_partial(red + kWarps, 1, sc.partials, sc.counter)) return;
    __shared__ double res[1];
    finish_reduction(res, 1, gridDim.x * gridDim.y, sc);
    run_epilogue(epi, res, 1, 1);
}

template <int P>
void mp_launch_residual(const StencilDesc& A, const double* f, const double* x, void* out, Scratch sc,
                        const Epi& epi, int gate, cudaStream_t stream) {
    using T = typename Mode<P>::T;
    int grid = grid_for(A.n, 152 * 4);
    mp_residual_kernel<P><<<grid, kThreads, 0, stream>>>(A, f, x, (T*)out, sc, epi, gate);
}

// ================================================================== Gram pass, double-float accumulation
// C[by*KA + i, j] = sum_rows V[row, by*KA + i] Y[row, j]; the next row's operands are
// loaded before the current row is accumulated.
template <int P, int KA, int KB>
__global__ void __launch_bounds__(kThreads) mp_gram_kernel(int64_t n, const typename Mode<P>::T* __restrict__ V,
                                                           int64_t ldv, int ka, const typename Mode<P>::T* __restrict__ Y,
                                                           int64_t ldy, Scratch sc, Epi epi, int gate) {
    using M = Mode<P>;
    using Vt = typename M::V;
    constexpr int NV = KA * KB;
    __shared__ double red[(kWarps + 1) * NV];
    __shared__ double res[kMaxCols * (kMaxS + 1)];
    if (!gate_open(epi.st, gate)) return;
    const int a0 = blockIdx.y * KA;
    const int na = min(KA, ka - a0);
    int64_t voff[KA];
#pragma unroll
    for (int i = 0; i < KA; ++i) voff[i] = (int64_t)min(a0 + i, ka - 1) * ldv;
    DfAcc acc[NV];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    Vt ya[KB], va[KA];
    auto load_row = [&](int64_t q, Vt (&yy)[KB], Vt (&vv)[KA]) {
#pragma unroll
        for (int j = 0; j < KB; ++j) yy[j] = M::load(Y + q + j * ldy);
#pragma unroll
        for (int i = 0; i < KA; ++i) vv[i] = M::load(V + q + voff[i]);
    };
    if (p < n) load_row(p, ya, va);
    int cnt = 0;
    while (p < n) {
        const int64_t pn = p + stride;
        Vt yb[KB], vb[KA];
        if (pn < n) load_row(pn, yb, vb);
#pragma unroll
        for (int i = 0; i < KA; ++i)
            if (i < na) {
#pragma unroll
                for (int j = 0; j < KB; ++j) acc_add(acc[i * KB + j], va[i], M::wide(ya[j]));
            }
        if (++cnt == kRenorm) {
            cnt = 0;
#pragma unroll
            for (int v = 0; v < NV; ++v) acc[v].normalize();
        }
#pragma unroll
        for (int j = 0; j < KB; ++j) ya[j] = yb[j];
#pragma unroll
        for (int i = 0; i < KA; ++i) va[i] = vb[i];
        p = pn;
    }
    block_reduce_df<NV>(acc, red);
    if (!publish_partial(red + kWarps * NV, NV, sc.partials, sc.counter)) return;
    const int gx = gridDim.x;
    for (int t = threadIdx.x; t < ka * KB; t += blockDim.x) {
        const int i = t % ka, j = t / ka, by = i / KA, ii = i % KA;
        double s = 0.0;
        for (int bx = 0; bx < gx; ++bx) s += ld_cg(sc.partials + (int64_t)(by * gx + bx) * NV + ii * KB + j);
        res[t] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) *sc.counter = 0u;
    run_epilogue(epi, res, ka, KB);
}

template <int P>
void mp_launch_gram(int64_t n, const void* V, int64_t ldv, int ka, const void* Y, int64_t ldy, int kb,
                    Scratch sc, const Epi& epi, int gate, cudaStream_t stream) {
    using T = typename Mode<P>::T;
    const int KAc = kb <= 4 ? 8 : 4;   // V columns per CTA, keeping the accumulators in registers
    const int gy = (ka + KAc - 1) / KAc;
    int gx = grid_for(n, kMpRedCtas * 2 / gy > 0 ? kMpRedCtas * 2 / gy : 1);
    dim3 grid(gx, gy);
    const T* Vp = (const T*)V;
    const T* Yp = (const T*)Y;
    switch (kb) {
#define SSTEP_MPG(KB, KA) \
    case KB: mp_gram_kernel<P, KA, KB><<<grid, kThreads, 0, stream>>>(n, Vp, ldv, ka, Yp, ldy, sc, epi, gate); break;
        SSTEP_MPG(1, 8)
        SSTEP_MPG(2, 8)
        SSTEP_MPG(3, 8)
        SSTEP_MPG(4, 8)
        SSTEP_MPG(5, 4)
        SSTEP_MPG(6, 4)
        SSTEP_MPG(7, 4)
        SSTEP_MPG(8, 4)
        SSTEP_MPG(9, 4)
#undef SSTEP_MPG
        default: break;
    }
}

// ================================================================== projection Y - V T (+ optional Gram)
// Yout[:, j] = Yin[:, j] + V (sgn T)[:, j] for j >= j0, summed in double-float and
// rounded once to the storage type. The basis columns are read in groups of kChunk,
// the next group's loads issued before the current group is accumulated. With GRAM
// (used for narrow outputs) the kb x kb Gram of Yout is reduced in the same pass.
template <int P, int KB, bool GRAM>
__global__ void __launch_bounds__(kThreads) mp_update_kernel(int64_t n, const typename Mode<P>::T* __restrict__ V,
                                                             int64_t ldv, int ka, const typename Mode<P>::T* Yin,
                                                             int64_t ldy, typename Mode<P>::T* Yout, int64_t ldo,
                                                             int j0, const double* __restrict__ T, int ldt,
                                                             double sgn, Scratch sc, Epi epi, int gate) {
    using M = Mode<P>;
    using Vt = typename M::V;
    constexpr int NV = GRAM ? KB * (KB + 1) / 2 : 1;
    __shared__ df64 Ts[kMaxCols * KB];
    __shared__ double red[(kWarps + 1) * NV];
    __shared__ double res[(kMaxS + 1) * (kMaxS + 1)];
    if (!gate_open(epi.st, gate)) return;
    // FP64 coefficients to float pairs: spread over the CTA (one conversion per entry)
    for (int t = threadIdx.x; t < ka * KB; t += blockDim.x) {
        const int i = t % ka, j = t / ka;
        Ts[i * KB + j] = df_from_double(sgn * T[i + (int64_t)j * ldt]);
    }
    __syncthreads();
    DfAcc gacc[NV];
    const bool inplace = (Yin == Yout) && (ldy == ldo);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int nch = (ka + kChunk - 1) / kChunk;
    int cnt = 0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
        Vt cur[kChunk];
        if (ka > 0) {
#pragma unroll
            for (int c = 0; c < kChunk; ++c) cur[c] = c < ka ? M::load(V + p + (int64_t)c * ldv) : M::zero();
        }
        Vt yv[KB];
#pragma unroll
        for (int j = 0; j < KB; ++j) yv[j] = M::load_rw(Yin + p + j * ldy);
        if (ka > 0) {
            DfAcc sum[KB];
            for (int ch = 0; ch < nch; ++ch) {
                const int base = ch * kChunk;
                Vt nxt[kChunk];
                const int nb = base + kChunk;
#pragma unroll
                for (int c = 0; c < kChunk; ++c) nxt[c] = (nb + c < ka) ? M::load(V + p + (int64_t)(nb + c) * ldv) : M::zero();
#pragma unroll
                for (int c = 0; c < kChunk; ++c) {
                    if (base + c < ka) {
#pragma unroll
                        for (int j = 0; j < KB; ++j)
                            if (j >= j0) acc_add(sum[j], cur[c], Ts[(base + c) * KB + j]);
                    }
                }
#pragma unroll
                for (int c = 0; c < kChunk; ++c) cur[c] = nxt[c];
#pragma unroll
                for (int j = 0; j < KB; ++j) sum[j].normalize();
            }
#pragma unroll
            for (int j = 0; j < KB; ++j)
                if (j >= j0) yv[j] = M::narrow(df_add(M::wide(yv[j]), df64{sum[j].hi, sum[j].lo}));
        }
#pragma unroll
        for (int j = 0; j < KB; ++j)
            if (!inplace || (j >= j0 && ka > 0)) M::store(Yout + p + j * ldo, yv[j]);
        if (GRAM) {
            int idx = 0;
#pragma unroll
            for (int q = 0; q < KB; ++q)
#pragma unroll
                for (int pp = 0; pp <= q; ++pp) {
                    acc_add(gacc[idx], yv[pp], M::wide(yv[q]));
                    ++idx;
                }
            if (++cnt == kRenorm) {
                cnt = 0;
#pragma unroll
                for (int v = 0; v < NV; ++v) gacc[v].normalize();
            }
        }
    }
    if (!GRAM) return;
    block_reduce_df<NV>(gacc, red);
    if (!publish_partial(red + kWarps * NV, NV, sc.partials, sc.counter)) return;
    __shared__ double packed[NV];
    finish_reduction(packed, NV, gridDim.x * gridDim.y, sc);
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
    run_epilogue(epi, res, KB, KB);
}

// ================================================================== Gram of one block (symmetric)
// G = Y^T Y for kb columns, upper triangle accumulated in double-float; the next
// row is loaded before the current one is accumulated.
template <int P, int KB>
__global__ void __launch_bounds__(kThreads) mp_symgram_kernel(int64_t n, const typename Mode<P>::T* __restrict__ Y,
                                                              int64_t ldy, Scratch sc, Epi epi, int gate) {
    using M = Mode<P>;
    using Vt = typename M::V;
    constexpr int NV = KB * (KB + 1) / 2;
    __shared__ double red[(kWarps + 1) * NV];
    __shared__ double res[(kMaxS + 1) * (kMaxS + 1)];
    if (!gate_open(epi.st, gate)) return;
    DfAcc acc[NV];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    Vt ya[KB];
    if (p < n) {
#pragma unroll
        for (int j = 0; j < KB; ++j) ya[j] = M::load(Y + p + j * ldy);
    }
    int cnt = 0;
    while (p < n) {
        const int64_t pn = p + stride;
        Vt yb[KB];
        if (pn < n) {
#pragma unroll
            for (int j = 0; j < KB; ++j) yb[j] = M::load(Y + pn + j * ldy);
        }
        int idx = 0;
#pragma unroll
        for (int q = 0; q < KB; ++q)
#pragma unroll
            for (int pp = 0; pp <= q; ++pp) {
                acc_add(acc[idx], ya[pp], M::wide(ya[q]));
                ++idx;
            }
        if (++cnt == kRenorm) {
            cnt = 0;
#pragma unroll
            for (int v = 0; v < NV; ++v) acc[v].normalize();
        }
#pragma unroll
        for (int j = 0; j < KB; ++j) ya[j] = yb[j];
        p = pn;
    }
    block_reduce_df<NV>(acc, red);
    if (!publish_partial(red + kWarps * NV, NV, sc.partials, sc.counter)) return;
    __shared__ double packed[NV];
    finish_reduction(packed, NV, gridDim.x * gridDim.y, sc);
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
    run_epilogue(epi, res, KB, KB);
}

template <int P>
void mp_launch_update(int64_t n, const void* V, int64_t ldv, int ka, const void* Yin, int64_t ldy, void* Yout,
                      int64_t ldo, int kb, int j0, const double* T, int ldt, double sgn, bool gram, Scratch sc,
                      const Epi& epi, int gate, cudaStream_t stream) {
    using Tt = typename Mode<P>::T;
    const Tt* Vp = (const Tt*)V;
    const Tt* Yi = (const Tt*)Yin;
    Tt* Yo = (Tt*)Yout;
    if (gram && kb > 2) {
        // wide blocks: the projection alone (light, many CTAs), then the block's Gram
        Epi none = epi;
        none.mode = EPI_NONE;
        mp_launch_update<P>(n, V, ldv, ka, Yin, ldy, Yout, ldo, kb, j0, T, ldt, sgn, false, sc, none, gate, stream);
        int grid = grid_for(n, kMpRedCtas);
        switch (kb) {
#define SSTEP_MPS(KB) \
    case KB: mp_symgram_kernel<P, KB><<<grid, kThreads, 0, stream>>>(n, Yo, ldo, sc, epi, gate); break;
            SSTEP_MPS(3)
            SSTEP_MPS(4)
            SSTEP_MPS(5)
            SSTEP_MPS(6)
            SSTEP_MPS(7)
            SSTEP_MPS(8)
            SSTEP_MPS(9)
#undef SSTEP_MPS
            default: break;
        }
        return;
    }
    int grid = grid_for(n, gram ? kMpRedCtas * 2 : kMpCtas);
    switch (kb) {
#define SSTEP_MPU(KB)                                                                                         \
    case KB:                                                                                                  \
        if (gram)                                                                                             \
            mp_update_kernel<P, KB, true><<<grid, kThreads, 0, stream>>>(n, Vp, ldv, ka, Yi, ldy, Yo, ldo, j0, \
                                                                         T, ldt, sgn, sc, epi, gate);        \
        else                                                                                                  \
            mp_update_kernel<P, KB, false><<<grid, kThreads, 0, stream>>>(n, Vp, ldv, ka, Yi, ldy, Yo, ldo,    \
                                                                          j0, T, ldt, sgn, sc, epi, gate);   \
        break;
        SSTEP_MPU(1)
        SSTEP_MPU(2)
        SSTEP_MPU(3)
        SSTEP_MPU(4)
        SSTEP_MPU(5)
        SSTEP_MPU(6)
        SSTEP_MPU(7)
        SSTEP_MPU(8)
        SSTEP_MPU(9)
#undef SSTEP_MPU
        default: break;
    }
}

// ================================================================== x += V y (FP64 iterate)
template <int P>
__global__ void __launch_bounds__(kThreads) mp_axpy_kernel(int64_t n, const typename Mode<P>::T* __restrict__ V,
                                                           int64_t ldv, double* __restrict__ x, Epi epi, int gate) {
    using M = Mode<P>;
    using Vt = typename M::V;
    __shared__ df64 ys[kMaxCols];
    if (!gate_open(epi.st, gate)) return;
    const int K = epi.st->K;
    for (int i = threadIdx.x; i < K; i += blockDim.x) ys[i] = df_from_double(epi.st->y[i]);
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int nch = (K + kChunk - 1) / kChunk;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
        Vt cur[kChunk];
#pragma unroll
        for (int c = 0; c < kChunk; ++c) cur[c] = c < K ? M::load(V + p + (int64_t)c * ldv) : M::zero();
        const double xold = x[p];
        DfAcc acc;
        for (int ch = 0; ch < nch; ++ch) {
            const int base = ch * kChunk, nb = base + kChunk;
            Vt nxt[kChunk];
#pragma unroll
            for (int c = 0; c < kChunk; ++c) nxt[c] = (nb + c < K) ? M::load(V + p + (int64_t)(nb + c) * ldv) : M::zero();
#pragma unroll
            for (int c = 0; c < kChunk; ++c)
                if (base + c < K) acc_add(acc, cur[c], ys[base + c]);
#pragma unroll
            for (int c = 0; c < kChunk; ++c) cur[c] = nxt[c];
        }
        x[p] = xold + acc.value();
    }
}

template <int P>
void mp_launch_axpy(int64_t n, const void* V, int64_t ldv, double* x, const Epi& epi, int gate,
                    cudaStream_t stream) {
    using T = typename Mode<P>::T;
    int grid = grid_for(n, kMpCtas * 2);
    mp_axpy_kernel<P><<<grid, kThreads, 0, stream>>>(n, (const T*)V, ldv, x, epi, gate);
}

// ================================================================== variable coefficients as float pairs
__global__ void split_fields_kernel(const double* __restrict__ src, float2* __restrict__ dst, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
        const df64 d = df_from_double(src[p]);
        dst[p] = make_float2(d.hi, d.lo);
    }
}

void launch_split_fields(const double* src, float2* dst, int64_t n, cudaStream_t stream) {
    split_fields_kernel<<<grid_for(n, 152 * 8), kThreads, 0, stream>>>(src, dst, n);
}

// ------------------------------------------------------------------ instantiations
#define SSTEP_MP_INST(P)                                                                                          \
    template void mp_launch_stencil<P>(const StencilDesc&, const void*, double, void*, double, void*,            \
                                       const double*, const SolverState*, int, cudaStream_t);                    \
    template void mp_launch_residual<P>(const StencilDesc&, const double*, const double*, void*, Scratch,        \
                                        const Epi&, int, cudaStream_t);                                          \
    template void mp_launch_gram<P>(int64_t, const void*, int64_t, int, const void*, int64_t, int, Scratch,      \
                                    const Epi&, int, cudaStream_t);                                              \
    template void mp_launch_update<P>(int64_t, const void*, int64_t, int, const void*, int64_t, void*, int64_t,  \
                                      int, int, const double*, int, double, bool, Scratch, const Epi&, int,      \
                                      cudaStream_t);                                                             \
    template void mp_launch_axpy<P>(int64_t, const void*, int64_t, double*, const Epi&, int, cudaStream_t);
SSTEP_MP_INST(PREC_DF64)
SSTEP_MP_INST(PREC_FP32)
#undef SSTEP_MP_INST

}  // namespace sstep
