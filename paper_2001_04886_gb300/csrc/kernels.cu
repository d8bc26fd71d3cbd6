// Streaming kernels of the FP64 path: stencil sweep, residual, tall-skinny Gram,
// block update, Orthomin updates, and the small FP64 work of Scalar1 / Scalar2 /
// the Hessenberg least squares, which runs in the last CTA of each reduction.
#include <math.h>

#include <algorithm>

#include "epilogue.cuh"

namespace sstep {

// 8 CTAs of 256 threads per SM at most, on the current device
static int max_ctas() { return 8 * device_sms(); }
constexpr int kGramKA = 8;             // V columns per Gram CTA (grid.y splits ka)
constexpr int kMaxNV = kGramKA * (kMaxS + 1);   // largest per-CTA partial vector

int fp64_gram_partials_doubles() { return max_ctas() * kMaxNV; }
int max_partials_doubles() { return std::max(std::max(max_ctas() * kMaxNV, oz_partials_doubles()), kOzAccWords); }

// ================================================================== stencil sweep
__device__ __forceinline__ void grid_xyz(const StencilDesc& A, int64_t p, int& x, int& y, int& z) {
    const unsigned up = (unsigned)p;
    const unsigned t = up / (unsigned)A.nx;
    x = (int)(up - t * (unsigned)A.nx);
    const unsigned zz = t / (unsigned)A.ny;
    y = (int)(t - zz * (unsigned)A.ny);
    z = (int)zz;
}

// high word of |v|: its maximum over a column is the column bound of the tensor-core Gram pass
__device__ __forceinline__ unsigned abs_hi(double v) {
    return (unsigned)((unsigned long long)__double_as_longlong(v) >> 32) & 0x7FFFFFFFu;
}

// warp maximum of the bounds, one atomicMax per warp and column (every lane of the warp
// must reach this call)
__device__ __forceinline__ void publish_bounds(unsigned ym, unsigned* ybnd, unsigned wm, unsigned* wbnd,
                                               unsigned* ybnd2 = nullptr, unsigned* wbnd2 = nullptr) {
    if (ybnd || ybnd2) {
        ym = __reduce_max_sync(0xffffffffu, ym);
        if ((threadIdx.x & 31) == 0 && ym) {
            if (ybnd) atomicMax(ybnd, ym);
            if (ybnd2) atomicMax(ybnd2, ym);
        }
    }
    if (wbnd || wbnd2) {
        wm = __reduce_max_sync(0xffffffffu, wm);
        if ((threadIdx.x & 31) == 0 && wm) {
            if (wbnd) atomicMax(wbnd, wm);
            if (wbnd2) atomicMax(wbnd2, wm);
        }
    }
}

// A CTA owns a (32 x 8)-point x-y tile and a chunk of z planes and marches through z,
// keeping planes z-1, z, z+1 of each (x, y) column in registers: a point costs one new
// load plus the four in-plane neighbours (L1 hits), with no per-point division. With
// constant coefficients the factor fy is folded into the 2d+1 coefficients once per
// thread, so a point costs 2d+1 FP64 operations instead of 2d+2.
__global__ void __launch_bounds__(kThreads) stencil_kernel(StencilDesc A, const double* __restrict__ v,
                                                           double fy, double* __restrict__ y, double fw,
                                                           double* __restrict__ w, const double* dscale,
                                                           const SolverState* st, int gate, int zchunk,
                                                           double shift, const double* __restrict__ u,
                                                           unsigned* ybnd, unsigned* wbnd, unsigned* ybnd2,
                                                           unsigned* wbnd2) {
    if (!gate_open(st, gate)) return;
    if (dscale) {
        const double d = *dscale;
        fy *= d;
        fw *= d;
    }
    const int tx = (A.nx + 31) / 32;
    const int x = (int)(blockIdx.x % tx) * 32 + threadIdx.x;
    const int yy = (int)(blockIdx.x / tx) * 8 + threadIdx.y;
    const int zb = blockIdx.y * zchunk, ze = min(A.nz, zb + zchunk);
    unsigned ym = 0, wm = 0;   // column bounds of this thread's outputs
    if (x < A.nx && yy < A.ny && zb < ze) {
    const bool three = A.dim == 3;
    const int64_t pl = (int64_t)A.nx * A.ny;
    int64_t p = (int64_t)zb * pl + (int64_t)yy * A.nx + x;
    double c[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) c[q] = fy * A.c[q];
    if (!u) c[0] = fy * (A.c[0] - shift);
    const double fs = -fy * shift;   // with u: the shift term -fy shift u_p
    double vm = (three && zb > 0) ? __ldg(v + p - pl) : 0.0;
    double vc = __ldg(v + p);
#pragma unroll 2
    for (int z = zb; z < ze; ++z, p += pl) {
        const double vp = (three && z + 1 < A.nz) ? __ldg(v + p + pl) : 0.0;
        double acc;
        if (!A.variable) {
            acc = c[0] * vc;
            if (x > 0) acc = fma(c[1], __ldg(v + p - 1), acc);
            if (x < A.nx - 1) acc = fma(c[2], __ldg(v + p + 1), acc);
            if (yy > 0) acc = fma(c[3], __ldg(v + p - A.nx), acc);
            if (yy < A.ny - 1) acc = fma(c[4], __ldg(v + p + A.nx), acc);
            if (three) {
                if (z > 0) acc = fma(c[5], vm, acc);
                if (z < A.nz - 1) acc = fma(c[6], vp, acc);
            }
        } else {
            acc = (__ldg(A.f[0] + p) - (u ? 0.0 : shift)) * vc;
            if (x > 0) acc = fma(__ldg(A.f[1] + p), __ldg(v + p - 1), acc);
            if (x < A.nx - 1) acc = fma(__ldg(A.f[2] + p), __ldg(v + p + 1), acc);
            if (yy > 0) acc = fma(__ldg(A.f[3] + p), __ldg(v + p - A.nx), acc);
            if (yy < A.ny - 1) acc = fma(__ldg(A.f[4] + p), __ldg(v + p + A.nx), acc);
            if (three) {
                if (z > 0) acc = fma(__ldg(A.f[5] + p), vm, acc);
                if (z < A.nz - 1) acc = fma(__ldg(A.f[6] + p), vp, acc);
            }
            acc *= fy;
        }
        if (u) acc = fma(fs, __ldg(u + p), acc);
        y[p] = acc;
        ym = max(ym, abs_hi(acc));
        if (w) {
            const double wv = fw * vc;
            w[p] = wv;
            wm = max(wm, abs_hi(wv));
        }
        vm = vc;
        vc = vp;
    }
    }
    publish_bounds(ym, ybnd, wm, wbnd, ybnd2, wbnd2);
}

// The common case of the powers: constant coefficients and no separate shift vector.
// With the factor known on the host the scaled coefficients fy c (fy (c_0 - shift) on
// the diagonal) come in from the host; with a device factor d (DSCALE: the first power
// of a block, d = 1/||u||) eight threads of each CTA form (fy d) c and fw d once in
// shared memory. Either way a point costs its 7 (5 in 2-D) FP64 multiply-adds (and one
// multiply where the scaled v is stored as well), the same operations as stencil_kernel.
struct ConstCoef {
    double c[7];       // !DSCALE: fy c (diagonal fy (c_0 - shift)); DSCALE: the raw c
    double fy, shift;  // DSCALE only
};

template <bool THREE, bool WCOPY, bool DSCALE>
__global__ void __launch_bounds__(kThreads) stencil_const_kernel(int nx, int ny, int nz, ConstCoef k,
                                                                 const double* __restrict__ v,
                                                                 double* __restrict__ y, double fw,
                                                                 double* __restrict__ w, const double* dscale,
                                                                 const SolverState* st, int gate, int zchunk,
                                                                 unsigned* ybnd, unsigned* wbnd, unsigned* ybnd2,
                                                                 unsigned* wbnd2) {
    if (!gate_open(st, gate)) return;
    __shared__ double sk[8];
    if (DSCALE) {
        const int t = threadIdx.y * 32 + threadIdx.x;
        if (t < 8) {
            const double d = *dscale, fyd = k.fy * d;
            double ct = k.c[0] - k.shift;   // t == 0; the others select their raw c without indexing
#pragma unroll
            for (int q = 1; q < 7; ++q)
                if (t == q) ct = k.c[q];
            sk[t] = t < 7 ? fyd * ct : fw * d;
        }
        __syncthreads();
    }
    const double c0 = DSCALE ? sk[0] : k.c[0], c1 = DSCALE ? sk[1] : k.c[1], c2 = DSCALE ? sk[2] : k.c[2];
    const double c3 = DSCALE ? sk[3] : k.c[3], c4 = DSCALE ? sk[4] : k.c[4], c5 = DSCALE ? sk[5] : k.c[5];
    const double c6 = DSCALE ? sk[6] : k.c[6], fwd = DSCALE ? sk[7] : fw;
    const int tx = (nx + 31) / 32;
    const int x = (int)(blockIdx.x % tx) * 32 + threadIdx.x;
    const int yy = (int)(blockIdx.x / tx) * 8 + threadIdx.y;
    const int zb = blockIdx.y * zchunk, ze = min(nz, zb + zchunk);
    unsigned ym = 0, wm = 0;   // column bounds of this thread's outputs
    if (x < nx && yy < ny && zb < ze) {
    const int64_t pl = (int64_t)nx * ny;
    int64_t p = (int64_t)zb * pl + (int64_t)yy * nx + x;
    const bool xl = x > 0, xr = x < nx - 1, yl = yy > 0, yr = yy < ny - 1;
    double vm = (THREE && zb > 0) ? __ldg(v + p - pl) : 0.0;
    double vc = __ldg(v + p);
#pragma unroll 2
    for (int z = zb; z < ze; ++z, p += pl) {
        const double vp = (THREE && z + 1 < nz) ? __ldg(v + p + pl) : 0.0;
        double acc = c0 * vc;
        if (xl) acc = fma(c1, __ldg(v + p - 1), acc);
        if (xr) acc = fma(c2, __ldg(v + p + 1), acc);
        if (yl) acc = fma(c3, __ldg(v + p - nx), acc);
        if (yr) acc = fma(c4, __ldg(v + p + nx), acc);
        if (THREE) {
            if (z > 0) acc = fma(c5, vm, acc);
            if (z < nz - 1) acc = fma(c6, vp, acc);
        }
        y[p] = acc;
        ym = max(ym, abs_hi(acc));
        if (WCOPY) {
            const double wv = fwd * vc;
            w[p] = wv;
            wm = max(wm, abs_hi(wv));
        }
        vm = vc;
        vc = vp;
    }
    }
    publish_bounds(ym, ybnd, wm, wbnd, ybnd2, wbnd2);
}

template <bool THREE, bool WCOPY, bool DSCALE>
void launch_const(const StencilDesc& A, const ConstCoef& k, const double* v, double* y, double fw, double* w,
                  const double* dscale, const SolverState* st, int gate, int zchunk, dim3 grid, dim3 block,
                  cudaStream_t stream, unsigned* ybnd, unsigned* wbnd, unsigned* ybnd2, unsigned* wbnd2) {
    stencil_const_kernel<THREE, WCOPY, DSCALE><<<grid, block, 0, stream>>>(A.nx, A.ny, A.nz, k, v, y, fw, w, dscale,
                                                                           st, gate, zchunk, ybnd, wbnd, ybnd2, wbnd2);
}

void launch_stencil(const StencilDesc& A, const double* v, double fy, double* y, double fw, double* w,
                    const double* dscale, const SolverState* st, int gate, cudaStream_t stream, double shift,
                    const double* u, unsigned* ybnd, unsigned* wbnd, unsigned* ybnd2, unsigned* wbnd2) {
    const int tiles = ((A.nx + 31) / 32) * ((A.ny + 7) / 8);
    // z chunks: about one wave of 8 CTAs per SM, at least one plane per chunk
    int chunks = max_ctas() / tiles;
    chunks = chunks < 1 ? 1 : (chunks > A.nz ? A.nz : chunks);
    const int zchunk = (A.nz + chunks - 1) / chunks;
    chunks = (A.nz + zchunk - 1) / zchunk;
    const dim3 grid(tiles, chunks), block(32, 8);
    if (!A.variable && !u) {
        ConstCoef k;
        k.fy = fy;
        k.shift = shift;
        for (int q = 0; q < 7; ++q) k.c[q] = dscale ? A.c[q] : fy * A.c[q];
        if (!dscale) k.c[0] = fy * (A.c[0] - shift);
        const bool three = A.dim == 3, wc = w != nullptr, ds = dscale != nullptr;
#define SSTEP_CONST(T3, WC, DS) \
    if (three == T3 && wc == WC && ds == DS) return launch_const<T3, WC, DS>(A, k, v, y, fw, w, dscale, st, gate, zchunk, grid, block, stream, ybnd, wbnd, ybnd2, wbnd2);
        SSTEP_CONST(true, false, false)
        SSTEP_CONST(true, true, true)
        SSTEP_CONST(true, true, false)
        SSTEP_CONST(true, false, true)
        SSTEP_CONST(false, false, false)
        SSTEP_CONST(false, true, true)
        SSTEP_CONST(false, true, false)
        SSTEP_CONST(false, false, true)
#undef SSTEP_CONST
    }
    stencil_kernel<<<grid, block, 0, stream>>>(A, v, fy, y, fw, w, dscale, st, gate, zchunk, shift, u, ybnd, wbnd,
                                               ybnd2, wbnd2);
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
    int grid = grid_for(A.n, max_ctas() / 2);
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
    int gx = grid_for(n, max_ctas() / gy > 0 ? max_ctas() / gy : 1);
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
                                                          int ldt, double sgn, Scratch sc, Epi epi, int gate,
                                                          unsigned* bnd, int bnd_hi) {
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
    unsigned bm[KB];   // column bounds of the outputs j0 <= j < bnd_hi
#pragma unroll
    for (int j = 0; j < KB; ++j) bm[j] = 0;
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
            bm[j] = max(bm[j], abs_hi(yv[j]));
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
    if (bnd) {
#pragma unroll
        for (int j = 0; j < KB; ++j)
            if (j >= j0 && j < bnd_hi) publish_bounds(bm[j], bnd + (j - j0), 0u, nullptr);
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
                   bool gram, Scratch sc, const Epi& epi, int gate, cudaStream_t stream, unsigned* bnd,
                   int bnd_hi) {
    int grid = grid_for(n, max_ctas() / 2);
    switch (kb) {
#define SSTEP_UPD_CASE(KB)                                                                                \
    case KB:                                                                                              \
        if (gram)                                                                                         \
            update_kernel<KB, true><<<grid, kThreads, 0, stream>>>(n, V, ldv, ka, Yin, ldy, Yout, ldo, j0, \
                                                                   T, ldt, sgn, sc, epi, gate, bnd,      \
                                                                   bnd_hi);                              \
        else                                                                                              \
            update_kernel<KB, false><<<grid, kThreads, 0, stream>>>(n, V, ldv, ka, Yin, ldy, Yout, ldo,    \
                                                                    j0, T, ldt, sgn, sc, epi, gate, bnd, \
                                                                    bnd_hi);                             \
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
    int grid = grid_for(n, max_ctas() / 2);
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
// R_j = sigma AR_{j-1}; with epi.ortho, R and AR first go through the upper triangular
// factor F stored below the B blocks (A^T A-orthonormal blocks). Reduces
// W = AP_new^T AP_new (packed) and m = AP_new^T r.
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
    const int nwin = epi.nwin, rows = (nwin + epi.ortho) * S;
    for (int t = threadIdx.x; t < rows * S; t += blockDim.x) {
        const int i = t % rows, j = t / rows;
        Bs[i * S + j] = epi.st->T[i + j * kMaxCols];
    }
    __syncthreads();
    const double* Fs = Bs + nwin * S * S;   // ortho: upper triangular factor of the R block
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
            pv[j] = (j == 0) ? rv : sigma * apv[j - 1];
        }
        if (epi.ortho) {   // [R, A R] F, F upper triangular: column j from columns q <= j
#pragma unroll
            for (int j = S - 1; j >= 0; --j) {
                double tp = 0.0, tap = 0.0;
#pragma unroll
                for (int q = 0; q <= j; ++q) {
                    tp = fma(pv[q], Fs[q * S + j], tp);
                    tap = fma(apv[q], Fs[q * S + j], tap);
                }
                pv[j] = tp;
                apv[j] = tap;
            }
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
    int grid = grid_for(n, max_ctas() / 2);
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

// ================================================================== variable-coefficient operator fields
__global__ void convdiff_fields_kernel(const double* __restrict__ beta, double h, int64_t n, double* __restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
        const double c = beta[p] * h / 2.0;
        out[p] = 4.0;
        out[n + p] = -1.0 - c;
        out[2 * n + p] = -1.0 + c;
        out[3 * n + p] = -1.0 - c;
        out[4 * n + p] = -1.0 + c;
    }
}

void launch_convdiff_fields(const double* beta, double h, int64_t n, double* out, cudaStream_t stream) {
    convdiff_fields_kernel<<<grid_for(n, max_ctas()), kThreads, 0, stream>>>(beta, h, n, out);
}

// ================================================================== least squares solve
// y = R^{-1} g by back substitution: R and g are staged in shared memory and each
// row's dot product is a warp reduction (fixed order), so the dependent chain is K
// short steps instead of K^2/2 global-memory round trips.
__global__ void lsq_solve_kernel(SolverState* st, int gate) {
    __shared__ double sR[(kMaxM + 1) * kMaxM];
    __shared__ double sg[kMaxM];
    if (!gate_open(st, gate)) return;
    const int K = st->K, ld = st->m + 1, lane = threadIdx.x;
    for (int t = lane; t < K * K; t += blockDim.x) sR[(t % K) + (t / K) * K] = st->R[(t % K) + (t / K) * ld];
    for (int t = lane; t < K; t += blockDim.x) sg[t] = st->g[t];
    __syncwarp();
    // column by column from the last: y_q by the lane that owns row q (rows lane and
    // lane + 32), then every lane folds R[i, q] y_q into the sums of its rows i < q. The
    // reciprocals of the diagonal are formed first, all at once, so no division sits on
    // the dependent chain of K steps (each product differs from the quotient by at most an ulp).
    static_assert(kMaxM <= 64, "two rows per lane");
    const int i0 = lane, i1 = lane + 32;
    const double r0 = i0 < K ? 1.0 / sR[i0 + i0 * K] : 0.0, r1 = i1 < K ? 1.0 / sR[i1 + i1 * K] : 0.0;
    double t0 = 0.0, t1 = 0.0, y0 = 0.0, y1 = 0.0;
    for (int q = K - 1; q >= 0; --q) {
        if (q == i0) y0 = mul(sub(sg[q], t0), r0);
        if (q == i1) y1 = mul(sub(sg[q], t1), r1);
        const double yq = __shfl_sync(0xffffffffu, q < 32 ? y0 : y1, q & 31);
        if (i0 < q) t0 = fma(sR[i0 + q * K], yq, t0);
        if (i1 < q) t1 = fma(sR[i1 + q * K], yq, t1);
    }
    if (i0 < K) st->y[i0] = y0;
    if (i1 < K) st->y[i1] = y1;
}

void launch_lsq_solve(SolverState* st, int gate, cudaStream_t stream) {
    lsq_solve_kernel<<<1, 32, 0, stream>>>(st, gate);
}

}  // namespace sstep
