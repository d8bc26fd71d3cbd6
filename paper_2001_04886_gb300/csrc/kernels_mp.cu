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
#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include "df64.cuh"
#include "epilogue.cuh"

namespace sstep {

// grid caps per multiprocessor of the current device
static int mp_red_ctas() { return 2 * device_sms(); }   // reductions with many accumulators: many rows per thread
static int mp_ctas() { return 4 * device_sms(); }       // light kernels
constexpr int kRenorm = 8;             // rows between accumulator renormalisations
static int max_ctas_mp() { return 8 * device_sms(); }   // grid bound of the reductions (the partials buffer size)
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
    // rows 2q and 2q+1 with one 16-byte access (columns are 256-byte aligned, ld even)
    static __device__ __forceinline__ void load2(const T* p, V& a, V& b) {
        const float4 t = __ldg((const float4*)p);
        a = df64{t.x, t.y};
        b = df64{t.z, t.w};
    }
    static __device__ __forceinline__ void load2_rw(const T* p, V& a, V& b) {
        const float4 t = *(const float4*)p;
        a = df64{t.x, t.y};
        b = df64{t.z, t.w};
    }
    static __device__ __forceinline__ void store2(T* p, V a, V b) { *(float4*)p = make_float4(a.hi, a.lo, b.hi, b.lo); }
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
    static __device__ __forceinline__ void load2(const T* p, V& a, V& b) {
        const float2 t = __ldg((const float2*)p);
        a = t.x;
        b = t.y;
    }
    static __device__ __forceinline__ void load2_rw(const T* p, V& a, V& b) {
        const float2 t = *(const float2*)p;
        a = t.x;
        b = t.y;
    }
    static __device__ __forceinline__ void store2(T* p, V a, V b) { *(float2*)p = make_float2(a, b); }
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
    if (threadIdx.x == 0 && threadIdx.y == 0) {
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

// CTAs of kThreads threads of `kernel` resident at once on the current device (cached)
int resident_ctas(const void* kernel) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find({kernel, dev});
    if (it != cache.end()) return it->second;
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = device_sms();
    cudaGetLastError();
    const int r = per_sm * sms;
    cache[{kernel, dev}] = r;
    return r;
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

// A CTA owns a (32 x 8)-point x-y tile and a chunk of z planes and marches through z:
// each thread keeps planes z-1, z, z+1 of its (x, y) column in registers, so a point
// costs one new load plus the four in-plane neighbours (L1 hits, loaded by the
// neighbouring threads), and the tile coordinates come from the launch shape with no
// per-point division.
template <int P>
__global__ void __launch_bounds__(kThreads) mp_stencil_kernel(StencilDesc A, const typename Mode<P>::T* __restrict__ v,
                                                              double fy, typename Mode<P>::T* __restrict__ y, double fw,
                                                              typename Mode<P>::T* __restrict__ w,
                                                              const double* dscale, const SolverState* st, int gate,
                                                              int zchunk, float2 c0s, float2 shs) {
    using M = Mode<P>;
    using Vt = typename M::V;
    __shared__ df64 fac[2];
    if (!gate_open(st, gate)) return;
    broadcast_factors(fy, fw, dscale, fac);
    const df64 vfy = fac[0], vfw = fac[1];
    // the centre coefficient of A - shift I: constant (split on the host), or per point
    const df64 c0 = df64{c0s.x, P == PREC_DF64 ? c0s.y : 0.f}, sh = df64{shs.x, shs.y};
    const int tx = (A.nx + 31) / 32;
    const int x = (int)(blockIdx.x % tx) * 32 + threadIdx.x;
    const int yy = (int)(blockIdx.x / tx) * 8 + threadIdx.y;
    const int zb = blockIdx.y * zchunk, ze = min(A.nz, zb + zchunk);
    if (x >= A.nx || yy >= A.ny || zb >= ze) return;      // no barrier below
    const bool three = A.dim == 3;
    const int64_t pl = (int64_t)A.nx * A.ny;
    int64_t p = (int64_t)zb * pl + (int64_t)yy * A.nx + x;
    Vt vm = (three && zb > 0) ? M::load(v + p - pl) : M::zero();
    Vt vc = M::load(v + p);
#pragma unroll 2
    for (int z = zb; z < ze; ++z, p += pl) {
        const Vt vp = (three && z + 1 < A.nz) ? M::load(v + p + pl) : M::zero();
        Vt nb[7];
        nb[0] = vc;
        nb[1] = x > 0 ? M::load(v + p - 1) : M::zero();
        nb[2] = x < A.nx - 1 ? M::load(v + p + 1) : M::zero();
        nb[3] = yy > 0 ? M::load(v + p - A.nx) : M::zero();
        nb[4] = yy < A.ny - 1 ? M::load(v + p + A.nx) : M::zero();
        nb[5] = vm;
        nb[6] = vp;
        if constexpr (P == PREC_DF64) {
            // centre, then the neighbours: exact products summed in double-float
            DfAcc acc;
            acc.add_prod(A.variable ? df_add(mp_coef<P>(A, 0, p), df_neg(sh)) : c0, nb[0]);
#pragma unroll
            for (int q = 1; q < 7; ++q)
                if (q < 2 * A.dim + 1) acc.add_prod(mp_coef<P>(A, q, p), nb[q]);
            acc.normalize();
            M::store(y + p, df_mul(vfy, df64{acc.hi, acc.lo}));
            if (w) M::store(w + p, df_mul(vfw, nb[0]));
        } else {
            float acc = __fmul_rn(A.variable ? __fsub_rn(mp_coef<P>(A, 0, p).hi, sh.hi) : c0.hi, nb[0]);
#pragma unroll
            for (int q = 1; q < 7; ++q)
                if (q < 2 * A.dim + 1) acc = __fmaf_rn(mp_coef<P>(A, q, p).hi, nb[q], acc);
            M::store(y + p, __fmul_rn(vfy.hi, acc));
            if (w) M::store(w + p, __fmul_rn(vfw.hi, nb[0]));
        }
        vm = vc;
        vc = vp;
    }
}

template <int P>
void mp_launch_stencil(const StencilDesc& A, const void* v, double fy, void* y, double fw, void* w,
                       const double* dscale, const SolverState* st, int gate, cudaStream_t stream, double shift) {
    using T = typename Mode<P>::T;
    const int tiles = ((A.nx + 31) / 32) * ((A.ny + 7) / 8);
    // z chunks: about one wave of 8 CTAs per SM, at least one plane per chunk
    int chunks = (8 * device_sms()) / tiles;
    chunks = chunks < 1 ? 1 : (chunks > A.nz ? A.nz : chunks);
    const int zchunk = (A.nz + chunks - 1) / chunks;
    chunks = (A.nz + zchunk - 1) / zchunk;
    // A.c[0] - shift and shift itself as float pairs (hi + lo to ~48 bits)
    const double c0 = A.c[0] - shift;
    const float c0h = (float)c0, shh = (float)shift;
    const float2 c0s = make_float2(c0h, (float)(c0 - (double)c0h));
    const float2 shs = make_float2(shh, (float)(shift - (double)shh));
    mp_stencil_kernel<P><<<dim3(tiles, chunks), dim3(32, 8), 0, stream>>>(A, (const T*)v, fy, (T*)y, fw, (T*)w, dscale,
                                                                          st, gate, zchunk, c0s, shs);
}

// ================================================================== fused matrix powers
// Y[:, 0] = vscale u, Y[:, j] = sigma A Y[:, j-1] for j = 1..S in one launch (constant
// coefficients). A CTA owns a (kTile x kTile) x-y tile and a chunk of z planes and
// marches through z: level 0 is the scaled start vector, and level j of plane z needs
// level j-1 on planes z-1, z, z+1, so level j trails level j-1 by one plane. Each level
// keeps a ring of its last 3 planes in shared memory over the tile plus a halo of S-j
// points (the halo shrinks by one per level); points outside the grid hold zero (the
// Dirichlet boundary). The S powers cost one read of u (halos from L2) and S writes.
constexpr int kTile = 16;

template <int S>
__host__ __device__ constexpr int lvl_w(int j) { return kTile + 2 * (S - j); }
template <int S>
__host__ __device__ constexpr int lvl_off(int j) {   // element offset of level j's ring
    int o = 0;
    for (int i = 0; i < j; ++i) o += 3 * lvl_w<S>(i) * lvl_w<S>(i);
    return o;
}

template <int P, int S>
__global__ void __launch_bounds__(kThreads) mp_powers_fused_kernel(StencilDesc A, const typename Mode<P>::T* __restrict__ u,
                                                                   typename Mode<P>::T* __restrict__ Y, int64_t ldy,
                                                                   double sigma, const double* dscale, int zchunk,
                                                                   const SolverState* st, int gate) {
    using M = Mode<P>;
    using Vt = typename M::V;
    extern __shared__ unsigned char smem_raw[];
    Vt* ring = reinterpret_cast<Vt*>(smem_raw);
    __shared__ df64 fac[2];
    if (!gate_open(st, gate)) return;
    broadcast_factors(sigma, 1.0, dscale, fac);          // fac[0] = sigma*vscale (unused), fac[1] = vscale
    __shared__ df64 sig_s;
    if (threadIdx.x == 0) sig_s = df_from_double(sigma);
    __syncthreads();
    const df64 vsc = fac[1], sg = sig_s;
    const int tilesx = (A.nx + kTile - 1) / kTile;
    const int x0 = (blockIdx.x % tilesx) * kTile, y0 = (blockIdx.x / tilesx) * kTile;
    const int zb = blockIdx.y * zchunk, ze = min(A.nz, zb + zchunk);
    const int64_t pl = (int64_t)A.nx * A.ny;
    df64 c[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) c[q] = df64{A.ch[q], P == PREC_DF64 ? A.cl[q] : 0.f};
    const bool three = A.dim == 3;
    for (int zc = zb - S; zc < ze + S; ++zc) {
        // level 0: plane zc of the scaled start vector
        if (zc >= 0 && zc < A.nz && zc >= zb - S && zc < ze + S) {
            constexpr int w0 = lvl_w<S>(0);
            Vt* dst = ring + lvl_off<S>(0) + (zc % 3) * w0 * w0;
            for (int t = threadIdx.x; t < w0 * w0; t += blockDim.x) {
                const int gx = x0 - S + t % w0, gy = y0 - S + t / w0;
                Vt v = M::zero();
                if (gx >= 0 && gx < A.nx && gy >= 0 && gy < A.ny) {
                    const int64_t gp = (int64_t)zc * pl + (int64_t)gy * A.nx + gx;
                    if constexpr (P == PREC_DF64) v = df_mul(vsc, M::load(u + gp));
                    else v = __fmul_rn(vsc.hi, M::load(u + gp));
                    const int lx = gx - x0, ly = gy - y0;
                    if (zc >= zb && zc < ze && lx >= 0 && lx < kTile && ly >= 0 && ly < kTile) M::store(Y + gp, v);
                }
                dst[t] = v;
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 1; j <= S; ++j) {
            const int z = zc - j;
            const bool active = z >= 0 && z < A.nz && z >= zb - (S - j) && z < ze + (S - j);
            if (active) {
                const int wp = lvl_w<S>(j - 1), wj = lvl_w<S>(j);
                const Vt* prev = ring + lvl_off<S>(j - 1);
                const Vt* pc = prev + (z % 3) * wp * wp;
                const Vt* pm = (three && z - 1 >= 0) ? prev + ((z + 2) % 3) * wp * wp : nullptr;
                const Vt* pp = (three && z + 1 < A.nz) ? prev + ((z + 1) % 3) * wp * wp : nullptr;
                Vt* dst = j < S ? ring + lvl_off<S>(j) + (z % 3) * wj * wj : nullptr;
                for (int t = threadIdx.x; t < wj * wj; t += blockDim.x) {
                    const int lx = t % wj, ly = t / wj;                 // in level j's region
                    const int gx = x0 - (S - j) + lx, gy = y0 - (S - j) + ly;
                    Vt r = M::zero();
                    if (gx >= 0 && gx < A.nx && gy >= 0 && gy < A.ny) {
                        const int q = (ly + 1) * wp + (lx + 1);              // same point in level j-1's region
                        if constexpr (P == PREC_DF64) {
                            DfAcc acc;
                            acc.add_prod(c[0], pc[q]);
                            acc.add_prod(c[1], pc[q - 1]);
                            acc.add_prod(c[2], pc[q + 1]);
                            acc.add_prod(c[3], pc[q - wp]);
                            acc.add_prod(c[4], pc[q + wp]);
                            if (pm) acc.add_prod(c[5], pm[q]);
                            if (pp) acc.add_prod(c[6], pp[q]);
                            acc.normalize();
                            r = df_mul(sg, df64{acc.hi, acc.lo});
                        } else {
                            float acc = __fmul_rn(c[0].hi, pc[q]);
                            acc = __fmaf_rn(c[1].hi, pc[q - 1], acc);
                            acc = __fmaf_rn(c[2].hi, pc[q + 1], acc);
                            acc = __fmaf_rn(c[3].hi, pc[q - wp], acc);
                            acc = __fmaf_rn(c[4].hi, pc[q + wp], acc);
                            if (pm) acc = __fmaf_rn(c[5].hi, pm[q], acc);
                            if (pp) acc = __fmaf_rn(c[6].hi, pp[q], acc);
                            r = __fmul_rn(sg.hi, acc);
                        }
                        const int tx = gx - x0, ty = gy - y0;
                        if (z >= zb && z < ze && tx >= 0 && tx < kTile && ty >= 0 && ty < kTile)
                            M::store(Y + (int64_t)j * ldy + (int64_t)z * pl + (int64_t)gy * A.nx + gx, r);
                    }
                    if (dst) dst[t] = r;
                }
            }
            __syncthreads();
        }
    }
}

template <int P>
bool mp_launch_powers_fused(const StencilDesc& A, const void* u, void* Y, int64_t ldy, int s, double sigma,
                            const double* dscale, const SolverState* st, int gate, cudaStream_t stream) {
    using T = typename Mode<P>::T;
    using Vt = typename Mode<P>::V;
    if (A.variable || !(s == 2 || s == 4 || s == 8)) return false;
    const int tiles = ((A.nx + kTile - 1) / kTile) * ((A.ny + kTile - 1) / kTile);
    // z chunks: enough CTAs to fill the GPU, no thinner than S planes (the recomputed halo)
    int zchunk = A.nz;
    while (zchunk > s && (int64_t)tiles * ((A.nz + zchunk - 1) / zchunk) < 3 * device_sms()) zchunk = (zchunk + 1) / 2;
    dim3 grid(tiles, (A.nz + zchunk - 1) / zchunk);
    switch (s) {
#define SSTEP_PF(S)                                                                                             \
    case S: {                                                                                                   \
        const size_t smem = sizeof(Vt) * lvl_off<S>(S);                                                        \
        cudaFuncSetAttribute(mp_powers_fused_kernel<P, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        mp_powers_fused_kernel<P, S><<<grid, kThreads, smem, stream>>>(A, (const T*)u, (T*)Y, ldy, sigma, dscale,  \
                                                                       zchunk, st, gate);                      \
        break;                                                                                                  \
    }
        SSTEP_PF(2)
        SSTEP_PF(4)
        SSTEP_PF(8)
#undef SSTEP_PF
        default: return false;
    }
    return true;
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
    int grid = grid_for(A.n, 4 * device_sms());
    mp_residual_kernel<P><<<grid, kThreads, 0, stream>>>(A, f, x, (T*)out, sc, epi, gate);
}

// ================================================================== Gram pass, double-float accumulation
// C[by*KA + i, j] = sum_rows V[row, by*KA + i] Y[row, j]. Each thread takes two
// consecutive rows per step (16-byte loads; the row past n in the last pair lies in
// the column padding and is masked out), and loads the next pair before it
// accumulates the current one.
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
    const int64_t npairs = (n + 1) / 2;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int cnt = 0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < npairs; q += stride) {
        const int64_t p = 2 * q;
        const bool second = p + 1 < n;
        Vt y0[KB], y1[KB], v0[KA], v1[KA];
#pragma unroll
        for (int j = 0; j < KB; ++j) M::load2(Y + p + j * ldy, y0[j], y1[j]);
#pragma unroll
        for (int i = 0; i < KA; ++i) M::load2(V + p + voff[i], v0[i], v1[i]);
        if (!second) {
#pragma unroll
            for (int i = 0; i < KA; ++i) v1[i] = M::zero();
        }
#pragma unroll
        for (int i = 0; i < KA; ++i)
            if (i < na) {
#pragma unroll
                for (int j = 0; j < KB; ++j) {
                    acc_add(acc[i * KB + j], v0[i], y0[j]);
                    acc_add(acc[i * KB + j], v1[i], y1[j]);
                }
            }
        if (++cnt == kRenorm / 2) {
            cnt = 0;
#pragma unroll
            for (int v = 0; v < NV; ++v) acc[v].normalize();
        }
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
    int gx = grid_for((n + 1) / 2, mp_red_ctas() * 2 / gy > 0 ? mp_red_ctas() * 2 / gy : 1);
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
// rounded once to the storage type. Two consecutive rows per thread (16-byte loads;
// every coefficient read from shared memory serves two products); the basis columns
// are read in groups of kChunk, the next group's loads issued before the current group
// is accumulated. With GRAM (used for narrow outputs) the kb x kb Gram of Yout is
// reduced in the same pass. Columns are allocated to an even length, so the row pair
// of an odd n reads and writes one padding entry, which the Gram leaves out.
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
    const int64_t npairs = (n + 1) / 2;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int nch = (ka + kChunk - 1) / kChunk;
    int cnt = 0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < npairs; q += stride) {
        const int64_t p = 2 * q;
        Vt y0[KB], y1[KB];
#pragma unroll
        for (int j = 0; j < KB; ++j) M::load2_rw(Yin + p + j * ldy, y0[j], y1[j]);
        if (ka > 0) {
            Vt c0[kChunk], c1[kChunk];
#pragma unroll
            for (int c = 0; c < kChunk; ++c) {
                if (c < ka) M::load2(V + p + (int64_t)c * ldv, c0[c], c1[c]);
                else c0[c] = c1[c] = M::zero();
            }
            DfAcc s0[KB], s1[KB];
            for (int ch = 0; ch < nch; ++ch) {
                const int base = ch * kChunk, nb = base + kChunk;
                Vt n0[kChunk], n1[kChunk];
#pragma unroll
                for (int c = 0; c < kChunk; ++c) {
                    if (nb + c < ka) M::load2(V + p + (int64_t)(nb + c) * ldv, n0[c], n1[c]);
                    else n0[c] = n1[c] = M::zero();
                }
#pragma unroll
                for (int c = 0; c < kChunk; ++c) {
                    if (base + c < ka) {
#pragma unroll
                        for (int j = 0; j < KB; ++j)
                            if (j >= j0) {
                                const df64 t = Ts[(base + c) * KB + j];
                                acc_add(s0[j], c0[c], t);
                                acc_add(s1[j], c1[c], t);
                            }
                    }
                }
#pragma unroll
                for (int c = 0; c < kChunk; ++c) {
                    c0[c] = n0[c];
                    c1[c] = n1[c];
                }
#pragma unroll
                for (int j = 0; j < KB; ++j) {
                    s0[j].normalize();
                    s1[j].normalize();
                }
            }
#pragma unroll
            for (int j = 0; j < KB; ++j)
                if (j >= j0) {
                    y0[j] = M::narrow(df_add(M::wide(y0[j]), df64{s0[j].hi, s0[j].lo}));
                    y1[j] = M::narrow(df_add(M::wide(y1[j]), df64{s1[j].hi, s1[j].lo}));
                }
        }
#pragma unroll
        for (int j = 0; j < KB; ++j)
            if (!inplace || (j >= j0 && ka > 0)) M::store2(Yout + p + j * ldo, y0[j], y1[j]);
        if (GRAM) {
            if (p + 1 >= n) {
#pragma unroll
                for (int j = 0; j < KB; ++j) y1[j] = M::zero();
            }
            int idx = 0;
#pragma unroll
            for (int qq = 0; qq < KB; ++qq)
#pragma unroll
                for (int pp = 0; pp <= qq; ++pp) {
                    acc_add(gacc[idx], y0[pp], y0[qq]);
                    acc_add(gacc[idx], y1[pp], y1[qq]);
                    ++idx;
                }
            if (++cnt == kRenorm / 2) {
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

// ================================================================== projection on row pairs
// Yout[:, j] = Yin[:, j] + V (sgn T)[:, j] for j >= j0, summed in double-float and
// rounded once. Two consecutive rows per thread: every coefficient read from shared
// memory serves two products, and the basis columns come in 16-byte loads, the next
// group of kChunk columns issued before the current group is accumulated.
template <int P, int KB>
__global__ void __launch_bounds__(kThreads) mp_project_kernel(int64_t n, const typename Mode<P>::T* __restrict__ V,
                                                              int64_t ldv, int ka, const typename Mode<P>::T* Yin,
                                                              int64_t ldy, typename Mode<P>::T* Yout, int64_t ldo,
                                                              int j0, const double* __restrict__ T, int ldt, double sgn,
                                                              Epi epi, int gate) {
    using M = Mode<P>;
    using Vt = typename M::V;
    __shared__ df64 Ts[kMaxCols * KB];
    if (!gate_open(epi.st, gate)) return;
    for (int t = threadIdx.x; t < ka * KB; t += blockDim.x) {
        const int i = t % ka, j = t / ka;
        Ts[i * KB + j] = df_from_double(sgn * T[i + (int64_t)j * ldt]);
    }
    __syncthreads();
    const bool inplace = (Yin == Yout) && (ldy == ldo);
    const int64_t npairs = (n + 1) / 2;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int nch = (ka + kChunk - 1) / kChunk;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < npairs; q += stride) {
        const int64_t p = 2 * q;
        Vt c0[kChunk], c1[kChunk];
#pragma unroll
        for (int c = 0; c < kChunk; ++c) {
            if (c < ka) M::load2(V + p + (int64_t)c * ldv, c0[c], c1[c]);
            else c0[c] = c1[c] = M::zero();
        }
        Vt y0[KB], y1[KB];
#pragma unroll
        for (int j = 0; j < KB; ++j) M::load2_rw(Yin + p + j * ldy, y0[j], y1[j]);
        DfAcc s0[KB], s1[KB];
        for (int ch = 0; ch < nch; ++ch) {
            const int base = ch * kChunk, nb = base + kChunk;
            Vt n0[kChunk], n1[kChunk];
#pragma unroll
            for (int c = 0; c < kChunk; ++c) {
                if (nb + c < ka) M::load2(V + p + (int64_t)(nb + c) * ldv, n0[c], n1[c]);
                else n0[c] = n1[c] = M::zero();
            }
#pragma unroll
            for (int c = 0; c < kChunk; ++c) {
                if (base + c < ka) {
#pragma unroll
                    for (int j = 0; j < KB; ++j)
                        if (j >= j0) {
                            const df64 t = Ts[(base + c) * KB + j];
                            acc_add(s0[j], c0[c], t);
                            acc_add(s1[j], c1[c], t);
                        }
                }
            }
#pragma unroll
            for (int c = 0; c < kChunk; ++c) {
                c0[c] = n0[c];
                c1[c] = n1[c];
            }
#pragma unroll
            for (int j = 0; j < KB; ++j) {
                s0[j].normalize();
                s1[j].normalize();
            }
        }
#pragma unroll
        for (int j = 0; j < KB; ++j) {
            if (j >= j0 && ka > 0) {
                y0[j] = M::narrow(df_add(M::wide(y0[j]), df64{s0[j].hi, s0[j].lo}));
                y1[j] = M::narrow(df_add(M::wide(y1[j]), df64{s1[j].hi, s1[j].lo}));
            }
            if (!inplace || (j >= j0 && ka > 0)) M::store2(Yout + p + j * ldo, y0[j], y1[j]);
        }
    }
}

// ================================================================== Gram of one block (symmetric)
// G = Y^T Y for kb columns; the packed upper triangle (entry (p, q), p <= q, at
// q(q+1)/2 + p) is split between two CTA groups by column q (q < QS and q >= QS,
// QS chosen to balance the entry counts) so neither group runs out of registers.
// Two rows per thread with 16-byte loads; double-float accumulation.
__host__ __device__ constexpr int tri(int q) { return q * (q + 1) / 2; }
__host__ __device__ constexpr int sym_split(int kb) {
    int best = 1, bestv = 1 << 30;
    for (int q = 1; q < kb; ++q) {
        const int a = tri(q), b = tri(kb) - tri(q);
        const int v = a > b ? a : b;
        if (v < bestv) {
            bestv = v;
            best = q;
        }
    }
    return best;
}

template <int P, int KB, int Q0, int Q1>
__device__ __forceinline__ void symgram_rows(int64_t n, const typename Mode<P>::T* __restrict__ Y, int64_t ldy,
                                             DfAcc* acc) {
    using M = Mode<P>;
    using Vt = typename M::V;
    constexpr int NV = tri(Q1) - tri(Q0);
    const int64_t npairs = (n + 1) / 2;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int cnt = 0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < npairs; q += stride) {
        const int64_t p = 2 * q;
        Vt y0[Q1], y1[Q1];
#pragma unroll
        for (int j = 0; j < Q1; ++j) M::load2(Y + p + j * ldy, y0[j], y1[j]);
        if (p + 1 >= n) {
#pragma unroll
            for (int j = 0; j < Q1; ++j) y1[j] = M::zero();
        }
        int idx = 0;
#pragma unroll
        for (int c = Q0; c < Q1; ++c)
#pragma unroll
            for (int r = 0; r <= c; ++r) {
                acc_add(acc[idx], y0[r], y0[c]);       // float x float in FP32 mode: exact product
                acc_add(acc[idx], y1[r], y1[c]);
                ++idx;
            }
        if (++cnt == kRenorm / 2) {
            cnt = 0;
#pragma unroll
            for (int v = 0; v < NV; ++v) acc[v].normalize();
        }
    }
}

template <int P, int KB>
__global__ void __launch_bounds__(kThreads) mp_symgram_kernel(int64_t n, const typename Mode<P>::T* __restrict__ Y,
                                                              int64_t ldy, Scratch sc, Epi epi, int gate) {
    constexpr int QS = sym_split(KB);
    constexpr int NV0 = tri(QS), NV1 = tri(KB) - tri(QS);
    constexpr int NVM = NV0 > NV1 ? NV0 : NV1;
    __shared__ double red[(kWarps + 1) * NVM];
    __shared__ double res[(kMaxS + 1) * (kMaxS + 1)];
    __shared__ double packed[tri(KB)];
    if (!gate_open(epi.st, gate)) return;
    DfAcc acc[NVM];
    if (blockIdx.y == 0) symgram_rows<P, KB, 0, QS>(n, Y, ldy, acc);
    else symgram_rows<P, KB, QS, KB>(n, Y, ldy, acc);
    block_reduce_df<NVM>(acc, red);
    if (!publish_partial(red + kWarps * NVM, NVM, sc.partials, sc.counter)) return;
    const int gx = gridDim.x;
    for (int e = threadIdx.x; e < tri(KB); e += blockDim.x) {
        const int g = e < NV0 ? 0 : 1, le = g == 0 ? e : e - NV0;
        double t = 0.0;
        for (int bx = 0; bx < gx; ++bx) t += ld_cg(sc.partials + (int64_t)(g * gx + bx) * NVM + le);
        packed[e] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) *sc.counter = 0u;
    for (int t = threadIdx.x; t < KB * KB; t += blockDim.x) {
        int pp = t % KB, q = t / KB;
        if (pp > q) {
            const int tmp = pp;
            pp = q;
            q = tmp;
        }
        res[t] = packed[tri(q) + pp];
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
    if (!gram) {
        int grid = grid_for((n + 1) / 2, mp_ctas());
        switch (kb) {
#define SSTEP_MPP(KB)                                                                                             \
    case KB:                                                                                                      \
        mp_project_kernel<P, KB><<<grid, kThreads, 0, stream>>>(n, Vp, ldv, ka, Yi, ldy, Yo, ldo, j0, T, ldt, sgn, \
                                                                epi, gate);                                      \
        break;
            SSTEP_MPP(1)
            SSTEP_MPP(2)
            SSTEP_MPP(3)
            SSTEP_MPP(4)
            SSTEP_MPP(5)
            SSTEP_MPP(6)
            SSTEP_MPP(7)
            SSTEP_MPP(8)
            SSTEP_MPP(9)
#undef SSTEP_MPP
            default: break;
        }
        return;
    }
    if (kb > 2) {
        // wide blocks: the projection alone (light, many CTAs), then the block's Gram over
        // one wave of CTAs (two column groups along grid.y)
        mp_launch_update<P>(n, V, ldv, ka, Yin, ldy, Yout, ldo, kb, j0, T, ldt, sgn, false, sc, epi, gate, stream);
        switch (kb) {
#define SSTEP_MPS(KB)                                                                                             \
    case KB: {                                                                                                    \
        const int wave = std::min(max_ctas_mp(), resident_ctas((const void*)mp_symgram_kernel<P, KB>));             \
        dim3 grid(grid_for((n + 1) / 2, wave / 2 > 0 ? wave / 2 : 1), 2);                                         \
        mp_symgram_kernel<P, KB><<<grid, kThreads, 0, stream>>>(n, Yo, ldo, sc, epi, gate);                       \
    } break;
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
    // one wave of CTAs (the partials buffer holds 8 CTAs per multiprocessor x kMaxNV doubles)
    switch (kb) {
        case 1: {
            const int grid = grid_for((n + 1) / 2, std::min(max_ctas_mp(), resident_ctas((const void*)mp_update_kernel<P, 1, true>)));
            mp_update_kernel<P, 1, true><<<grid, kThreads, 0, stream>>>(n, Vp, ldv, ka, Yi, ldy, Yo, ldo, j0, T, ldt, sgn,
                                                                        sc, epi, gate);
        } break;
        case 2: {
            const int grid = grid_for((n + 1) / 2, std::min(max_ctas_mp(), resident_ctas((const void*)mp_update_kernel<P, 2, true>)));
            mp_update_kernel<P, 2, true><<<grid, kThreads, 0, stream>>>(n, Vp, ldv, ka, Yi, ldy, Yo, ldo, j0, T, ldt, sgn,
                                                                        sc, epi, gate);
        } break;
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
    int grid = grid_for(n, mp_ctas() * 2);
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
    split_fields_kernel<<<grid_for(n, 8 * device_sms()), kThreads, 0, stream>>>(src, dst, n);
}

// ------------------------------------------------------------------ instantiations
#define SSTEP_MP_INST(P)                                                                                          \
    template void mp_launch_stencil<P>(const StencilDesc&, const void*, double, void*, double, void*,            \
                                       const double*, const SolverState*, int, cudaStream_t, double);            \
    template void mp_launch_residual<P>(const StencilDesc&, const double*, const double*, void*, Scratch,        \
                                        const Epi&, int, cudaStream_t);                                          \
    template void mp_launch_gram<P>(int64_t, const void*, int64_t, int, const void*, int64_t, int, Scratch,      \
                                    const Epi&, int, cudaStream_t);                                              \
    template void mp_launch_update<P>(int64_t, const void*, int64_t, int, const void*, int64_t, void*, int64_t,  \
                                      int, int, const double*, int, double, bool, Scratch, const Epi&, int,      \
                                      cudaStream_t);                                                             \
    template void mp_launch_axpy<P>(int64_t, const void*, int64_t, double*, const Epi&, int, cudaStream_t);      \
    template bool mp_launch_powers_fused<P>(const StencilDesc&, const void*, void*, int64_t, int, double,         \
                                            const double*, const SolverState*, int, cudaStream_t);
SSTEP_MP_INST(PREC_DF64)
SSTEP_MP_INST(PREC_FP32)
#undef SSTEP_MP_INST

}  // namespace sstep
