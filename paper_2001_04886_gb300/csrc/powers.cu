// Fused matrix powers of the FP64 s-step block with TMA-staged tiles (Alg. 4.1 step 3;
// Sec. 1: s products for about one sweep over the start vector).
//
// Y[:, 0] = d u and Y[:, j] = sigma (A - theta_{j-1} I) Y[:, j-1] for j = 1..S (d = the
// scale of the start vector, 1 / ||u||, read on the device; constant coefficients). A CTA
// owns a TX x TY tile of the x-y plane and a chunk of z planes and marches through z.
// Level 0 is the start vector: each of its planes, the tile plus an S-point halo, is one
// TMA box copy (cp.async.bulk.tensor.3d) into a ring of four shared-memory slots, issued a
// plane ahead and completed on an mbarrier; the grid boundary is the copy's zero fill.
// Level j (1..S) of plane z needs level j - 1 on planes z - 1, z, z + 1 over a halo one point
// wider, so it trails level j - 1 by one plane and keeps a ring of three planes over the
// tile plus S - j halo points; level S is written to global memory only. Every point of
// every level is computed with the separate sweep's coefficients and in its order of
// multiply-adds, neighbours outside the grid skipped, so the columns equal the separate
// sweeps' (stencil_const_kernel) bit for bit; the tile's points of each level are stored
// and their column bound recorded. The halos recompute points (at S = 8 on a 32 x 16 tile
// about 1.8x the sweeps' multiply-adds in x-y, 2.7x with the z halo of 16-plane chunks),
// which the FP64 pipe pays: at 128^3 this launch takes about 3x the separate sweeps, so
// the solver uses it only when SSTEP_FUSED_POWERS=1.
#include <cuda.h>

#include "kernels.cuh"

namespace sstep {
namespace {

constexpr int kPTX = 32, kPTY = 16;      // tile in x, y
constexpr int kPThreads = 256;
constexpr long kPSpin = 1L << 24;        // bounded mbarrier polls

template <int S>
struct PCfg {
    static constexpr int w(int j) { return kPTX + 2 * (S - j); }
    static constexpr int h(int j) { return kPTY + 2 * (S - j); }
    static constexpr int area(int j) { return w(j) * h(j); }
    // byte offset of level j's ring: level 0 holds 4 slots, levels 1..S-1 three
    static constexpr int off(int j) {
        int o = 0;
        for (int i = 0; i < j; ++i) o += (i == 0 ? 4 : 3) * area(i) * 8;
        return o;
    }
    static constexpr int kSmem = off(S);
    static_assert(kSmem <= 227 * 1024 - 1024, "shared memory");
};

__device__ __forceinline__ uint32_t s_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool p_wait(uint32_t bar, uint32_t parity, long limit) {
    uint32_t done = 0;
    for (long it = 0; it < limit && !done; ++it)
        asm volatile("{\n.reg .pred P;\nmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\nselp.b32 %0, 1, 0, P;\n}"
                     : "=r"(done)
                     : "r"(bar), "r"(parity)
                     : "memory");
    return done != 0;
}

struct PowerOut {
    unsigned* b1[kMaxS + 1];   // column-bound records of column j (two per column, either null)
    unsigned* b2[kMaxS + 1];
    double theta[kMaxS];       // shift of power j + 1
};

template <int S, bool THREE>
__global__ void __launch_bounds__(kPThreads, 1)
    powers_fused_kernel(const __grid_constant__ CUtensorMap tmap, int nx, int ny, int nz, double c0, double c1,
                        double c2, double c3, double c4, double c5, double c6, double sigma, const double* dscale,
                        double* __restrict__ Y, int64_t ldy, int zchunk, PowerOut po, const SolverState* st, int gate,
                        unsigned* err) {
    using C = PCfg<S>;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[4];
    __shared__ double kc[S + 1][7];   // coefficients of each level (level 0: the scale of the copy)
    __shared__ int failed;
    if (!gate_open(st, gate)) return;
    const int tid = threadIdx.x;
    const double d = *dscale;
    if (tid <= S) {
        // level 1: (sigma d) (A - theta_0 I); level j >= 2: sigma (A - theta_{j-1} I); level 0: d
        const double a[7] = {c0, c1, c2, c3, c4, c5, c6};
        if (tid == 0) {
            kc[0][0] = 1.0 * d;
        } else {
            const double f = tid == 1 ? sigma * d : sigma;
            kc[tid][0] = f * (a[0] - po.theta[tid - 1]);
            for (int q = 1; q < 7; ++q) kc[tid][q] = f * a[q];
        }
    }
    if (tid == 0) {
        failed = 0;
        for (int b = 0; b < 4; ++b)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_addr(&full[b])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    __syncthreads();
    const int tilesx = (nx + kPTX - 1) / kPTX;
    const int x0 = (int)(blockIdx.x % tilesx) * kPTX, y0 = (int)(blockIdx.x / tilesx) * kPTY;
    const int zb = blockIdx.y * zchunk, ze = min(nz, zb + zchunk);
    const int64_t pl = (int64_t)nx * ny;
    constexpr uint32_t kBox = (uint32_t)C::area(0) * 8u;
    // level-0 plane zc into slot it % 4 (it counts the planes of this CTA from 0)
    auto issue = [&](int it, int zc) {
        const int b = it & 3;
        const uint32_t bar = s_addr(&full[b]);
        const uint32_t dst = s_addr(smem + C::off(0) + b * C::area(0) * 8);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kBox) : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
            ::"r"(dst), "l"(&tmap), "r"(x0 - S), "r"(y0 - S), "r"(zc), "r"(bar)
            : "memory");
    };
    const int zfirst = zb - S, zlast = ze + S;   // level-0 planes this CTA reads: [zfirst, zlast)
    unsigned bm[S + 1];
#pragma unroll
    for (int j = 0; j <= S; ++j) bm[j] = 0u;
    if (tid == 0) issue(0, zfirst);
    int issued = 0;   // the last plane count issued (every one is waited for before the CTA ends)
    for (int zc = zfirst; zc < zlast + S; ++zc) {
        const int it = zc - zfirst;
        if (zc < zlast) {
            if (tid == 0 && zc + 1 < zlast) issue(it + 1, zc + 1);
            if (zc + 1 < zlast) issued = it + 1;
            if (!p_wait(s_addr(&full[it & 3]), (uint32_t)((it >> 2) & 1), kPSpin)) failed = 1;
        }
        __syncthreads();
        if (failed) {   // no copy may land after the CTA has gone: wait (bounded) for those in flight
            if (tid == 0)
                for (int q = it; q <= issued; ++q) p_wait(s_addr(&full[q & 3]), (uint32_t)((q >> 2) & 1), kPSpin);
            break;
        }
        // level 0: the copy d u of the tile's points of plane zc
        if (zc >= zb && zc < ze) {
            const double* l0 = reinterpret_cast<const double*>(smem + C::off(0) + (it & 3) * C::area(0) * 8);
            for (int t = tid; t < kPTX * kPTY; t += kPThreads) {
                const int lx = t % kPTX, ly = t / kPTX, gx = x0 + lx, gy = y0 + ly;
                if (gx < nx && gy < ny) {
                    const double wv = kc[0][0] * l0[(ly + S) * C::w(0) + lx + S];
                    Y[(int64_t)zc * pl + (int64_t)gy * nx + gx] = wv;
                    bm[0] = max(bm[0], (unsigned)(__double_as_longlong(fabs(wv)) >> 32));
                }
            }
        }
#pragma unroll
        for (int j = 1; j <= S; ++j) {
            const int z = zc - j;                       // level j's plane this step
            if (z >= zb - (S - j) && z < ze + (S - j) && z >= 0 && z < nz) {
                const int wp = C::w(j - 1), wj = C::w(j), hj = C::h(j);
                // level j-1's planes z - 1, z, z + 1: level 0 in its 4-slot ring by plane
                // count, the others in 3-slot rings by plane index
                const double* base = reinterpret_cast<const double*>(smem + C::off(j - 1));
                auto plane = [&](int zz) -> const double* {
                    if (j == 1) return base + ((zz - zfirst) & 3) * C::area(0);
                    return base + (((zz % 3) + 3) % 3) * C::area(j - 1);
                };
                const double* pc = plane(z);
                const double* pm = plane(z - 1);
                const double* pp = plane(z + 1);
                double* dst = j < S ? reinterpret_cast<double*>(smem + C::off(j)) + (z % 3) * C::area(j) : nullptr;
                const double k0 = kc[j][0], k1 = kc[j][1], k2 = kc[j][2], k3 = kc[j][3], k4 = kc[j][4], k5 = kc[j][5],
                             k6 = kc[j][6];
                const bool store = z >= zb && z < ze;
                for (int t = tid; t < wj * hj; t += kPThreads) {
                    const int lx = t % wj, ly = t / wj;
                    const int gx = x0 - (S - j) + lx, gy = y0 - (S - j) + ly;
                    double r = 0.0;
                    if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) {
                        const int q = (ly + 1) * wp + (lx + 1);
                        double acc = k0 * pc[q];
                        if (gx > 0) acc = fma(k1, pc[q - 1], acc);
                        if (gx < nx - 1) acc = fma(k2, pc[q + 1], acc);
                        if (gy > 0) acc = fma(k3, pc[q - wp], acc);
                        if (gy < ny - 1) acc = fma(k4, pc[q + wp], acc);
                        if (THREE) {
                            if (z > 0) acc = fma(k5, pm[q], acc);
                            if (z < nz - 1) acc = fma(k6, pp[q], acc);
                        }
                        r = acc;
                        const int tx = gx - x0, ty = gy - y0;
                        if (store && tx >= 0 && tx < kPTX && ty >= 0 && ty < kPTY) {
                            Y[(int64_t)j * ldy + (int64_t)z * pl + (int64_t)gy * nx + gx] = r;
                            bm[j] = max(bm[j], (unsigned)(__double_as_longlong(fabs(r)) >> 32));
                        }
                    }
                    if (dst) dst[t] = r;
                }
            }
            __syncthreads();
        }
    }
    // column bounds: warp maximum, one atomic per warp and record
    const int lane = tid & 31;
#pragma unroll
    for (int j = 0; j <= S; ++j) {
        const unsigned m = __reduce_max_sync(0xffffffffu, bm[j]);
        if (lane == 0 && m) {
            if (po.b1[j]) atomicMax(po.b1[j], m);
            if (po.b2[j]) atomicMax(po.b2[j], m);
        }
    }
    if (failed && tid == 0) {
        if (err) atomicExch(err, 1u);
        if (st) {
            SolverState* sw = const_cast<SolverState*>(st);
            sw->status = SSTEP_ERR_TIMEOUT;
            sw->building = 0;
            sw->active = 0;
        }
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        return (EncodeTiledFn)p;
    }();
    return fn;
}

template <int S, bool THREE>
void launch_pf(const CUtensorMap& tm, const StencilDesc& A, double sigma, const double* dscale, double* Y, int64_t ldy,
               const PowerOut& po, const SolverState* st, int gate, cudaStream_t stream, unsigned* err) {
    using C = PCfg<S>;
    static bool attr[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attr[dev]) {
        cudaFuncSetAttribute(powers_fused_kernel<S, THREE>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem);
        if (dev >= 0 && dev < 64) attr[dev] = true;
    }
    const int tiles = ((A.nx + kPTX - 1) / kPTX) * ((A.ny + kPTY - 1) / kPTY);
    // z chunks: about one CTA per SM, no thinner than 2 S planes (the recomputed z halo)
    int zchunk = A.nz;
    while (zchunk > 2 * S && (int64_t)tiles * ((A.nz + zchunk - 1) / zchunk) < device_sms()) zchunk = (zchunk + 1) / 2;
    const dim3 grid(tiles, (A.nz + zchunk - 1) / zchunk);
    powers_fused_kernel<S, THREE><<<grid, kPThreads, C::kSmem, stream>>>(
        tm, A.nx, A.ny, A.nz, A.c[0], A.c[1], A.c[2], A.c[3], A.c[4], A.c[5], A.c[6], sigma, dscale, Y, ldy, zchunk, po,
        st, gate, err);
}

}  // namespace

bool launch_powers_fused(const StencilDesc& A, const double* u, double sigma, const double* dscale, double* Y,
                         int64_t ldy, int s, const double* theta, unsigned* const* b1, unsigned* const* b2,
                         const SolverState* st, int gate, cudaStream_t stream, unsigned* err) {
    EncodeTiledFn fn = encode_fn();
    if (!fn || A.variable || !(s == 2 || s == 4 || s == 8) || (A.nx & 1) || ((uintptr_t)u & 15) ||
        ((uintptr_t)Y & 7) || A.nx > 1 << 20 || A.ny > 1 << 20 || A.nz > 1 << 20)
        return false;
    // u as an nx x ny x nz FP64 tensor; the box is the tile plus s halo points on each side
    alignas(128) CUtensorMap tm;
    const cuuint64_t dims[3] = {(cuuint64_t)A.nx, (cuuint64_t)A.ny, (cuuint64_t)A.nz};
    const cuuint64_t strides[2] = {(cuuint64_t)A.nx * 8, (cuuint64_t)A.nx * A.ny * 8};
    const cuuint32_t box[3] = {(cuuint32_t)(kPTX + 2 * s), (cuuint32_t)(kPTY + 2 * s), 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (fn(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, const_cast<double*>(u), dims, strides, box, estr,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    PowerOut po;
    for (int j = 0; j <= kMaxS; ++j) {
        po.b1[j] = (b1 && j <= s) ? b1[j] : nullptr;
        po.b2[j] = (b2 && j <= s) ? b2[j] : nullptr;
    }
    for (int j = 0; j < kMaxS; ++j) po.theta[j] = (theta && j < s) ? theta[j] : 0.0;
    const bool three = A.dim == 3;
#define SSTEP_PFC(S_)                                                                                          \
    if (s == S_) {                                                                                             \
        if (three) launch_pf<S_, true>(tm, A, sigma, dscale, Y, ldy, po, st, gate, stream, err);              \
        else launch_pf<S_, false>(tm, A, sigma, dscale, Y, ldy, po, st, gate, stream, err);                   \
        return true;                                                                                           \
    }
    SSTEP_PFC(2)
    SSTEP_PFC(4)
    SSTEP_PFC(8)
#undef SSTEP_PFC
    return false;
}

}  // namespace sstep
