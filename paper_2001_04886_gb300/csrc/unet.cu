// Learned initial guess: a 4-level convolutional U-Net that maps (f, beta) on an
// H x W grid to x0, trained on the GPU with these kernels only.
//
// Weights are stored in BF16 (an FP32 master copy is kept for Adam); every
// product accumulates in FP32; activations are FP32, NCHW. A debug mode runs the
// same kernels with FP32 weights (for tight gradient checks against the CPU
// oracle).
//
// Architecture (channels 16, 32, 64, 64; 3x3 convolutions with padding 1, ReLU):
//   enc1: 2->16->16 (HxW)   pool   enc2: 16->32->32 (H/2)   pool
//   enc3: 32->64->64 (H/4)  pool   bottom: 64->64->64 (H/8)
//   up + concat enc3 -> dec3: 128->64->64;  up + concat enc2 -> dec2: 96->32->32
//   up + concat enc1 -> dec1: 48->16->16;   out: 1x1 conv 16->1 (no ReLU),
//   then `smooth` passes of the fixed separable filter [1 2 1]/4 x [1 2 1]/4 (zero
//   outside the grid). The solutions are smooth; the filter removes the high-frequency
//   noise of the prediction, which the operator would amplify in the residual.
// Pooling is 2x2 averaging, upsampling is nearest-neighbour. Parameters are one
// flat FP32 vector: per layer the weights [co][ci][kh][kw], then the biases [co].
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <new>
#include <type_traits>
#include <vector>

#include "../../include/sstep.h"

namespace sstep {
int device_sms();   // multiprocessors of the current device (ozaki.cu)
}

namespace unet {

constexpr int kT = 256;

struct ConvSpec {
    int cin, cout, k;   // k = 3 or 1
    int relu;
};

// the 15 convolutions in forward order
constexpr int kNumLayers = 15;
constexpr ConvSpec kLayers[kNumLayers] = {
    {2, 16, 3, 1},   {16, 16, 3, 1},  {16, 32, 3, 1}, {32, 32, 3, 1}, {32, 64, 3, 1},
    {64, 64, 3, 1},  {64, 64, 3, 1},  {64, 64, 3, 1}, {128, 64, 3, 1}, {64, 64, 3, 1},
    {96, 32, 3, 1},  {32, 32, 3, 1},  {48, 16, 3, 1}, {16, 16, 3, 1}, {16, 1, 1, 0}};

inline int64_t layer_params(const ConvSpec& c) { return (int64_t)c.cout * c.cin * c.k * c.k + c.cout; }

// ------------------------------------------------------------------ kernels
template <typename WT>
__device__ __forceinline__ float wload(const WT* w, int64_t i);
template <>
__device__ __forceinline__ float wload<float>(const float* w, int64_t i) { return w[i]; }
template <>
__device__ __forceinline__ float wload<__nv_bfloat16>(const __nv_bfloat16* w, int64_t i) {
    return __bfloat162float(w[i]);
}

// Direct 3x3 convolution, zero padding. A CTA computes a 16x16 pixel tile for 16
// output channels: the input tile with its halo and the 16x9 weights of one input
// channel at a time are staged in shared memory.
// TRANSPOSED: the backward-data form, dX[ci] = sum_co W[co][ci] (rotated 180 deg) * dY[co]:
// here `in` is dY (Cin = forward Cout) and `out` is dX (Cout = forward Cin).
template <typename WT, bool TRANSPOSED>
__global__ void __launch_bounds__(kT) conv3x3_kernel(const float* __restrict__ in, int Cin, const WT* __restrict__ W,
                                                     const float* __restrict__ bias, float* __restrict__ out,
                                                     int Cout, int H, int Wd, int relu, int accumulate) {
    __shared__ float tile[18][18];
    __shared__ float wsm[16][9];
    const int ngroups = (Cout + 15) / 16;
    const int b = blockIdx.z / ngroups, co0 = (blockIdx.z % ngroups) * 16;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int x = blockIdx.x * 16 + tx, y = blockIdx.y * 16 + ty;
    const int nco = min(16, Cout - co0);
    float acc[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) acc[c] = (bias && c < nco) ? bias[co0 + c] : 0.f;
    const int64_t plane = (int64_t)H * Wd;
    for (int ci = 0; ci < Cin; ++ci) {
        const float* src = in + ((int64_t)b * Cin + ci) * plane;
        for (int t = threadIdx.x; t < 18 * 18; t += kT) {
            const int yy = blockIdx.y * 16 + t / 18 - 1, xx = blockIdx.x * 16 + t % 18 - 1;
            tile[t / 18][t % 18] = (yy >= 0 && yy < H && xx >= 0 && xx < Wd) ? src[(int64_t)yy * Wd + xx] : 0.f;
        }
        for (int t = threadIdx.x; t < 16 * 9; t += kT) {
            const int c = t / 9, k = t % 9;
            float w = 0.f;
            if (c < nco) {
                if (!TRANSPOSED) w = wload(W, ((int64_t)(co0 + c) * Cin + ci) * 9 + k);
                else w = wload(W, ((int64_t)ci * Cout + (co0 + c)) * 9 + (8 - k));   // W[fwd co=ci][fwd ci=co0+c]
            }
            wsm[c][k] = w;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const float v = tile[ty + k / 3][tx + k % 3];
#pragma unroll
            for (int c = 0; c < 16; ++c) acc[c] = fmaf(wsm[c][k], v, acc[c]);
        }
        __syncthreads();
    }
    if (x >= Wd || y >= H) return;
    for (int c = 0; c < nco; ++c) {
        float v = acc[c];
        if (relu) v = fmaxf(v, 0.f);
        float* dst = out + ((int64_t)b * Cout + co0 + c) * plane + (int64_t)y * Wd + x;
        *dst = accumulate ? *dst + v : v;
    }
}

// ------------------------------------------------------------------ 3x3 convolution on the tensor cores
// Implicit GEMM with tcgen05: D[pixel][n] = sum over (tap, channel) A[pixel][(tap, c)] B[n][(tap, c)]
// for a tile of 128 consecutive pixels of one image (one CTA of 128 threads, thread m <->
// pixel m, which is TMEM lane m of the accumulator). The K dimension runs over the 9 taps x
// the input channels in chunks of 16. The FP32 activation of every product is split into
// three BF16 parts (hi + mid + lo represents all 24 bits of its significand), and each
// part is multiplied by the BF16 weight in its own MMA: the products are exact and the
// tensor core accumulates them in FP32, so the layer computes what the CUDA-core kernel
// computes (BF16 weights, FP32 activations, FP32 accumulation) up to the order of the sums.
// Operands are staged by the threads in shared memory in the K-major no-swizzle layout
// (8-row x 16-byte core matrices, 128 B between K-adjacent and 256 B between row-adjacent
// core matrices), two stages deep: while the MMAs of chunk i run, the threads gather chunk
// i + 1. One thread issues the MMAs and commits them to the stage's mbarrier; every wait
// is bounded and a wait that runs out sets *err, skips the rest of the work and still
// frees the tensor memory. TRANSPOSED: the backward-data form (weights W[co][ci] read as
// B[n = ci][c = co] with the taps rotated by 180 degrees).
namespace tc {

constexpr int kM = 128;                 // pixels per CTA (MMA M)
constexpr int kK = 16;                  // K per MMA (BF16)
constexpr int kLbo = 128, kSbo = 256;   // core-matrix strides (bytes)
constexpr long kSpin = 1L << 24;        // bounded mbarrier polls

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t kmaj(int r, int kq) {   // byte offset of row r, 8-element K group kq
    return (uint32_t)((r >> 3) * kSbo + kq * kLbo + (r & 7) * 16);
}

__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(kLbo >> 4) << 16) | ((uint64_t)(kSbo >> 4) << 32) |
           ((uint64_t)1 << 46);
}

__host__ __device__ constexpr uint32_t idesc(int n) {   // BF16 x BF16 -> FP32, K-major A and B, M = 128
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
}

__host__ __device__ constexpr int tmem_cols(int n) { return n <= 32 ? 32 : (n <= 64 ? 64 : (n <= 128 ? 128 : 256)); }

__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, long limit = kSpin) {
    uint32_t done = 0;
    for (long it = 0; it < limit && !done; ++it)
        asm volatile("{\n.reg .pred P;\nmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\nselp.b32 %0, 1, 0, P;\n}"
                     : "=r"(done)
                     : "r"(bar), "r"(parity)
                     : "memory");
    return done != 0;
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 a, __nv_bfloat16 b) {
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// v = h + m + l exactly: three BF16 parts of an FP32 value (8 significand bits each)
__device__ __forceinline__ void split3(float v, __nv_bfloat16& h, __nv_bfloat16& m, __nv_bfloat16& l) {
    h = __float2bfloat16_rn(v);
    const float r1 = __fsub_rn(v, __bfloat162float(h));
    m = __float2bfloat16_rn(r1);
    l = __float2bfloat16_rn(__fsub_rn(r1, __bfloat162float(m)));
}

template <int NP, bool TRANSPOSED>
__global__ void __launch_bounds__(kM) conv3x3_tc_kernel(const float* __restrict__ in, int Kc,
                                                        const __nv_bfloat16* __restrict__ W,
                                                        const float* __restrict__ bias, float* __restrict__ out,
                                                        int N, int H, int Wd, int relu, int accumulate, int* err,
                                                        long spin) {
    constexpr int kABytes = kM * kK * 2;          // one BF16 part of the A chunk
    constexpr int kBBytes = NP * kK * 2;
    constexpr int kStage = 3 * kABytes + kBBytes;
    constexpr uint32_t kCols = tmem_cols(NP);
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ uint32_t tmem_base;
    __shared__ int failed;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int b = blockIdx.y;
    const int64_t HW = (int64_t)H * Wd;
    const int64_t p = (int64_t)blockIdx.x * kM + tid;   // this thread's pixel (A row / TMEM lane)
    const bool live = p < HW;
    const int py = live ? (int)(p / Wd) : 0, px = live ? (int)(p - (int64_t)py * Wd) : 0;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        failed = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    const int kgroups = (Kc + kK - 1) / kK;
    const int nchunks = 9 * kgroups;
    const float* inb = in + (int64_t)b * Kc * HW;
    bool ok = true;
    for (int i = 0; i < nchunks && ok; ++i) {
        const int st = i & 1;
        if (i >= 2) {   // the MMAs that read this stage (chunk i - 2) are done
            if (!wait_bar(smem_u32(&bars[st]), (uint32_t)(((i >> 1) - 1) & 1), spin)) {
                failed = 1;
            }
            __syncthreads();
            if (failed) {   // drain: the MMAs of chunks i - 2 and i - 1 are still in flight
                wait_bar(smem_u32(&bars[st]), (uint32_t)(((i >> 1) - 1) & 1));
                wait_bar(smem_u32(&bars[st ^ 1]), (uint32_t)(((i - 1) >> 1) & 1));
                ok = false;
                break;
            }
        }
        const int tap = i / kgroups, c0 = (i - tap * kgroups) * kK;
        const int dy = tap / 3 - 1, dx = tap % 3 - 1;
        unsigned char* stage = smem + st * kStage;
        // A: the 16 channels of this pixel at the tap offset, split into three BF16 parts
        {
            const int yy = py + dy, xx = px + dx;
            const bool in_img = live && yy >= 0 && yy < H && xx >= 0 && xx < Wd;
            const int64_t q = (int64_t)yy * Wd + xx;
            uint32_t w0[8], w1[8], w2[8];
#pragma unroll
            for (int c = 0; c < kK; c += 2) {
                float v[2];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int ch = c0 + c + e;
                    v[e] = (in_img && ch < Kc) ? __ldg(inb + (int64_t)ch * HW + q) : 0.f;
                }
                __nv_bfloat16 h[2], m[2], l[2];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    h[e] = __float2bfloat16_rn(v[e]);
                    const float r1 = __fsub_rn(v[e], __bfloat162float(h[e]));
                    m[e] = __float2bfloat16_rn(r1);
                    l[e] = __float2bfloat16_rn(__fsub_rn(r1, __bfloat162float(m[e])));
                }
                w0[c / 2] = pack2(h[0], h[1]);
                w1[c / 2] = pack2(m[0], m[1]);
                w2[c / 2] = pack2(l[0], l[1]);
            }
#pragma unroll
            for (int kq = 0; kq < 2; ++kq) {
                const uint32_t off = kmaj(tid, kq);
                *(uint4*)(stage + 0 * kABytes + off) = make_uint4(w0[4 * kq], w0[4 * kq + 1], w0[4 * kq + 2], w0[4 * kq + 3]);
                *(uint4*)(stage + 1 * kABytes + off) = make_uint4(w1[4 * kq], w1[4 * kq + 1], w1[4 * kq + 2], w1[4 * kq + 3]);
                *(uint4*)(stage + 2 * kABytes + off) = make_uint4(w2[4 * kq], w2[4 * kq + 1], w2[4 * kq + 2], w2[4 * kq + 3]);
            }
        }
        // B: NP rows x 16 channels of weights for this tap (8 channels = 16 bytes per thread and pass)
        for (int t = tid; t < NP * 2; t += kM) {
            const int n = t >> 1, kq = t & 1;
            uint32_t wv[4];
#pragma unroll
            for (int c = 0; c < 8; c += 2) {
                __nv_bfloat16 e2[2];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int ch = c0 + kq * 8 + c + e;
                    __nv_bfloat16 w = __float2bfloat16_rn(0.f);
                    if (n < N && ch < Kc) {
                        if (!TRANSPOSED) w = W[((int64_t)n * Kc + ch) * 9 + tap];
                        else w = W[((int64_t)ch * N + n) * 9 + (8 - tap)];
                    }
                    e2[e] = w;
                }
                wv[c / 2] = pack2(e2[0], e2[1]);
            }
            *(uint4*)(stage + 3 * kABytes + kmaj(n, kq)) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint64_t db = sdesc(smem_u32(stage + 3 * kABytes));
#pragma unroll
            for (int part = 0; part < 3; ++part) {
                const uint64_t da = sdesc(smem_u32(stage + part * kABytes));
                const uint32_t acc = (i > 0 || part > 0) ? 1u : 0u;
                asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                             ::"r"(tmem), "l"(da), "l"(db), "r"(idesc(NP)), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&bars[st])));
        }
    }
    // the last commit covers every MMA this thread issued
    if (ok && nchunks > 0) {   // both stages' last commits, so no arrive is pending at exit
        const int last = nchunks - 1;
        if (!wait_bar(smem_u32(&bars[last & 1]), (uint32_t)((last >> 1) & 1), spin)) failed = 1;
        if (last >= 1 && !wait_bar(smem_u32(&bars[(last - 1) & 1]), (uint32_t)(((last - 1) >> 1) & 1), spin))
            failed = 1;
        __syncthreads();
        ok = !failed;
        if (!ok) {   // drain both stages' last commits before the tensor memory is freed
            wait_bar(smem_u32(&bars[last & 1]), (uint32_t)((last >> 1) & 1));
            if (last >= 1) wait_bar(smem_u32(&bars[(last - 1) & 1]), (uint32_t)(((last - 1) >> 1) & 1));
        }
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok) {
        const int64_t obase = (int64_t)b * N * HW;
#pragma unroll
        for (int n0 = 0; n0 < NP; n0 += 16) {
            uint32_t r[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)n0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            if (live) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int n = n0 + j;
                    if (n < N) {
                        float v = __uint_as_float(r[j]);
                        if (bias) v += bias[n];
                        if (relu) v = fmaxf(v, 0.f);
                        float* dst = out + obase + (int64_t)n * HW + p;
                        *dst = accumulate ? *dst + v : v;
                    }
                }
            }
        }
    } else if (tid == 0) {
        atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols));
}

// dynamic shared memory: two stages, padded so that no more CTAs than the tensor memory
// holds (512 columns per SM) are resident at once
template <int NP>
size_t smem_bytes() {
    constexpr size_t need = 2 * (3 * kM * kK * 2 + NP * kK * 2);
    const size_t per_sm = 228 * 1024, ctas = 512 / tmem_cols(NP);
    const size_t pad = per_sm / ctas + 1;
    return need > pad ? need : pad;
}

template <int NP, bool TRANSPOSED>
int launch_np(const float* in, int Kc, const __nv_bfloat16* W, const float* bias, float* out, int N, int B, int H,
              int Wd, int relu, int accumulate, int* err, long spin, cudaStream_t s) {
    const size_t smem = smem_bytes<NP>();
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(conv3x3_tc_kernel<NP, TRANSPOSED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
            return -1;
        attr = true;
    }
    const int64_t HW = (int64_t)H * Wd;
    dim3 grid((unsigned)((HW + kM - 1) / kM), (unsigned)B);
    conv3x3_tc_kernel<NP, TRANSPOSED><<<grid, kM, smem, s>>>(in, Kc, W, bias, out, N, H, Wd, relu, accumulate, err,
                                                             spin);
    return 0;
}

// Weight gradient on the tensor cores. With r = ci*9 + tap and the pixels P of all
// images as the reduction index, dW[co][r] = sum_P g[co][P] x_r[P], where x_r is input
// channel ci shifted by the tap (zero outside the image). CTA (z, t) accumulates the
// rows of input channels 14 t .. 14 t + 13 (126 rows; rows 126-127 of the M tile stay
// zero) against all NP output channels over the 16-pixel chunks [z cpc, (z+1) cpc):
// A = x (128 rows x 16 pixels, K-major), B = g (NP rows x 16 pixels, K-major). A thread
// gathers the 3 x 3 neighbourhoods of two pixels in one channel (the nine rows of that
// channel), so the index arithmetic is done once per pixel. Both are FP32, split into three BF16 parts (h + m + l, exact); the six part
// products of weight down to 2^-16 are accumulated in FP32 in tensor memory (the three
// dropped ones are below 2^-24 of the product, under the accumulation's own rounding).
// Partial sums go to partial[z][co][r]; wgrad_reduce_kernel adds them in z order.
constexpr int kWgCh = 14;   // input channels per M tile of the weight gradient (126 of 128 rows)

template <int NP>
__global__ void __launch_bounds__(kM) wgrad_tc_kernel(const float* __restrict__ in, int Cin,
                                                      const float* __restrict__ g, int Cout, int B, int H, int Wd,
                                                      int cpc, float* __restrict__ partial, int* err, long spin) {
    constexpr int kABytes = kM * kK * 2;          // one BF16 part of the A chunk
    constexpr int kBBytes = NP * kK * 2;          // one BF16 part of the B chunk
    constexpr int kStage = 3 * kABytes + 3 * kBBytes;
    constexpr uint32_t kCols = tmem_cols(NP);
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ uint32_t tmem_base;
    __shared__ int failed;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int rows = Cin * 9, ci0 = blockIdx.y * kWgCh;
    const int64_t HW = (int64_t)H * Wd, npix = (int64_t)B * HW;
    const int64_t all_chunks = (npix + kK - 1) / kK, c0 = (int64_t)blockIdx.x * cpc;
    const int nchunks = (int)(c0 < all_chunks ? (all_chunks - c0 < cpc ? all_chunks - c0 : cpc) : 0);
    // staging roles: pixels 2 pp and 2 pp + 1 of a chunk (pp = 4 kq + kp4); A: channel
    // ci0 + cl (its nine tap rows cl*9 + tap, threads with cl >= 14 stage none); B: output
    // channels cl + 16 j. The 32 lanes of a warp store to 32 distinct banks (cl*9 = cl mod 8).
    const int kp4 = tid & 3, rg = (tid >> 2) & 7, kq = (tid >> 5) & 1, rhi = tid >> 6;
    const int pp = kq * 4 + kp4, cl = rg + 8 * rhi;
    const bool a_task = cl < kWgCh && ci0 + cl < Cin;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        failed = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (tid < 24) {   // rows 126 and 127 of A: zero in both stages and all three parts
        const int stg = tid / 12, part = (tid / 4) % 3, row = 126 + ((tid >> 1) & 1), k8 = tid & 1;
        *(uint4*)(smem + stg * kStage + part * kABytes + kmaj(row, k8)) = make_uint4(0u, 0u, 0u, 0u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    // the FP32 operands of one chunk, all loads of a chunk in flight together; the next
    // chunk is loaded while the current one's MMAs run
    float va[9][2], vb[NP / 16][2];
    auto load_chunk = [&](int64_t c) {
        int64_t base[2], q[2];
        int py[2], px[2];
        bool live[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int64_t P = c * kK + 2 * pp + e;
            live[e] = P < npix;
            base[e] = live[e] ? P / HW : 0;
            q[e] = live[e] ? P - base[e] * HW : 0;
            py[e] = (int)(q[e] / Wd);
            px[e] = (int)(q[e] - (int64_t)py[e] * Wd);
        }
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const bool on = a_task && live[e];
            const float* src = in + (base[e] * Cin + ci0 + (on ? cl : 0)) * HW + q[e];
            const bool up = py[e] > 0, down = py[e] < H - 1, left = px[e] > 0, right = px[e] < Wd - 1;
#pragma unroll
            for (int tap = 0; tap < 9; ++tap) {
                const int dy = tap / 3 - 1, dx = tap % 3 - 1;
                const bool inb = on && (dy >= 0 || up) && (dy <= 0 || down) && (dx >= 0 || left) && (dx <= 0 || right);
                va[tap][e] = inb ? __ldg(src + dy * Wd + dx) : 0.f;
            }
        }
#pragma unroll
        for (int j = 0; j < NP / 16; ++j) {
            const int co = rg + 8 * rhi + 16 * j;
#pragma unroll
            for (int e = 0; e < 2; ++e)
                vb[j][e] = (co < Cout && live[e]) ? __ldg(g + (base[e] * Cout + co) * HW + q[e]) : 0.f;
        }
    };
    if (nchunks > 0) load_chunk(c0);
    bool ok = true;
    for (int i = 0; i < nchunks && ok; ++i) {
        const int st = i & 1;
        if (i >= 2) {   // the MMAs that read this stage (chunk i - 2) are done
            if (!wait_bar(smem_u32(&bars[st]), (uint32_t)(((i >> 1) - 1) & 1), spin)) failed = 1;
            __syncthreads();
            if (failed) {   // drain: the MMAs of chunks i - 2 and i - 1 are still in flight
                wait_bar(smem_u32(&bars[st]), (uint32_t)(((i >> 1) - 1) & 1));
                wait_bar(smem_u32(&bars[st ^ 1]), (uint32_t)(((i - 1) >> 1) & 1));
                ok = false;
                break;
            }
        }
        unsigned char* stage = smem + st * kStage;
        // A: the nine tap rows of channel ci0 + cl at the two pixels
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            if (cl >= kWgCh) break;
            const int rl = cl * 9 + tap;
            __nv_bfloat16 h[2], m[2], l[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) split3(va[tap][e], h[e], m[e], l[e]);
            const uint32_t off = kmaj(rl, kq) + kp4 * 4;
            *(uint32_t*)(stage + 0 * kABytes + off) = pack2(h[0], h[1]);
            *(uint32_t*)(stage + 1 * kABytes + off) = pack2(m[0], m[1]);
            *(uint32_t*)(stage + 2 * kABytes + off) = pack2(l[0], l[1]);
        }
        // B: the output gradients of channels rg + 8 rhi + 16 j at the two pixels
#pragma unroll
        for (int j = 0; j < NP / 16; ++j) {
            const int co = rg + 8 * rhi + 16 * j;
            __nv_bfloat16 h[2], m[2], l[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) split3(vb[j][e], h[e], m[e], l[e]);
            const uint32_t off = kmaj(co, kq) + kp4 * 4;
            unsigned char* bs = stage + 3 * kABytes;
            *(uint32_t*)(bs + 0 * kBBytes + off) = pack2(h[0], h[1]);
            *(uint32_t*)(bs + 1 * kBBytes + off) = pack2(m[0], m[1]);
            *(uint32_t*)(bs + 2 * kBBytes + off) = pack2(l[0], l[1]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            // part pairs (A, B): hh, hm, mh, mm, hl, lh
            const int pa[6] = {0, 0, 1, 1, 0, 2}, pb[6] = {0, 1, 0, 1, 2, 0};
#pragma unroll
            for (int t = 0; t < 6; ++t) {
                const uint64_t da = sdesc(smem_u32(stage + pa[t] * kABytes));
                const uint64_t db = sdesc(smem_u32(stage + 3 * kABytes + pb[t] * kBBytes));
                const uint32_t acc = (i > 0 || t > 0) ? 1u : 0u;
                asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                             ::"r"(tmem), "l"(da), "l"(db), "r"(idesc(NP)), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&bars[st])));
        }
        if (i + 1 < nchunks) load_chunk(c0 + i + 1);   // in flight while the MMAs run
    }
    if (ok && nchunks > 0) {   // both stages' last commits, so no arrive is pending at exit
        const int last = nchunks - 1;
        if (!wait_bar(smem_u32(&bars[last & 1]), (uint32_t)((last >> 1) & 1), spin)) failed = 1;
        if (last >= 1 && !wait_bar(smem_u32(&bars[(last - 1) & 1]), (uint32_t)(((last - 1) >> 1) & 1), spin))
            failed = 1;
        __syncthreads();
        ok = !failed;
        if (!ok) {   // drain both stages' last commits before the tensor memory is freed
            wait_bar(smem_u32(&bars[last & 1]), (uint32_t)((last >> 1) & 1));
            if (last >= 1) wait_bar(smem_u32(&bars[(last - 1) & 1]), (uint32_t)(((last - 1) >> 1) & 1));
        }
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok) {
        // this thread's TMEM lane is row tid of the tile: channel ci0 + tid / 9
        const int r = (tid < kWgCh * 9 && ci0 + tid / 9 < Cin) ? ci0 * 9 + tid : rows;
#pragma unroll
        for (int n0 = 0; n0 < NP; n0 += 16) {
            uint32_t v[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)n0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            if (r < rows) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int co = n0 + j;
                    if (co < Cout)
                        partial[((int64_t)blockIdx.x * Cout + co) * rows + r] = nchunks > 0 ? __uint_as_float(v[j]) : 0.f;
                }
            }
        }
    } else if (tid == 0) {
        atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols));
}

// Grid of the tensor-core weight gradient: z ranges of at least 8 chunks of 16 pixels,
// about 1200 CTAs over the M tiles (up to 8 resident per SM), partials of at most 2^23 floats
struct WgradTcShape {
    int z, cpc, mtiles;
};

inline WgradTcShape wgrad_tc_shape(int Cin, int Cout, int64_t npix) {
    WgradTcShape w;
    w.mtiles = (Cin + kWgCh - 1) / kWgCh;
    const int64_t chunks = (npix + kK - 1) / kK;
    int64_t z = (1200 + w.mtiles - 1) / w.mtiles;
    const int64_t zcap = ((int64_t)1 << 23) / ((int64_t)Cout * Cin * 9);
    z = z < zcap ? z : zcap;
    const int64_t zmax = (chunks + 7) / 8;
    z = z < zmax ? z : zmax;
    z = z < 1 ? 1 : z;
    w.cpc = (int)((chunks + z - 1) / z);
    w.z = (int)((chunks + w.cpc - 1) / w.cpc);
    return w;
}

template <int NP>
size_t wgrad_smem_bytes() {
    constexpr size_t need = 2 * (3 * kM * kK * 2 + 3 * NP * kK * 2);
    const size_t per_sm = 228 * 1024, ctas = 512 / tmem_cols(NP);
    const size_t pad = per_sm / ctas + 1;
    return need > pad ? need : pad;
}

template <int NP>
int launch_wgrad_np(const float* in, int Cin, const float* g, int Cout, int B, int H, int Wd, float* partial, int* nz,
                    int* err, long spin, cudaStream_t s) {
    const size_t smem = wgrad_smem_bytes<NP>();
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(wgrad_tc_kernel<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return -1;
        attr = true;
    }
    const WgradTcShape w = wgrad_tc_shape(Cin, Cout, (int64_t)B * H * Wd);
    wgrad_tc_kernel<NP><<<dim3((unsigned)w.z, (unsigned)w.mtiles), kM, smem, s>>>(in, Cin, g, Cout, B, H, Wd, w.cpc,
                                                                                   partial, err, spin);
    *nz = w.z;
    return 0;
}

// partial[z][co][ci*9 + tap] for z < *nz (Cout up to 64); -1: not handled here
int wgrad(const float* in, int Cin, const float* g, int Cout, int B, int H, int Wd, float* partial, int* nz, int* err,
          long spin, cudaStream_t s) {
    if (Cout <= 16) return launch_wgrad_np<16>(in, Cin, g, Cout, B, H, Wd, partial, nz, err, spin, s);
    if (Cout <= 32) return launch_wgrad_np<32>(in, Cin, g, Cout, B, H, Wd, partial, nz, err, spin, s);
    if (Cout <= 64) return launch_wgrad_np<64>(in, Cin, g, Cout, B, H, Wd, partial, nz, err, spin, s);
    return -1;
}

// out (N channels) = conv3x3(in (Kc channels)); N up to 128. spin: polls per bounded wait
// before it counts as timed out (kSpin normally; a test lowers it to exercise the path)
template <bool TRANSPOSED>
int conv3x3(const float* in, int Kc, const __nv_bfloat16* W, const float* bias, float* out, int N, int B, int H, int Wd,
            int relu, int accumulate, int* err, long spin, cudaStream_t s) {
    if (N <= 16) return launch_np<16, TRANSPOSED>(in, Kc, W, bias, out, N, B, H, Wd, relu, accumulate, err, spin, s);
    if (N <= 32) return launch_np<32, TRANSPOSED>(in, Kc, W, bias, out, N, B, H, Wd, relu, accumulate, err, spin, s);
    if (N <= 48) return launch_np<48, TRANSPOSED>(in, Kc, W, bias, out, N, B, H, Wd, relu, accumulate, err, spin, s);
    if (N <= 64) return launch_np<64, TRANSPOSED>(in, Kc, W, bias, out, N, B, H, Wd, relu, accumulate, err, spin, s);
    if (N <= 96) return launch_np<96, TRANSPOSED>(in, Kc, W, bias, out, N, B, H, Wd, relu, accumulate, err, spin, s);
    if (N <= 128) return launch_np<128, TRANSPOSED>(in, Kc, W, bias, out, N, B, H, Wd, relu, accumulate, err, spin, s);
    return -1;
}

}  // namespace tc

// Weight gradient, tiled: dW[co][ci][k] = sum_{b,y,x} g[b,co,y,x] in[b,ci,y+ky-1,x+kx-1].
// A CTA owns 16 output x 16 input channels (one thread per (co, ci) pair, 9 taps in
// registers) and one chunk of rows of one image; bands of kWgRows rows of g and of the
// input (with a zero halo) are staged in shared memory, the input rows padded so the 16
// channels of a warp fall in distinct banks. Each CTA writes its 16 x 16 x 9 partial sums;
// wgrad_reduce_kernel adds the partials of all chunks in chunk order (deterministic).
constexpr int kWgRows = 2;

struct WgradShape {
    int rows_per_chunk, chunks_per_image;
    int in_stride, g_stride;   // floats per staged input / gradient channel
    size_t smem;
};

// other_ctas: the CTAs of the grid's channel dimensions times the batch; the row chunks
// are chosen so the grid has about 600 CTAs (a wave at 4 CTAs per SM)
inline WgradShape wgrad_shape(int H, int Wd, int other_ctas) {
    WgradShape w;
    const int max_chunks = (H + kWgRows - 1) / kWgRows;
    int chunks = (600 + other_ctas - 1) / (other_ctas > 0 ? other_ctas : 1);
    chunks = chunks < 1 ? 1 : (chunks > max_chunks ? max_chunks : chunks);
    int rows = (H + chunks - 1) / chunks;
    rows = (rows + kWgRows - 1) / kWgRows * kWgRows;
    w.rows_per_chunk = rows < H ? rows : H;
    w.chunks_per_image = (H + w.rows_per_chunk - 1) / w.rows_per_chunk;
    int st = (kWgRows + 2) * (Wd + 2);
    st += ((1 - st) % 32 + 32) % 32;   // stride = 1 (mod 32): a warp's 16 input channels in 16 banks
    w.in_stride = st;
    w.g_stride = kWgRows * Wd + 1;     // odd: the warp's two output channels in different banks
    w.smem = sizeof(float) * (16 * (size_t)st + 16 * (size_t)w.g_stride);
    return w;
}

__global__ void __launch_bounds__(kT) conv3x3_wgrad_tiled_kernel(const float* __restrict__ in, int Cin,
                                                                 const float* __restrict__ g, int Cout, int H, int Wd,
                                                                 int rows_per_chunk, int chunks_per_image,
                                                                 int in_stride, int g_stride,
                                                                 float* __restrict__ partial) {
    extern __shared__ float wsm_dyn[];
    float* in_s = wsm_dyn;                          // [16][in_stride]
    float* g_s = wsm_dyn + 16 * in_stride;          // [16][g_stride], kWgRows * Wd used
    const int co0 = blockIdx.x * 16, ci0 = blockIdx.y * 16;
    const int b = blockIdx.z / chunks_per_image, ch = blockIdx.z - b * chunks_per_image;
    const int y0 = ch * rows_per_chunk, y1 = min(H, y0 + rows_per_chunk);
    const int col = threadIdx.x / 16, cil = threadIdx.x % 16;
    const int64_t plane = (int64_t)H * Wd;
    const int W2 = Wd + 2;
    float acc[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[k] = 0.f;
    for (int yb = y0; yb < y1; yb += kWgRows) {
        const int nr = min(kWgRows, y1 - yb);
        // input rows yb-1 .. yb+kWgRows with a zero halo column on each side
        for (int t = threadIdx.x; t < 16 * (kWgRows + 2) * W2; t += kT) {
            const int c = t / ((kWgRows + 2) * W2), rem = t - c * (kWgRows + 2) * W2;
            const int r = rem / W2, xx = rem - r * W2 - 1, yy = yb - 1 + r;
            float v = 0.f;
            if (ci0 + c < Cin && yy >= 0 && yy < H && yy <= yb + nr && xx >= 0 && xx < Wd)
                v = in[((int64_t)b * Cin + ci0 + c) * plane + (int64_t)yy * Wd + xx];
            in_s[c * in_stride + rem] = v;
        }
        for (int t = threadIdx.x; t < 16 * kWgRows * Wd; t += kT) {
            const int c = t / (kWgRows * Wd), rem = t - c * kWgRows * Wd;
            const int r = rem / Wd;
            g_s[c * g_stride + rem] = (co0 + c < Cout && r < nr)
                                          ? g[((int64_t)b * Cout + co0 + c) * plane + (int64_t)(yb + r) * Wd + (rem - r * Wd)]
                                          : 0.f;
        }
        __syncthreads();
        const float* gr = g_s + col * g_stride;
        const float* ir = in_s + cil * in_stride;
        for (int r = 0; r < nr; ++r)
            for (int x = 0; x < Wd; ++x) {
                const float gv = gr[r * Wd + x];
                const float* base = ir + r * W2 + x;
#pragma unroll
                for (int k = 0; k < 9; ++k) acc[k] = fmaf(gv, base[(k / 3) * W2 + k % 3], acc[k]);
            }
        __syncthreads();
    }
    const int co = co0 + col, ci = ci0 + cil;
    if (co < Cout && ci < Cin) {
        float* dst = partial + (((int64_t)blockIdx.z * Cout + co) * Cin + ci) * 9;
#pragma unroll
        for (int k = 0; k < 9; ++k) dst[k] = acc[k];
    }
}

// dW[w] = sum_z partial[z][w], z in order
__global__ void wgrad_reduce_kernel(const float* __restrict__ partial, int nz, int64_t nw, float* __restrict__ dW) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += stride) {
        float t = 0.f;
        for (int z = 0; z < nz; ++z) t += partial[(int64_t)z * nw + w];
        dW[w] = t;
    }
}

// db[c] = sum_{b,y,x} g[b,c,y,x]   (one CTA per channel)
// Channel sums over pixels in chunks: CTA (c, z) sums chunk z (kRedChunk pixels of one
// image) of channel c into partial[z][c]; wgrad_reduce_kernel adds the chunks in order.
// Bias gradient: v = g[b][c][p]. 1x1 weight gradient (one output channel): v =
// g[b][0][p] in[b][c][p].
constexpr int kRedChunk = 4096;

__global__ void __launch_bounds__(kT) chan_sum_partial_kernel(const float* __restrict__ g, const float* __restrict__ in,
                                                              int C, int64_t plane, int chunks,
                                                              float* __restrict__ partial) {
    const int c = blockIdx.x, z = blockIdx.y, b = z / chunks, piece = z - b * chunks;
    const int64_t p0 = (int64_t)piece * kRedChunk, p1 = min(plane, p0 + kRedChunk);
    float t = 0.f;
    if (in) {
        const float* gp = g + (int64_t)b * plane;
        const float* ip = in + ((int64_t)b * C + c) * plane;
        for (int64_t p = p0 + threadIdx.x; p < p1; p += kT) t = fmaf(gp[p], ip[p], t);
    } else {
        const float* gp = g + ((int64_t)b * C + c) * plane;
        for (int64_t p = p0 + threadIdx.x; p < p1; p += kT) t += gp[p];
    }
    __shared__ float red[kT / 32];
    for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        float sum = 0.f;
        for (int w = 0; w < kT / 32; ++w) sum += red[w];
        partial[(int64_t)z * C + c] = sum;
    }
}

// 1x1 convolution C -> 1: out = sum_c W[c] in[c] + b
template <typename WT>
__global__ void conv1x1_fwd_kernel(const float* __restrict__ in, int C, const WT* __restrict__ W,
                                   const float* __restrict__ bias, float* __restrict__ out, int B, int64_t plane) {
    for (int64_t p = blockIdx.x * (int64_t)kT + threadIdx.x; p < (int64_t)B * plane; p += (int64_t)gridDim.x * kT) {
        const int b = (int)(p / plane);
        const int64_t r = p - (int64_t)b * plane;
        float acc = bias[0];
        for (int c = 0; c < C; ++c) acc = fmaf(wload(W, c), in[((int64_t)b * C + c) * plane + r], acc);
        out[p] = acc;
    }
}

// backward of the 1x1 layer: dIn[c] = W[c] g
template <typename WT>
__global__ void conv1x1_dgrad_kernel(const float* __restrict__ g, int C, const WT* __restrict__ W,
                                     float* __restrict__ din, int B, int64_t plane) {
    for (int64_t p = blockIdx.x * (int64_t)kT + threadIdx.x; p < (int64_t)B * plane; p += (int64_t)gridDim.x * kT) {
        const int b = (int)(p / plane);
        const int64_t r = p - (int64_t)b * plane;
        for (int c = 0; c < C; ++c) din[((int64_t)b * C + c) * plane + r] = wload(W, c) * g[p];
    }
}

// dW[c] = sum g * in[c]   (one CTA per c)

// g *= (y > 0): the ReLU of the layer that produced y
__global__ void relu_mask_kernel(float* __restrict__ g, const float* __restrict__ y, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT)
        if (!(y[i] > 0.f)) g[i] = 0.f;
}

// 2x2 average pooling of channels [0, C) of `in` (C_in_total channels) into out (C channels)
__global__ void pool_fwd_kernel(const float* __restrict__ in, float* __restrict__ out, int BC, int H, int Wd) {
    const int Ho = H / 2, Wo = Wd / 2;
    for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < (int64_t)BC * Ho * Wo; i += (int64_t)gridDim.x * kT) {
        const int64_t bc = i / ((int64_t)Ho * Wo);
        const int64_t r = i - bc * Ho * Wo;
        const int y = (int)(r / Wo), x = (int)(r % Wo);
        const float* s = in + bc * H * Wd + (int64_t)(2 * y) * Wd + 2 * x;
        out[i] = 0.25f * (s[0] + s[1] + s[Wd] + s[Wd + 1]);
    }
}

// dIn[2y+a][2x+b] = 0.25 dOut[y][x]
__global__ void pool_bwd_kernel(const float* __restrict__ gout, float* __restrict__ gin, int BC, int H, int Wd,
                                int accumulate) {
    for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < (int64_t)BC * H * Wd; i += (int64_t)gridDim.x * kT) {
        const int64_t bc = i / ((int64_t)H * Wd);
        const int64_t r = i - bc * H * Wd;
        const int y = (int)(r / Wd), x = (int)(r % Wd);
        const float v = 0.25f * gout[bc * (H / 2) * (Wd / 2) + (int64_t)(y / 2) * (Wd / 2) + x / 2];
        gin[i] = accumulate ? gin[i] + v : v;
    }
}

// nearest 2x upsampling of src (B, C, H/2, W/2) into channels [0, C) of dst (B, Ctot, H, W)
__global__ void up_fwd_kernel(const float* __restrict__ src, float* __restrict__ dst, int B, int C, int Ctot, int H,
                              int Wd) {
    const int64_t plane = (int64_t)H * Wd;
    for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < (int64_t)B * C * plane; i += (int64_t)gridDim.x * kT) {
        const int64_t bc = i / plane;
        const int b = (int)(bc / C), c = (int)(bc % C);
        const int64_t r = i - bc * plane;
        const int y = (int)(r / Wd), x = (int)(r % Wd);
        dst[((int64_t)b * Ctot + c) * plane + r] = src[bc * (plane / 4) + (int64_t)(y / 2) * (Wd / 2) + x / 2];
    }
}

// backward of up_fwd: gsrc[y][x] = sum of the 2x2 block of channels [0, C) of gdst
__global__ void up_bwd_kernel(const float* __restrict__ gdst, float* __restrict__ gsrc, int B, int C, int Ctot, int H,
                              int Wd) {
    const int Ho = H / 2, Wo = Wd / 2;
    const int64_t plane = (int64_t)H * Wd;
    for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < (int64_t)B * C * Ho * Wo; i += (int64_t)gridDim.x * kT) {
        const int64_t bc = i / ((int64_t)Ho * Wo);
        const int b = (int)(bc / C), c = (int)(bc % C);
        const int64_t r = i - bc * Ho * Wo;
        const int y = (int)(r / Wo), x = (int)(r % Wo);
        const float* s = gdst + ((int64_t)b * Ctot + c) * plane + (int64_t)(2 * y) * Wd + 2 * x;
        gsrc[i] = s[0] + s[1] + s[Wd] + s[Wd + 1];
    }
}

// copy channels: dst[b, c0 + c] = src[b, c] (or the reverse with `gather`), accumulate optional
__global__ void chan_copy_kernel(const float* __restrict__ src, int Cs, int s0, float* __restrict__ dst, int Cd,
                                 int d0, int C, int B, int64_t plane, int accumulate) {
    for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < (int64_t)B * C * plane; i += (int64_t)gridDim.x * kT) {
        const int64_t bc = i / plane;
        const int b = (int)(bc / C), c = (int)(bc % C);
        const int64_t r = i - bc * plane;
        const float v = src[((int64_t)b * Cs + s0 + c) * plane + r];
        float* d = dst + ((int64_t)b * Cd + d0 + c) * plane + r;
        *d = accumulate ? *d + v : v;
    }
}

// loss = mean (out - t)^2 per batch: per-CTA partials, then one CTA sums them in order;
// g = 2 (out - t) / N
__global__ void mse_kernel(const float* __restrict__ out, const float* __restrict__ t, float* __restrict__ g, int64_t n,
                           float* __restrict__ partial) {
    float s = 0.f;
    const float inv = 1.f / (float)n;
    for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) {
        const float d = out[i] - t[i];
        s = fmaf(d, d, s);
        if (g) g[i] = 2.f * d * inv;
    }
    __shared__ float red[kT / 32];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float a = 0.f;
        for (int w = 0; w < kT / 32; ++w) a += red[w];
        partial[blockIdx.x] = a * inv;
    }
}

// Residual term of the loss for the convection-diffusion operator the features encode:
// channel 0 = f / s_f, channel 1 = beta / 20; row p of A (h^2-scaled, h = 1/(H+1)) is
// 4 u_p + sum_d [(-1 - c_p) u_{p-e_d} + (-1 + c_p) u_{p+e_d}], c_p = 20 beta_hat_p h / 2.
// r = kappa (A out) - f_hat (the output is the solution divided by kappa s_f), and per-CTA
// partial sums of r^2 / n.
__global__ void resid_kernel(const float* __restrict__ out, const float* __restrict__ feat, float* __restrict__ r,
                             int B, int H, int Wd, float h, float kappa, float* __restrict__ partial) {
    const int64_t plane = (int64_t)H * Wd, n = (int64_t)B * plane;
    const float inv = 1.f / (float)n;
    float s = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) {
        const int b = (int)(i / plane);
        const int64_t q = i - (int64_t)b * plane;
        const int y = (int)(q / Wd), x = (int)(q % Wd);
        const float* u = out + (int64_t)b * plane;
        const float c = 20.f * feat[((int64_t)b * 2 + 1) * plane + q] * h * 0.5f;
        float a = 4.f * u[q];
        if (x > 0) a = fmaf(-1.f - c, u[q - 1], a);
        if (x < Wd - 1) a = fmaf(-1.f + c, u[q + 1], a);
        if (y > 0) a = fmaf(-1.f - c, u[q - Wd], a);
        if (y < H - 1) a = fmaf(-1.f + c, u[q + Wd], a);
        const float ri = kappa * a - feat[((int64_t)b * 2) * plane + q];
        r[i] = ri;
        s = fmaf(ri, ri, s);
    }
    __shared__ float red[kT / 32];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float a = 0.f;
        for (int w = 0; w < kT / 32; ++w) a += red[w];
        partial[blockIdx.x] = a * inv;
    }
}

// g += scale * A^T r, (A^T r)_p = 4 r_p + sum_d [(-1 - c_{p+e_d}) r_{p+e_d} + (-1 + c_{p-e_d}) r_{p-e_d}]
__global__ void resid_grad_kernel(const float* __restrict__ r, const float* __restrict__ feat, float* __restrict__ g,
                                  int B, int H, int Wd, float h, float scale) {
    const int64_t plane = (int64_t)H * Wd, n = (int64_t)B * plane;
    for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) {
        const int b = (int)(i / plane);
        const int64_t q = i - (int64_t)b * plane;
        const int y = (int)(q / Wd), x = (int)(q % Wd);
        const float* rr = r + (int64_t)b * plane;
        const float* bh = feat + ((int64_t)b * 2 + 1) * plane;
        const float k = 20.f * h * 0.5f;
        float a = 4.f * rr[q];
        if (x < Wd - 1) a = fmaf(-1.f - k * bh[q + 1], rr[q + 1], a);
        if (x > 0) a = fmaf(-1.f + k * bh[q - 1], rr[q - 1], a);
        if (y < H - 1) a = fmaf(-1.f - k * bh[q + Wd], rr[q + Wd], a);
        if (y > 0) a = fmaf(-1.f + k * bh[q - Wd], rr[q - Wd], a);
        g[i] = fmaf(scale, a, g[i]);
    }
}

__global__ void sum_partials_kernel(const float* __restrict__ partial, int n, float* __restrict__ out) {
    if (threadIdx.x == 0) {
        float a = 0.f;
        for (int i = 0; i < n; ++i) a += partial[i];
        *out = a;
    }
}

// loss[0] = mse + w * residual term
__global__ void combine_loss_kernel(float* loss, float w) {
    if (threadIdx.x == 0) loss[0] = loss[0] + w * loss[1];
}

// Adam (Kingma & Ba 2015) on the FP32 master weights, then the BF16 copy
__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, __nv_bfloat16* __restrict__ wb, int64_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        wb[i] = __float2bfloat16_rn(wi);
    }
}

__global__ void to_bf16_kernel(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT)
        wb[i] = __float2bfloat16_rn(w[i]);
}

inline int blocks_for(int64_t n) {
    int64_t b = (n + kT - 1) / kT;
    return (int)(b < 16 * sstep::device_sms() ? (b < 1 ? 1 : b) : 16 * sstep::device_sms());
}

// ------------------------------------------------------------------ the network
struct Net {
    int H = 0, W = 0, Bmax = 0, bf16 = 1, smooth = 0;
    float res_w = 0.f, kappa = 1.f;
    float* r = nullptr;
    float *out_raw = nullptr, *tmp = nullptr, *blur = nullptr;
    int64_t nparams = 0;
    int64_t off[kNumLayers] = {0};
    float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16* wb = nullptr;
    int64_t step = 0;
    // activations and their gradients (B x C x H x W at the level's size)
    std::vector<float*> bufs;
    float *x_in, *a1, *e1, *p1, *a2, *e2, *p2, *a3, *e3, *p3, *ab, *bt, *u3, *a4, *d3, *u2, *a5, *d2, *u1, *a6, *d1, *out;
    float *g_a1, *g_e1, *g_p1, *g_a2, *g_e2, *g_p2, *g_a3, *g_e3, *g_p3, *g_ab, *g_bt, *g_u3, *g_a4, *g_d3, *g_u2, *g_a5,
        *g_d2, *g_u1, *g_a6, *g_d1, *g_out, *g_in;
    float* partial = nullptr;
    float* loss = nullptr;
    int tc = 1;            // BF16 mode: 3x3 convolutions on the tensor cores (tcgen05)
    float* wpart = nullptr;   // weight-gradient partial sums (chunks x weights of a layer)
    int* err = nullptr;    // set by a tensor-core kernel whose bounded wait ran out
    long spin = tc::kSpin; // polls per bounded wait
};

float* alloc(Net& n, int64_t count) {
    float* p = nullptr;
    if (cudaMalloc((void**)&p, sizeof(float) * (count > 0 ? count : 1)) != cudaSuccess) return nullptr;
    n.bufs.push_back(p);
    return p;
}

template <typename WT>
void conv(const Net& n, int layer, const float* in, float* out, int B, int H, int Wd, const WT* Wbase, cudaStream_t s) {
    const ConvSpec& c = kLayers[layer];
    const WT* W = Wbase + n.off[layer];
    const float* bias = n.w + n.off[layer] + (int64_t)c.cout * c.cin * c.k * c.k;
    if (c.k == 1) {
        conv1x1_fwd_kernel<WT><<<blocks_for((int64_t)B * H * Wd), kT, 0, s>>>(in, c.cin, W, bias, out, B, (int64_t)H * Wd);
        return;
    }
    if constexpr (std::is_same<WT, __nv_bfloat16>::value) {
        if (n.tc && tc::conv3x3<false>(in, c.cin, W, bias, out, c.cout, B, H, Wd, c.relu, 0, n.err, n.spin, s) == 0)
            return;
    }
    dim3 grid((Wd + 15) / 16, (H + 15) / 16, B * ((c.cout + 15) / 16));
    conv3x3_kernel<WT, false><<<grid, kT, 0, s>>>(in, c.cin, W, bias, out, c.cout, H, Wd, c.relu, 0);
}

// gradient of one conv layer: g (of its output, ReLU mask already applied) -> dW, db, and dIn (if din)
template <typename WT>
void conv_back(const Net& n, int layer, const float* in, const float* g, float* din, int B, int H, int Wd,
               const WT* Wbase, cudaStream_t s) {
    const ConvSpec& c = kLayers[layer];
    const WT* W = Wbase + n.off[layer];
    float* dW = n.g + n.off[layer];
    float* db = dW + (int64_t)c.cout * c.cin * c.k * c.k;
    const int64_t plane = (int64_t)H * Wd;
    if (c.k == 1) {
        const int chunks = (int)((plane + kRedChunk - 1) / kRedChunk), nz = B * chunks;
        chan_sum_partial_kernel<<<dim3(c.cin, nz), kT, 0, s>>>(g, in, c.cin, plane, chunks, n.wpart);
        wgrad_reduce_kernel<<<blocks_for(c.cin), kT, 0, s>>>(n.wpart, nz, c.cin, dW);
        chan_sum_partial_kernel<<<dim3(1, nz), kT, 0, s>>>(g, nullptr, 1, plane, chunks, n.wpart);
        wgrad_reduce_kernel<<<1, kT, 0, s>>>(n.wpart, nz, 1, db);
        if (din) conv1x1_dgrad_kernel<WT><<<blocks_for(B * plane), kT, 0, s>>>(g, c.cin, W, din, B, plane);
        return;
    }
    bool wdone = false;
    if constexpr (std::is_same<WT, __nv_bfloat16>::value) {
        int nz = 0;
        if (n.tc && tc::wgrad(in, c.cin, g, c.cout, B, H, Wd, n.wpart, &nz, n.err, n.spin, s) == 0) {
            const int64_t nw = (int64_t)c.cout * c.cin * 9;
            wgrad_reduce_kernel<<<blocks_for(nw), kT, 0, s>>>(n.wpart, nz, nw, dW);
            wdone = true;
        }
    }
    if (!wdone) {
        const int cog = (c.cout + 15) / 16, cig = (c.cin + 15) / 16;
        const WgradShape ws = wgrad_shape(H, Wd, cog * cig * B);
        const int nz = B * ws.chunks_per_image;
        dim3 grid(cog, cig, nz);
        static size_t smem_set = 48 * 1024;
        if (ws.smem > smem_set) {
            if (cudaFuncSetAttribute(conv3x3_wgrad_tiled_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)ws.smem) == cudaSuccess)
                smem_set = ws.smem;
        }
        conv3x3_wgrad_tiled_kernel<<<grid, kT, ws.smem, s>>>(in, c.cin, g, c.cout, H, Wd, ws.rows_per_chunk,
                                                             ws.chunks_per_image, ws.in_stride, ws.g_stride, n.wpart);
        const int64_t nw = (int64_t)c.cout * c.cin * 9;
        wgrad_reduce_kernel<<<blocks_for(nw), kT, 0, s>>>(n.wpart, nz, nw, dW);
    }
    {
        const int chunks = (int)((plane + kRedChunk - 1) / kRedChunk), nz = B * chunks;
        chan_sum_partial_kernel<<<dim3(c.cout, nz), kT, 0, s>>>(g, nullptr, c.cout, plane, chunks, n.wpart);
        wgrad_reduce_kernel<<<blocks_for(c.cout), kT, 0, s>>>(n.wpart, nz, c.cout, db);
    }
    if (din) {
        if constexpr (std::is_same<WT, __nv_bfloat16>::value) {
            if (n.tc && tc::conv3x3<true>(g, c.cout, W, nullptr, din, c.cin, B, H, Wd, 0, 0, n.err, n.spin, s) == 0)
                return;
        }
        dim3 grid((Wd + 15) / 16, (H + 15) / 16, B * ((c.cin + 15) / 16));
        conv3x3_kernel<WT, true><<<grid, kT, 0, s>>>(g, c.cout, W, nullptr, din, c.cin, H, Wd, 0, 0);
    }
}

// k passes of the symmetric blur: src -> dst (src is left unchanged); the filter is its
// own adjoint, so the backward pass uses the same routine
void smooth_passes(Net& n, const float* src, float* dst, int B, cudaStream_t s) {
    if (!n.smooth) return;
    dim3 grid((n.W + 15) / 16, (n.H + 15) / 16, B);
    const float* cur = src;
    for (int k = 0; k < n.smooth; ++k) {
        // alternate so that the last pass lands in dst: passes k with (smooth-1-k) even write dst
        float* o = ((n.smooth - 1 - k) % 2 == 0) ? dst : n.tmp;
        conv3x3_kernel<float, false><<<grid, kT, 0, s>>>(cur, 1, n.blur, nullptr, o, 1, n.H, n.W, 0, 0);
        cur = o;
    }
}

template <typename WT>
void forward(Net& n, const float* x, int B, cudaStream_t s) {
    const WT* Wt = (const WT*)(n.bf16 ? (const void*)n.wb : (const void*)n.w);
    const int H = n.H, W = n.W, H2 = H / 2, W2 = W / 2, H4 = H / 4, W4 = W / 4, H8 = H / 8, W8 = W / 8;
    conv<WT>(n, 0, x, n.a1, B, H, W, Wt, s);
    conv<WT>(n, 1, n.a1, n.e1, B, H, W, Wt, s);
    pool_fwd_kernel<<<blocks_for((int64_t)B * 16 * H2 * W2), kT, 0, s>>>(n.e1, n.p1, B * 16, H, W);
    conv<WT>(n, 2, n.p1, n.a2, B, H2, W2, Wt, s);
    conv<WT>(n, 3, n.a2, n.e2, B, H2, W2, Wt, s);
    pool_fwd_kernel<<<blocks_for((int64_t)B * 32 * H4 * W4), kT, 0, s>>>(n.e2, n.p2, B * 32, H2, W2);
    conv<WT>(n, 4, n.p2, n.a3, B, H4, W4, Wt, s);
    conv<WT>(n, 5, n.a3, n.e3, B, H4, W4, Wt, s);
    pool_fwd_kernel<<<blocks_for((int64_t)B * 64 * H8 * W8), kT, 0, s>>>(n.e3, n.p3, B * 64, H4, W4);
    conv<WT>(n, 6, n.p3, n.ab, B, H8, W8, Wt, s);
    conv<WT>(n, 7, n.ab, n.bt, B, H8, W8, Wt, s);
    up_fwd_kernel<<<blocks_for((int64_t)B * 64 * H4 * W4), kT, 0, s>>>(n.bt, n.u3, B, 64, 128, H4, W4);
    chan_copy_kernel<<<blocks_for((int64_t)B * 64 * H4 * W4), kT, 0, s>>>(n.e3, 64, 0, n.u3, 128, 64, 64, B,
                                                                           (int64_t)H4 * W4, 0);
    conv<WT>(n, 8, n.u3, n.a4, B, H4, W4, Wt, s);
    conv<WT>(n, 9, n.a4, n.d3, B, H4, W4, Wt, s);
    up_fwd_kernel<<<blocks_for((int64_t)B * 64 * H2 * W2), kT, 0, s>>>(n.d3, n.u2, B, 64, 96, H2, W2);
    chan_copy_kernel<<<blocks_for((int64_t)B * 32 * H2 * W2), kT, 0, s>>>(n.e2, 32, 0, n.u2, 96, 64, 32, B,
                                                                           (int64_t)H2 * W2, 0);
    conv<WT>(n, 10, n.u2, n.a5, B, H2, W2, Wt, s);
    conv<WT>(n, 11, n.a5, n.d2, B, H2, W2, Wt, s);
    up_fwd_kernel<<<blocks_for((int64_t)B * 32 * H * W), kT, 0, s>>>(n.d2, n.u1, B, 32, 48, H, W);
    chan_copy_kernel<<<blocks_for((int64_t)B * 16 * H * W), kT, 0, s>>>(n.e1, 16, 0, n.u1, 48, 32, 16, B,
                                                                         (int64_t)H * W, 0);
    conv<WT>(n, 12, n.u1, n.a6, B, H, W, Wt, s);
    conv<WT>(n, 13, n.a6, n.d1, B, H, W, Wt, s);
    conv<WT>(n, 14, n.d1, n.smooth ? n.out_raw : n.out, B, H, W, Wt, s);
    smooth_passes(n, n.out_raw, n.out, B, s);
}

void mask(float* g, const float* y, int64_t cnt, cudaStream_t s) {
    relu_mask_kernel<<<blocks_for(cnt), kT, 0, s>>>(g, y, cnt);
}

// backward from g_out (d loss / d out) to every parameter gradient
template <typename WT>
void backward(Net& n, const float* x, int B, cudaStream_t s) {
    const WT* Wt = (const WT*)(n.bf16 ? (const void*)n.wb : (const void*)n.w);
    const int H = n.H, W = n.W, H2 = H / 2, W2 = W / 2, H4 = H / 4, W4 = W / 4, H8 = H / 8, W8 = W / 8;
    const int64_t P1 = (int64_t)H * W, P2 = (int64_t)H2 * W2, P4 = (int64_t)H4 * W4, P8 = (int64_t)H8 * W8;
    if (n.smooth) {
        smooth_passes(n, n.g_out, n.out_raw, B, s);   // d loss / d (pre-filter output), reusing out_raw
        conv_back<WT>(n, 14, n.d1, n.out_raw, n.g_d1, B, H, W, Wt, s);
    } else {
        conv_back<WT>(n, 14, n.d1, n.g_out, n.g_d1, B, H, W, Wt, s);
    }
    mask(n.g_d1, n.d1, B * 16 * P1, s);
    conv_back<WT>(n, 13, n.a6, n.g_d1, n.g_a6, B, H, W, Wt, s);
    mask(n.g_a6, n.a6, B * 16 * P1, s);
    conv_back<WT>(n, 12, n.u1, n.g_a6, n.g_u1, B, H, W, Wt, s);
    // u1 = [up(d2) | e1]
    up_bwd_kernel<<<blocks_for(B * 32 * P2), kT, 0, s>>>(n.g_u1, n.g_d2, B, 32, 48, H, W);
    chan_copy_kernel<<<blocks_for(B * 16 * P1), kT, 0, s>>>(n.g_u1, 48, 32, n.g_e1, 16, 0, 16, B, P1, 0);
    mask(n.g_d2, n.d2, B * 32 * P2, s);
    conv_back<WT>(n, 11, n.a5, n.g_d2, n.g_a5, B, H2, W2, Wt, s);
    mask(n.g_a5, n.a5, B * 32 * P2, s);
    conv_back<WT>(n, 10, n.u2, n.g_a5, n.g_u2, B, H2, W2, Wt, s);
    up_bwd_kernel<<<blocks_for(B * 64 * P4), kT, 0, s>>>(n.g_u2, n.g_d3, B, 64, 96, H2, W2);
    chan_copy_kernel<<<blocks_for(B * 32 * P2), kT, 0, s>>>(n.g_u2, 96, 64, n.g_e2, 32, 0, 32, B, P2, 0);
    mask(n.g_d3, n.d3, B * 64 * P4, s);
    conv_back<WT>(n, 9, n.a4, n.g_d3, n.g_a4, B, H4, W4, Wt, s);
    mask(n.g_a4, n.a4, B * 64 * P4, s);
    conv_back<WT>(n, 8, n.u3, n.g_a4, n.g_u3, B, H4, W4, Wt, s);
    up_bwd_kernel<<<blocks_for(B * 64 * P8), kT, 0, s>>>(n.g_u3, n.g_bt, B, 64, 128, H4, W4);
    chan_copy_kernel<<<blocks_for(B * 64 * P4), kT, 0, s>>>(n.g_u3, 128, 64, n.g_e3, 64, 0, 64, B, P4, 0);
    mask(n.g_bt, n.bt, B * 64 * P8, s);
    conv_back<WT>(n, 7, n.ab, n.g_bt, n.g_ab, B, H8, W8, Wt, s);
    mask(n.g_ab, n.ab, B * 64 * P8, s);
    conv_back<WT>(n, 6, n.p3, n.g_ab, n.g_p3, B, H8, W8, Wt, s);
    pool_bwd_kernel<<<blocks_for(B * 64 * P4), kT, 0, s>>>(n.g_p3, n.g_e3, B * 64, H4, W4, 1);
    mask(n.g_e3, n.e3, B * 64 * P4, s);
    conv_back<WT>(n, 5, n.a3, n.g_e3, n.g_a3, B, H4, W4, Wt, s);
    mask(n.g_a3, n.a3, B * 64 * P4, s);
    conv_back<WT>(n, 4, n.p2, n.g_a3, n.g_p2, B, H4, W4, Wt, s);
    pool_bwd_kernel<<<blocks_for(B * 32 * P2), kT, 0, s>>>(n.g_p2, n.g_e2, B * 32, H2, W2, 1);
    mask(n.g_e2, n.e2, B * 32 * P2, s);
    conv_back<WT>(n, 3, n.a2, n.g_e2, n.g_a2, B, H2, W2, Wt, s);
    mask(n.g_a2, n.a2, B * 32 * P2, s);
    conv_back<WT>(n, 2, n.p1, n.g_a2, n.g_p1, B, H2, W2, Wt, s);
    pool_bwd_kernel<<<blocks_for(B * 16 * P1), kT, 0, s>>>(n.g_p1, n.g_e1, B * 16, H, W, 1);
    mask(n.g_e1, n.e1, B * 16 * P1, s);
    conv_back<WT>(n, 1, n.a1, n.g_e1, n.g_a1, B, H, W, Wt, s);
    mask(n.g_a1, n.a1, B * 16 * P1, s);
    conv_back<WT>(n, 0, x, n.g_a1, nullptr, B, H, W, Wt, s);
}

int loss_and_grad(Net& n, const float* input, const float* target, int B, cudaStream_t s) {
    const int64_t cnt = (int64_t)B * n.H * n.W;
    const int nb = 64;
    mse_kernel<<<nb, kT, 0, s>>>(n.out, target, n.g_out, cnt, n.partial);
    if (n.res_w > 0.f) {
        const float h = 1.f / (float)(n.H + 1);
        resid_kernel<<<nb, kT, 0, s>>>(n.out, input, n.r, B, n.H, n.W, h, n.kappa, n.partial + nb);
        resid_grad_kernel<<<blocks_for(cnt), kT, 0, s>>>(n.r, input, n.g_out, B, n.H, n.W, h,
                                                         2.f * n.res_w * n.kappa / (float)cnt);
        sum_partials_kernel<<<1, 32, 0, s>>>(n.partial, nb, n.loss);
        sum_partials_kernel<<<1, 32, 0, s>>>(n.partial + nb, nb, n.loss + 1);
        combine_loss_kernel<<<1, 32, 0, s>>>(n.loss, n.res_w);
        return 0;
    }
    sum_partials_kernel<<<1, 32, 0, s>>>(n.partial, nb, n.loss);
    return 0;
}

// ------------------------------------------------------------------ the form's scalings
// The network sees each system scaled to O(1): features (f / s_f, beta / 20) with s_f the
// RMS of f, and it predicts x / (kappa s_f) with kappa = 1 / (2 pi^2 h^2) (the inverse of
// the smallest eigenvalue of the h^2-scaled Laplacian), so the targets are O(1) on any grid.

constexpr double kBetaScale = 20.0;

// one CTA per system: s_f = sqrt(mean f^2) (FP64, summed in a fixed order; 1 when f = 0)
// and the two feature planes
__global__ void __launch_bounds__(kT) features_kernel(const double* __restrict__ f, const double* __restrict__ beta,
                                                      int64_t hw, float* __restrict__ input, double* __restrict__ fscale) {
    __shared__ double part[kT / 32];
    const int64_t b = blockIdx.x;
    const double* fb = f + b * hw;
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < hw; i += kT) acc = fma(fb[i], fb[i], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    __shared__ double sf;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kT / 32; ++w) t += part[w];
        const double v = sqrt(t / (double)hw);
        sf = v > 0.0 ? v : 1.0;
        fscale[b] = sf;
    }
    __syncthreads();
    const double inv = 1.0 / sf;
    float* in0 = input + b * 2 * hw;
    float* in1 = in0 + hw;
    const double* bb = beta + b * hw;
    for (int64_t i = threadIdx.x; i < hw; i += kT) {
        in0[i] = (float)(fb[i] * inv);
        in1[i] = (float)(bb[i] / kBetaScale);
    }
}

// target = x / (kappa s_f) as FP32 (training pairs)
__global__ void __launch_bounds__(kT) targets_kernel(const double* __restrict__ x, const double* __restrict__ fscale,
                                                     int64_t hw, int64_t total, double kappa, float* __restrict__ target) {
    for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < total; i += (int64_t)gridDim.x * kT)
        target[i] = (float)(x[i] / (kappa * fscale[i / hw]));
}

// x0 = kappa s_f out (FP64)
__global__ void __launch_bounds__(kT) unscale_kernel(const float* __restrict__ out, const double* __restrict__ fscale,
                                                     int64_t hw, int64_t total, double kappa, double* __restrict__ x0) {
    for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < total; i += (int64_t)gridDim.x * kT)
        x0[i] = kappa * fscale[i / hw] * (double)out[i];
}

inline double kappa_of(int H) {
    const double h = 1.0 / (double)(H + 1);
    return 1.0 / (2.0 * 3.14159265358979323846 * 3.14159265358979323846 * h * h);
}

}  // namespace unet

using namespace unet;

struct x0net_s {
    Net n;
};

extern "C" {

int x0net_create(x0net* out, int H, int W, int batch_max, int bf16_weights, int smooth_passes) {
    if (!out || H < 8 || W < 8 || H % 8 || W % 8 || batch_max < 1 || smooth_passes < 0 || smooth_passes > 16)
        return SSTEP_ERR_ARG;
    *out = nullptr;
    x0net_s* X = new (std::nothrow) x0net_s;
    if (!X) return SSTEP_ERR_OOM;
    Net& n = X->n;
    n.H = H;
    n.W = W;
    n.Bmax = batch_max;
    n.bf16 = bf16_weights ? 1 : 0;
    n.smooth = smooth_passes;
    int64_t o = 0;
    for (int l = 0; l < kNumLayers; ++l) {
        n.off[l] = o;
        o += layer_params(kLayers[l]);
    }
    n.nparams = o;
    const int64_t B = batch_max, P1 = (int64_t)H * W, P2 = P1 / 4, P4 = P1 / 16, P8 = P1 / 64;
    bool ok = true;
    auto A = [&](int64_t c) {
        float* p = alloc(n, c);
        if (!p) ok = false;
        return p;
    };
    n.w = A(o);
    n.g = A(o);
    n.m = A(o);
    n.v = A(o);
    if (cudaMalloc((void**)&n.wb, sizeof(__nv_bfloat16) * o) != cudaSuccess) ok = false;
    if (cudaMalloc((void**)&n.err, sizeof(int)) != cudaSuccess) ok = false;
    else cudaMemset(n.err, 0, sizeof(int));
    n.a1 = A(B * 16 * P1); n.e1 = A(B * 16 * P1); n.p1 = A(B * 16 * P2);
    n.a2 = A(B * 32 * P2); n.e2 = A(B * 32 * P2); n.p2 = A(B * 32 * P4);
    n.a3 = A(B * 64 * P4); n.e3 = A(B * 64 * P4); n.p3 = A(B * 64 * P8);
    n.ab = A(B * 64 * P8); n.bt = A(B * 64 * P8);
    n.u3 = A(B * 128 * P4); n.a4 = A(B * 64 * P4); n.d3 = A(B * 64 * P4);
    n.u2 = A(B * 96 * P2); n.a5 = A(B * 32 * P2); n.d2 = A(B * 32 * P2);
    n.u1 = A(B * 48 * P1); n.a6 = A(B * 16 * P1); n.d1 = A(B * 16 * P1); n.out = A(B * P1);
    n.g_a1 = A(B * 16 * P1); n.g_e1 = A(B * 16 * P1); n.g_p1 = A(B * 16 * P2);
    n.g_a2 = A(B * 32 * P2); n.g_e2 = A(B * 32 * P2); n.g_p2 = A(B * 32 * P4);
    n.g_a3 = A(B * 64 * P4); n.g_e3 = A(B * 64 * P4); n.g_p3 = A(B * 64 * P8);
    n.g_ab = A(B * 64 * P8); n.g_bt = A(B * 64 * P8);
    n.g_u3 = A(B * 128 * P4); n.g_a4 = A(B * 64 * P4); n.g_d3 = A(B * 64 * P4);
    n.g_u2 = A(B * 96 * P2); n.g_a5 = A(B * 32 * P2); n.g_d2 = A(B * 32 * P2);
    n.g_u1 = A(B * 48 * P1); n.g_a6 = A(B * 16 * P1); n.g_d1 = A(B * 16 * P1); n.g_out = A(B * P1);
    n.partial = A(256);
    {   // the largest (chunks x weights) over the 3x3 layers at their levels
        int64_t need = 1;
        const int lvl[kNumLayers] = {1, 1, 2, 2, 4, 4, 8, 8, 4, 4, 2, 2, 1, 1, 1};
        for (int l = 0; l < kNumLayers; ++l) {
            const int cog = (kLayers[l].cout + 15) / 16, cig = (kLayers[l].cin + 15) / 16;
            for (int bb = 1; bb <= B; ++bb) {   // the chunking depends on the batch of the call
                if (kLayers[l].k == 3) {
                    const WgradShape ws = wgrad_shape(H / lvl[l], W / lvl[l], cog * cig * bb);
                    const int64_t nw = (int64_t)kLayers[l].cout * kLayers[l].cin * 9;
                    const int64_t v = bb * ws.chunks_per_image * nw;
                    need = v > need ? v : need;
                    const tc::WgradTcShape wt =
                        tc::wgrad_tc_shape(kLayers[l].cin, kLayers[l].cout, (int64_t)bb * (H / lvl[l]) * (W / lvl[l]));
                    need = wt.z * nw > need ? wt.z * nw : need;
                }
                // channel sums (bias and 1x1 gradients): chunks of kRedChunk pixels
                const int64_t px = (int64_t)(H / lvl[l]) * (W / lvl[l]);
                const int64_t v2 = bb * ((px + kRedChunk - 1) / kRedChunk) * (int64_t)(kLayers[l].cin + kLayers[l].cout);
                need = v2 > need ? v2 : need;
            }
        }
        n.wpart = A(need);
    }
    n.loss = A(2);
    n.r = A(B * P1);
    n.out_raw = A(B * P1);
    n.tmp = A(B * P1);
    n.blur = A(9);
    if (!ok) {
        cudaGetLastError();
        x0net_destroy(X);
        return SSTEP_ERR_OOM;
    }
    const float w1[3] = {0.25f, 0.5f, 0.25f};
    float bl[9];
    for (int k = 0; k < 9; ++k) bl[k] = w1[k / 3] * w1[k % 3];
    cudaMemcpy(n.blur, bl, sizeof(bl), cudaMemcpyHostToDevice);
    cudaMemset(n.m, 0, sizeof(float) * o);
    cudaMemset(n.v, 0, sizeof(float) * o);
    cudaMemset(n.w, 0, sizeof(float) * o);
    *out = X;
    return SSTEP_OK;
}

int x0net_destroy(x0net X) {
    if (!X) return SSTEP_ERR_ARG;
    for (float* p : X->n.bufs) cudaFree(p);
    if (X->n.wb) cudaFree(X->n.wb);
    if (X->n.err) cudaFree(X->n.err);
    delete X;
    return SSTEP_OK;
}

int x0net_set_residual_weight(x0net X, float w, float kappa) {
    if (!X || !(w >= 0.f) || !(kappa > 0.f)) return SSTEP_ERR_ARG;
    X->n.res_w = w;
    X->n.kappa = kappa;
    return SSTEP_OK;
}

int x0net_num_params(x0net X, int64_t* n) {
    if (!X || !n) return SSTEP_ERR_ARG;
    *n = X->n.nparams;
    return SSTEP_OK;
}

int x0net_set_params(x0net X, const float* params, void* stream) {
    if (!X || !params) return SSTEP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Net& n = X->n;
    if (cudaMemcpyAsync(n.w, params, sizeof(float) * n.nparams, cudaMemcpyDefault, s) != cudaSuccess)
        return SSTEP_ERR_CUDA;
    to_bf16_kernel<<<blocks_for(n.nparams), kT, 0, s>>>(n.w, n.wb, n.nparams);
    cudaMemsetAsync(n.m, 0, sizeof(float) * n.nparams, s);
    cudaMemsetAsync(n.v, 0, sizeof(float) * n.nparams, s);
    n.step = 0;
    return cudaGetLastError() == cudaSuccess ? SSTEP_OK : SSTEP_ERR_CUDA;
}

int x0net_get_params(x0net X, float* params, void* stream) {
    if (!X || !params) return SSTEP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(params, X->n.w, sizeof(float) * X->n.nparams, cudaMemcpyDefault, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return SSTEP_ERR_CUDA;
    return SSTEP_OK;
}

int x0net_get_state(x0net X, float* params, float* m, float* v, int64_t* step, void* stream) {
    if (!X || !params || !m || !v || !step) return SSTEP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const Net& n = X->n;
    const size_t bytes = sizeof(float) * n.nparams;
    if (cudaMemcpyAsync(params, n.w, bytes, cudaMemcpyDefault, s) != cudaSuccess ||
        cudaMemcpyAsync(m, n.m, bytes, cudaMemcpyDefault, s) != cudaSuccess ||
        cudaMemcpyAsync(v, n.v, bytes, cudaMemcpyDefault, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        return SSTEP_ERR_CUDA;
    *step = n.step;
    return SSTEP_OK;
}

int x0net_set_state(x0net X, const float* params, const float* m, const float* v, int64_t step, void* stream) {
    if (!X || !params || !m || !v || step < 0) return SSTEP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Net& n = X->n;
    const size_t bytes = sizeof(float) * n.nparams;
    if (cudaMemcpyAsync(n.w, params, bytes, cudaMemcpyDefault, s) != cudaSuccess ||
        cudaMemcpyAsync(n.m, m, bytes, cudaMemcpyDefault, s) != cudaSuccess ||
        cudaMemcpyAsync(n.v, v, bytes, cudaMemcpyDefault, s) != cudaSuccess)
        return SSTEP_ERR_CUDA;
    to_bf16_kernel<<<blocks_for(n.nparams), kT, 0, s>>>(n.w, n.wb, n.nparams);
    n.step = step;
    return cudaStreamSynchronize(s) == cudaSuccess && cudaGetLastError() == cudaSuccess ? SSTEP_OK : SSTEP_ERR_CUDA;
}

int x0net_forward(x0net X, const float* input, float* output, int batch, void* stream) {
    if (!X || !input || !output || batch < 1 || batch > X->n.Bmax) return SSTEP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Net& n = X->n;
    if (n.bf16) forward<__nv_bfloat16>(n, input, batch, s);
    else forward<float>(n, input, batch, s);
    if (cudaMemcpyAsync(output, n.out, sizeof(float) * batch * n.H * n.W, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return SSTEP_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? SSTEP_OK : SSTEP_ERR_CUDA;
}

int x0net_features(int H, int W, int batch, const double* f, const double* beta, float* input, double* f_scale,
                   void* stream) {
    if (H < 1 || W < 1 || batch < 1 || !f || !beta || !input || !f_scale) return SSTEP_ERR_ARG;
    const int64_t hw = (int64_t)H * W;
    unet::features_kernel<<<batch, unet::kT, 0, (cudaStream_t)stream>>>(f, beta, hw, input, f_scale);
    return cudaGetLastError() == cudaSuccess ? SSTEP_OK : SSTEP_ERR_CUDA;
}

int x0net_targets(int H, int W, int batch, const double* x, const double* f_scale, float* target, void* stream) {
    if (H < 1 || W < 1 || batch < 1 || !x || !f_scale || !target) return SSTEP_ERR_ARG;
    const int64_t hw = (int64_t)H * W, total = hw * batch;
    unet::targets_kernel<<<unet::blocks_for(total), unet::kT, 0, (cudaStream_t)stream>>>(x, f_scale, hw, total,
                                                                                      unet::kappa_of(H), target);
    return cudaGetLastError() == cudaSuccess ? SSTEP_OK : SSTEP_ERR_CUDA;
}

int x0net_predict(x0net X, const float* input, const double* f_scale, int batch, double* x0, void* stream) {
    if (!X || !input || !f_scale || !x0 || batch < 1 || batch > X->n.Bmax) return SSTEP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    unet::Net& n = X->n;
    if (n.bf16) unet::forward<__nv_bfloat16>(n, input, batch, s);
    else unet::forward<float>(n, input, batch, s);
    const int64_t hw = (int64_t)n.H * n.W, total = hw * batch;
    unet::unscale_kernel<<<unet::blocks_for(total), unet::kT, 0, s>>>(n.out, f_scale, hw, total, unet::kappa_of(n.H),
                                                                       x0);
    return cudaGetLastError() == cudaSuccess ? SSTEP_OK : SSTEP_ERR_CUDA;
}

int x0net_gradient(x0net X, const float* input, const float* target, int batch, float* loss, float* grads,
                   void* stream) {
    if (!X || !input || !target || batch < 1 || batch > X->n.Bmax) return SSTEP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Net& n = X->n;
    if (n.bf16) forward<__nv_bfloat16>(n, input, batch, s);
    else forward<float>(n, input, batch, s);
    loss_and_grad(n, input, target, batch, s);
    if (n.bf16) backward<__nv_bfloat16>(n, input, batch, s);
    else backward<float>(n, input, batch, s);
    if (loss && cudaMemcpyAsync(loss, n.loss, sizeof(float), cudaMemcpyDefault, s) != cudaSuccess) return SSTEP_ERR_CUDA;
    if (grads && cudaMemcpyAsync(grads, n.g, sizeof(float) * n.nparams, cudaMemcpyDefault, s) != cudaSuccess)
        return SSTEP_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SSTEP_ERR_CUDA;
    int e = 0;
    if (cudaMemcpy(&e, n.err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return SSTEP_ERR_CUDA;
    return e ? SSTEP_ERR_TIMEOUT : SSTEP_OK;
}

int x0net_set_tensor_cores(x0net X, int on) {
    if (!X) return SSTEP_ERR_ARG;
    X->n.tc = on ? 1 : 0;
    return SSTEP_OK;
}

int x0net_status(x0net X, void* stream) {
    if (!X) return SSTEP_ERR_ARG;
    int e = 0;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess ||
        cudaMemcpy(&e, X->n.err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
        (e && cudaMemset(X->n.err, 0, sizeof(int)) != cudaSuccess))
        return SSTEP_ERR_CUDA;
    return e ? SSTEP_ERR_TIMEOUT : SSTEP_OK;
}

int x0net_set_wait_limit(x0net X, int64_t polls) {
    if (!X) return SSTEP_ERR_ARG;
    X->n.spin = polls >= 0 ? (long)polls : tc::kSpin;
    return SSTEP_OK;
}

int x0net_train_step(x0net X, const float* input, const float* target, int batch, float lr, float* loss_dev,
                     void* stream) {
    if (!X || !input || !target || batch < 1 || batch > X->n.Bmax) return SSTEP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Net& n = X->n;
    if (n.bf16) forward<__nv_bfloat16>(n, input, batch, s);
    else forward<float>(n, input, batch, s);
    loss_and_grad(n, input, target, batch, s);
    if (n.bf16) backward<__nv_bfloat16>(n, input, batch, s);
    else backward<float>(n, input, batch, s);
    n.step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)n.step), c2 = 1.f - powf(b2, (float)n.step);
    adam_kernel<<<blocks_for(n.nparams), kT, 0, s>>>(n.w, n.g, n.m, n.v, n.wb, n.nparams, lr, b1, b2, 1e-8f, c1, c2);
    if (loss_dev &&
        cudaMemcpyAsync(loss_dev, n.loss, sizeof(float), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return SSTEP_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? SSTEP_OK : SSTEP_ERR_CUDA;
}

}  // extern "C"
