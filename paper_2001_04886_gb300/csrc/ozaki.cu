// The Gram pass C = V^T Y of the s-step block on the tensor cores (tcgen05), exact in
// fixed point (ozaki.cuh has the arithmetic and its error bound).
//
// One CTA owns a contiguous range of rows and walks it in stages of 64 rows. Every thread
// loads the FP64 entries of its (column, row pair) items straight from global memory into
// registers (the next stage's loads are issued before the current stage is split), turns
// each entry into its 8 balanced digits, and stores them as FP16 pairs in shared memory in
// the K-major no-swizzle layout of the MMA operands (K = the rows): A holds the digits of
// the V columns (M = digit x column, two 128-row tiles per 32 columns: digits 0-3 and
// 4-7), B those of the Y columns (N = digit x column, 80 rows). One thread issues
// tcgen05.mma.kind::f16 (FP16 x FP16 -> FP32 in tensor memory) for the kept digit pairs
// and commits to the stage's mbarrier; the shared-memory stage is double buffered.
// After at most 1024 rows (16 stages), while every FP32 sum in tensor memory is still an
// exact integer, the warps drain the accumulators into 128-bit integers in registers.
// At the end of its range the CTA publishes its exact integer partial sums; the last CTA
// to arrive adds them in CTA order (exact, so the result does not depend on the grid) and
// rounds each entry to FP64 once, then runs the solver epilogue like the FP64 kernel.
// Every mbarrier wait is bounded: a wait that runs out marks the result NaN (the solver
// then stops on its NaN checks) and the kernel still frees its tensor memory.
#include <cuda_fp16.h>

#include <algorithm>

#include "epilogue.cuh"
#include "ozaki.cuh"

namespace sstep {
namespace {

constexpr int kOzThreads = 256;
constexpr int kOzWarps = kOzThreads / 32;
constexpr int kStageRows = 64;                       // rows per stage (K of 4 MMAs)
constexpr int kTileBytes = 128 * kStageRows * 2;     // one A tile: 128 rows x 64 K x FP16
constexpr int kBRows = 80;                           // B rows: 8 digits x up to 9 columns, padded
constexpr int kBBytes = kBRows * kStageRows * 2;     // B: 80 rows x 64 K x FP16
constexpr int kN0 = 80, kN1 = 48;                    // MMA N of the digit-0..3 and digit-4..7 tiles
constexpr int kGroupCols = kN0 + kN1;                // tensor-memory columns per 32 V columns
constexpr int kStagesPerChunk = oz::kChunkRows / kStageRows;
constexpr long kOzSpin = 1L << 24;                   // bounded mbarrier polls

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (row m, k) of a K-major operand: 8-row x 16-byte core matrices,
// 128 B between K-adjacent and 1024 B between row-adjacent core matrices
__device__ __forceinline__ uint32_t op_off(int m, int k) {
    return (uint32_t)((m >> 3) * 1024 + (k >> 3) * 128 + (m & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor (no swizzle, LBO 128 B, SBO 1024 B)
__device__ __forceinline__ uint64_t op_desc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46);
}

// instruction descriptor: FP16 x FP16 -> FP32, K-major A and B, M = 128, N = n
__host__ __device__ constexpr uint32_t oz_idesc(int n) {
    return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// digit t of two biased words (rows r and r + 1 of a column) as an FP16 pair: the byte is
// placed in the mantissa of 1024.0 (FP16 bits 0x6400 | byte = 1024 + byte) and 1152 is
// subtracted, which leaves byte - 128 exactly
template <int T>
__device__ __forceinline__ uint32_t digit_pair(uint64_t w0, uint64_t w1) {
    constexpr int i = oz::kDigits - 1 - T;   // byte index
    constexpr int k = i & 3;
    constexpr uint32_t sel = (uint32_t)(k | (k << 4) | ((4 + k) << 8) | ((4 + k) << 12));
    const uint32_t a = i < 4 ? (uint32_t)w0 : (uint32_t)(w0 >> 32);
    const uint32_t b = i < 4 ? (uint32_t)w1 : (uint32_t)(w1 >> 32);
    const uint32_t x = (__byte_perm(a, b, sel) & 0x00FF00FFu) | 0x64006400u;
    const __half2 h = __hsub2(*reinterpret_cast<const __half2*>(&x), __halves2half2(__float2half(1152.f), __float2half(1152.f)));
    return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ __forceinline__ bool oz_wait(uint32_t bar, uint32_t parity, long limit) {
    uint32_t done = 0;
    for (long it = 0; it < limit && !done; ++it)
        asm volatile("{\n.reg .pred P;\nmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\nselp.b32 %0, 1, 0, P;\n}"
                     : "=r"(done)
                     : "r"(bar), "r"(parity)
                     : "memory");
    return done != 0;
}

__device__ __forceinline__ void mma_f16(uint32_t dtmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                 ::"r"(dtmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

template <int NC>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, uint32_t (&r)[NC]) {
#pragma unroll
    for (int c = 0; c < NC; c += 16) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[c + 0]), "=r"(r[c + 1]), "=r"(r[c + 2]), "=r"(r[c + 3]), "=r"(r[c + 4]), "=r"(r[c + 5]),
              "=r"(r[c + 6]), "=r"(r[c + 7]), "=r"(r[c + 8]), "=r"(r[c + 9]), "=r"(r[c + 10]), "=r"(r[c + 11]),
              "=r"(r[c + 12]), "=r"(r[c + 13]), "=r"(r[c + 14]), "=r"(r[c + 15])
            : "r"(taddr + (uint32_t)c));
    }
    asm volatile("tcgen05.wait::ld.sync.aligned;");
}

// ------------------------------------------------------------------ column bounds
// out[c] = max over the n entries of column c of the high word of |x| (atomicMax, so out
// must start at 0); one grid row of CTAs per column
__global__ void __launch_bounds__(kThreads) colmax_kernel(int64_t n, const double* __restrict__ X, int64_t ld,
                                                          unsigned* __restrict__ out) {
    const double* col = X + (int64_t)blockIdx.y * ld;
    unsigned m = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride)
        m = max(m, oz::abs_hiword((uint32_t)(__double_as_longlong(__ldg(col + p)) >> 32)));
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out + blockIdx.y, m);
}

}  // namespace
}  // namespace sstep

namespace sstep {
namespace {

// The digit-pair sums of one drained tile: TMEM lane (warp quarter q, lane) is the V
// digit ta of column a; its columns are (tb, b), b fastest. Each exact FP32 integer S is
// added into acc[b] with weight 256^(kCut - tb); the thread's contribution is acc >> 8 ta
// (every kept term has kCut - tb >= ta, so the shift is exact).
template <int KB, int NC>
__device__ __forceinline__ void drain_tile(uint32_t taddr, int ta, oz::i128 (&acc)[KB]) {
#pragma unroll
    for (int c0 = 0; c0 < NC; c0 += 16) {
        if (c0 >= (oz::kCut + 1 - ta) * KB) break;   // warp-uniform: the rest are dropped pairs
        uint32_t r[16];
        tmem_ld<16>(taddr + (uint32_t)c0, r);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int col = c0 + j, tb = col / KB, b = col % KB;
            if (col < NC && tb < oz::kDigits && tb <= oz::kCut - ta) {
                const int S = __float2int_rn(__uint_as_float(r[j]));
                acc[b] += (oz::i128)S << (8 * (oz::kCut - tb));
            }
        }
    }
}

template <int G, int KB>
__global__ void __launch_bounds__(kOzThreads, G == 1 ? 2 : 1)
    gram_oz_kernel(int64_t n, const double* __restrict__ V, int64_t ldv, int ka, const unsigned* __restrict__ vmax,
                   const double* __restrict__ Y, int64_t ldy, const unsigned* __restrict__ ymax, Scratch sc, Epi epi,
                   int gate, long spin) {
    constexpr int kStageBytes = 2 * G * kTileBytes + kBBytes;
    constexpr uint32_t kCols = G == 1 ? 128u : 256u;   // kGroupCols accumulator columns per 32 V columns
    constexpr int kItems = 4 * G + (KB + 7) / 8;        // column octets per warp and stage
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ uint32_t tmem_base;
    __shared__ int failed;
    __shared__ uint32_t ex[kMaxCols + kMaxS + 1];
    __shared__ double res[kMaxCols * (kMaxS + 1)];
    if (!gate_open(epi.st, gate)) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int c = tid; c < ka + KB; c += kOzThreads) ex[c] = oz::bound_exponent(c < ka ? vmax[c] : ymax[c - ka]);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                     "r"(kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        failed = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bars[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bars[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base, sbase = smem_addr(smem);

    // item j of this warp: column octet j (V octets first, then Y octets), the warp's K
    // group of 8 rows; lane: column c8 of the octet, rows kk and kk + 1 of the stage
    const int noct_v = (ka + 7) >> 3, noct = noct_v + (KB + 7) / 8;
    const int c8 = lane >> 2, kk = warp * 8 + (lane & 3) * 2;
    const int64_t nst = (n + kStageRows - 1) / kStageRows;
    const int64_t s0 = nst * blockIdx.x / gridDim.x, s1 = nst * (blockIdx.x + 1) / gridDim.x;
    const int h = warp >> 2, q = warp & 3, ta = 4 * h + q;   // drain role: V digit ta

    oz::i128 acc[G][KB];
#pragma unroll
    for (int g = 0; g < G; ++g)
#pragma unroll
        for (int b = 0; b < KB; ++b) acc[g][b] = 0;

    auto load = [&](int64_t st, double2 (&buf)[kItems]) {
        const int64_t r = st * kStageRows + kk;
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            buf[j] = make_double2(0.0, 0.0);
            if (j < noct) {
                const bool isv = j < noct_v;
                const int c = isv ? j * 8 + c8 : (j - noct_v) * 8 + c8;
                if (c < (isv ? ka : KB)) {
                    const double* col = isv ? V + (int64_t)c * ldv : Y + (int64_t)c * ldy;
                    if (r + 1 < n) {
                        if (((uintptr_t)(col + r) & 15) == 0) buf[j] = __ldg(reinterpret_cast<const double2*>(col + r));
                        else buf[j] = make_double2(__ldg(col + r), __ldg(col + r + 1));
                    } else if (r < n) {
                        buf[j].x = __ldg(col + r);
                    }
                }
            }
        }
    };

    int64_t last_commit[2] = {-1, -1};
    bool ok = true;
    double2 cur[kItems];
    if (s0 < s1) load(s0, cur);
    for (int64_t st = s0; st < s1; ++st) {
        const int64_t gs = st - s0;
        const int sb = (int)(gs & 1);
        double2 nxt[kItems];
        if (st + 1 < s1) load(st + 1, nxt);
        if (gs >= 2) {   // the MMAs of stage gs - 2 read this buffer
            if (!oz_wait(smem_addr(&bars[sb]), (uint32_t)(((gs - 2) >> 1) & 1), spin)) failed = 1;
            __syncthreads();
            if (failed) {
                ok = false;
                break;
            }
        }
        unsigned char* sp = smem + sb * kStageBytes;
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            if (j < noct) {
                const bool isv = j < noct_v;
                const int c = isv ? j * 8 + c8 : (j - noct_v) * 8 + c8;
                if (c < (isv ? ka : KB)) {
                    const uint32_t e = ex[isv ? c : ka + c];
                    const uint64_t b0 = (uint64_t)__double_as_longlong(cur[j].x), b1 = (uint64_t)__double_as_longlong(cur[j].y);
                    const uint64_t w0 = oz::fixed_biased((uint32_t)b0, (uint32_t)(b0 >> 32), e);
                    const uint64_t w1 = oz::fixed_biased((uint32_t)b1, (uint32_t)(b1 >> 32), e);
                    uint32_t d[oz::kDigits];
                    d[0] = digit_pair<0>(w0, w1);
                    d[1] = digit_pair<1>(w0, w1);
                    d[2] = digit_pair<2>(w0, w1);
                    d[3] = digit_pair<3>(w0, w1);
                    d[4] = digit_pair<4>(w0, w1);
                    d[5] = digit_pair<5>(w0, w1);
                    d[6] = digit_pair<6>(w0, w1);
                    d[7] = digit_pair<7>(w0, w1);
                    if (isv) {
                        unsigned char* base = sp + (c >> 5) * 2 * kTileBytes;
#pragma unroll
                        for (int t = 0; t < oz::kDigits; ++t)
                            *reinterpret_cast<uint32_t*>(base + (t >> 2) * kTileBytes + op_off((t & 3) * 32 + (c & 31), kk)) = d[t];
                    } else {
                        unsigned char* base = sp + 2 * G * kTileBytes;
#pragma unroll
                        for (int t = 0; t < oz::kDigits; ++t)
                            *reinterpret_cast<uint32_t*>(base + op_off(t * KB + c, kk)) = d[t];
                    }
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        const int sic = (int)(gs % kStagesPerChunk);
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t so = sbase + (uint32_t)(sb * kStageBytes);
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                    const uint32_t accf = (sic > 0 || ks > 0) ? 1u : 0u;
                    const uint32_t a0 = so + (uint32_t)(2 * g * kTileBytes + ks * 256);
                    const uint64_t db = op_desc(so + (uint32_t)(2 * G * kTileBytes + ks * 256));
                    mma_f16(tmem + (uint32_t)(g * kGroupCols), op_desc(a0), db, oz_idesc(kN0), accf);
                    mma_f16(tmem + (uint32_t)(g * kGroupCols + kN0), op_desc(a0 + kTileBytes), db, oz_idesc(kN1), accf);
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_addr(&bars[sb])));
        }
        last_commit[sb] = gs;
        if (sic == kStagesPerChunk - 1 || st + 1 == s1) {   // drain the chunk's exact sums
            if (!oz_wait(smem_addr(&bars[sb]), (uint32_t)((gs >> 1) & 1), spin)) failed = 1;
            __syncthreads();
            if (failed) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(g * kGroupCols);
                if (h == 0) drain_tile<KB, kN0>(taddr, ta, acc[g]);
                else drain_tile<KB, kN1>(taddr + (uint32_t)kN0, ta, acc[g]);
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
        }
#pragma unroll
        for (int j = 0; j < kItems; ++j) cur[j] = nxt[j];
    }
    if (!ok) {   // a wait ran out: let the MMAs in flight finish before the tensor memory is freed
        for (int b = 0; b < 2; ++b)
            if (last_commit[b] >= 0) oz_wait(smem_addr(&bars[b]), (uint32_t)((last_commit[b] >> 1) & 1), kOzSpin);
        if (tid == 0) atomicExch(sc.counter + 1, 1u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols));

    // the CTA's exact partial sums: per (digit ta, column a, column b) in shared memory (the
    // stage buffers are free), then summed over ta; published as the two 64-bit words of
    // each 128-bit integer
    oz::i128* part = reinterpret_cast<oz::i128*>(smem);   // [8][32 G][KB]
#pragma unroll
    for (int g = 0; g < G; ++g)
#pragma unroll
        for (int b = 0; b < KB; ++b) part[(ta * 32 * G + g * 32 + lane) * KB + b] = acc[g][b] >> (8 * ta);
    __syncthreads();
    double* red = reinterpret_cast<double*>(smem + oz::kDigits * 32 * G * KB * sizeof(oz::i128));
    for (int e = tid; e < ka * KB; e += kOzThreads) {
        const int a = e % ka, b = e / ka;
        oz::i128 s = 0;
        for (int t = 0; t < oz::kDigits; ++t) s += part[(t * 32 * G + a) * KB + b];
        red[2 * e] = __longlong_as_double((long long)(uint64_t)s);
        red[2 * e + 1] = __longlong_as_double((long long)(uint64_t)((oz::u128)s >> 64));
    }
    __syncthreads();
    if (!publish_partial(red, 2 * ka * KB, sc.partials, sc.counter)) return;
    // last CTA: exact sums over the CTAs in order, one rounding per entry
    const bool err = ((volatile unsigned*)sc.counter)[1] != 0u;
    const int nctas = gridDim.x;
    for (int e = tid; e < ka * KB; e += kOzThreads) {
        oz::i128 s = 0;
        for (int bx = 0; bx < nctas; ++bx) {
            const double* p = sc.partials + (int64_t)bx * (2 * ka * KB) + 2 * e;
            const uint64_t lo = (uint64_t)__double_as_longlong(ld_cg(p)), hi = (uint64_t)__double_as_longlong(ld_cg(p + 1));
            s += (oz::i128)(((oz::u128)hi << 64) | (oz::u128)lo);
        }
        const uint32_t ea = ex[e % ka], eb = ex[ka + e / ka];
        res[e] = (err || ea == oz::kNonFinite || eb == oz::kNonFinite) ? __longlong_as_double(0x7FF8000000000000ll)
                                                                       : oz::i128_to_double(s, oz::gram_scale_exp(ea, eb));
    }
    __syncthreads();
    if (tid == 0) {
        sc.counter[0] = 0u;
        sc.counter[1] = 0u;
    }
    run_epilogue(epi, res, ka, KB);
}

}  // namespace
}  // namespace sstep

namespace sstep {

int device_sms() {
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        dev = 0;
    }
    if (dev < 0 || dev >= 64) dev = 0;
    if (!cached[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) {
            cudaGetLastError();
            v = 1;
        }
        cached[dev] = v;
    }
    return cached[dev];
}

// one CTA per SM with ka <= 64 or two with ka <= 32: at most 2 SMs x 2 x 32 x 9 doubles
int oz_partials_doubles() { return 2 * device_sms() * 2 * 32 * (kMaxS + 1); }

void launch_colmax(int64_t n, const double* X, int64_t ld, int ncols, unsigned* out, cudaStream_t stream) {
    if (n <= 0 || ncols <= 0) return;
    const int per_col = std::max(1, std::min(grid_for(n, 4 * device_sms()), (4 * device_sms() + ncols - 1) / ncols));
    colmax_kernel<<<dim3(per_col, ncols), kThreads, 0, stream>>>(n, X, ld, out);
}

namespace {
template <int G, int KB>
void launch_oz(int64_t n, const double* V, int64_t ldv, int ka, const unsigned* vmax, const double* Y, int64_t ldy,
               const unsigned* ymax, Scratch sc, const Epi& epi, int gate, cudaStream_t stream, long spin) {
    constexpr int kSmem = 2 * (2 * G * kTileBytes + kBBytes);
    static bool attr[64] = {false};   // once per device
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attr[dev]) {
        cudaFuncSetAttribute(gram_oz_kernel<G, KB>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
        if (dev >= 0 && dev < 64) attr[dev] = true;
    }
    const int64_t nst = (n + kStageRows - 1) / kStageRows;
    int grid = (G == 1 ? 2 : 1) * device_sms();
    if (grid > nst) grid = (int)std::max<int64_t>(nst, 1);
    gram_oz_kernel<G, KB><<<grid, kOzThreads, kSmem, stream>>>(n, V, ldv, ka, vmax, Y, ldy, ymax, sc, epi, gate, spin);
}
}  // namespace

long g_oz_spin = kOzSpin;

bool launch_gram_oz(int64_t n, const double* V, int64_t ldv, int ka, const unsigned* vmax, const double* Y,
                    int64_t ldy, int kb, const unsigned* ymax, Scratch sc, const Epi& epi, int gate,
                    cudaStream_t stream) {
    if (ka < 1 || ka > kMaxCols || kb < 1 || kb > kMaxS + 1 || n < 1 || n > ((int64_t)1 << 27)) return false;
    if (((uintptr_t)V & 7) || ((uintptr_t)Y & 7)) return false;
    const bool one = ka <= 32;
    switch (kb) {
#define SSTEP_OZ_CASE(KB)                                                                                       \
    case KB:                                                                                                    \
        if (one) launch_oz<1, KB>(n, V, ldv, ka, vmax, Y, ldy, ymax, sc, epi, gate, stream, g_oz_spin);         \
        else launch_oz<2, KB>(n, V, ldv, ka, vmax, Y, ldy, ymax, sc, epi, gate, stream, g_oz_spin);             \
        return true;
        SSTEP_OZ_CASE(1)
        SSTEP_OZ_CASE(2)
        SSTEP_OZ_CASE(3)
        SSTEP_OZ_CASE(4)
        SSTEP_OZ_CASE(5)
        SSTEP_OZ_CASE(6)
        SSTEP_OZ_CASE(7)
        SSTEP_OZ_CASE(8)
        SSTEP_OZ_CASE(9)
#undef SSTEP_OZ_CASE
        default: return false;
    }
}

}  // namespace sstep
