// The Gram pass C = V^T Y of the s-step block on the tensor cores (tcgen05), exact in
// fixed point (ozaki.cuh has the arithmetic and its error bound).
//
// One CTA per SM owns a contiguous range of rows and walks it in stages (128 rows, or 64
// when V has more than 32 columns). The split warps load the FP64 entries of their
// (column, row pair) items straight from global memory into registers (the next stage's
// loads are issued before the current stage is split), turn each entry into its 8
// balanced digits and store them as FP16 pairs in shared memory in the K-major no-swizzle
// layout of the MMA operands (K = the rows): A holds the digits of the V columns (M =
// digit x column, two 128-row tiles per 32 columns: digits 0-3 and 4-7), B those of the Y
// columns (N = digit x column, 80 rows). A dedicated MMA warp waits for a stage to be full
// (an mbarrier every split warp arrives on), issues tcgen05.mma.kind::f16 (FP16 x FP16 ->
// FP32 in tensor memory) for the kept digit pairs and commits to the stage's empty
// barrier; shared-memory stages and tensor-memory accumulators are both double buffered,
// so no CTA-wide barrier sits in the loop. After at most 1024 rows, while every FP32 sum
// is still an exact integer, the split warps drain the accumulators into 128-bit integers
// (while the MMAs of the next chunk run into the other accumulator buffer). At the end the
// CTA adds its exact partial sums into a 128-bit accumulator per entry with 64-bit
// atomicAdds (carry handled: integer addition is exact and order-free, so the result does
// not depend on the grid), and the last CTA to arrive rounds each entry to FP64 once and
// runs the solver epilogue like the FP64 kernel. Every mbarrier wait is bounded: a wait
// that runs out marks the result NaN (the solver then stops on its checks) and the kernel
// still waits for its tensor-core work in flight and frees its tensor memory.
#include <cuda_fp16.h>

#include <algorithm>
#include <type_traits>

#include "epilogue.cuh"
#include "ozaki.cuh"

namespace sstep {
namespace {

constexpr int kN1 = 48;                              // MMA N of the digit-4..7 tile (G >= 1): digits tb <= 4
constexpr long kOzSpin = 1L << 24;                   // bounded mbarrier polls

// Shapes of one instantiation: G groups of 32 V columns, KB Y columns.
// (14 split warps + the MMA warp: at most 4 warps per SM sub-partition, so 128 registers
// per thread; a stage of 112 rows is 7 MMA K-steps and 9 stages make a chunk of 1008 rows.)
// G = 0: at most 16 V columns, one A tile of all 8 digits x 16 columns; G = 1, 2: up to
// 32 G V columns, two tiles per 32 columns (digits 0-3 and 4-7). B row t BST + b holds
// digit t of Y column b: BST = 8 for KB <= 8, and for KB = 9 16 (G = 0) or 9 (G >= 1), so
// that, except in the last case, a digit's rows start on an 8-row core-matrix boundary and
// an octet's unused columns fall in rows that no kept sum reads.
template <int G, int KB>
struct OzCfg {
    static constexpr int kBst = KB <= 8 ? 8 : (G == 0 ? 16 : KB);
    static constexpr bool kFastB = kBst % 8 == 0;               // digit t's B rows at t kBst / 8 row groups
    // MMA N of the digit-0..3 tile (G = 0: the one tile): every B row, rounded up to 16;
    // B rows allocated: those, plus the spare rows 72..79 of BST = 9
    static constexpr int kN0 = (8 * kBst + 15) / 16 * 16;
    static constexpr int kBRows = kN0;
    static constexpr int kGroupCols = kN0 + kN1;                // tensor-memory columns per 32 V columns (G >= 1)
    static constexpr int kSplitWarps = G <= 1 ? 14 : 8;
    static constexpr int kThreads = (kSplitWarps + 1) * 32;   // + the MMA warp
    static constexpr int kRows = 8 * kSplitWarps;             // rows per stage (one K group per split warp)
    static constexpr int kSbo = kRows * 16;                   // bytes between 8-row groups of an operand
    static constexpr int kTile = 128 * kRows * 2;             // one A tile (FP16)
    static constexpr int kB = kBRows * kRows * 2;             // B
    static constexpr int kAT = G == 0 ? 1 : 2 * G;            // A tiles per stage
    static constexpr int kGroups = G == 0 ? 1 : G;            // column groups
    static constexpr int kColsPer = G == 0 ? 16 : 32;         // V columns per group
    static constexpr int kStage = kAT * kTile + kB;
    static constexpr int kNStages = G == 0 ? (kBst > 8 ? 3 : 4) : 2;
    static constexpr int kSmem = kNStages * kStage;
    static constexpr int kStagesPerChunk = oz::kChunkRows / kRows;
    static constexpr int kBuf = G == 0 ? 128 : G * kGroupCols;   // accumulator columns per buffer
    static_assert(2 * kBuf <= 512, "tensor memory");
    static constexpr uint32_t kCols = 2 * kBuf <= 256 ? 256u : 512u;
    static_assert(kRows % 16 == 0 && kStagesPerChunk * kRows <= oz::kChunkRows, "stage shape");
    static_assert(kN0 <= 128 && 8 * kBst <= kBRows && (G == 0 || 5 * kBst <= kN1), "B shape");
    static_assert(kSmem <= 227 * 1024, "shared memory");
};
constexpr int kDrainWarps = 8;   // split warps 0..7 drain: TMEM lane quarter warp % 4, tile warp / 4

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }


// byte offset of element (row m, k) of a K-major operand: 8-row x 16-byte core matrices,
// 128 B between K-adjacent and SBO bytes between row-adjacent core matrices
template <int SBO>
__device__ __forceinline__ uint32_t op_off(int m, int k) {
    return (uint32_t)((m >> 3) * SBO + (k >> 3) * 128 + (m & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor (no swizzle, LBO 128 B)
template <int SBO>
__device__ __forceinline__ uint64_t op_desc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(SBO >> 4) << 32) |
           ((uint64_t)1 << 46);
}

__device__ __forceinline__ void bar_init(uint64_t* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count));
}

__device__ __forceinline__ void bar_arrive(uint64_t* b) {
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(smem_addr(b)) : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(b))
                 : "memory");
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

// digits T and T + 1 (T even: bytes i = 7 - T and i - 1 of the same 32-bit word) of two
// rows as two FP16 pairs: one byte permute gathers the four bytes, two more interleave
// them with the FP16 exponent byte 0x64 (1024 + byte), and 1152 is subtracted
template <int T>
__device__ __forceinline__ void digit_pairs2(uint32_t a, uint32_t b, uint32_t& dt, uint32_t& dt1) {
    constexpr int k = (oz::kDigits - 1 - T) & 3;   // byte of digit T within its word; k - 1 holds digit T + 1
    constexpr uint32_t sel = (uint32_t)(k | ((4 + k) << 4) | ((k - 1) << 8) | ((3 + k) << 12));
    const uint32_t p = __byte_perm(a, b, sel);                 // [a_k, b_k, a_k-1, b_k-1]
    const uint32_t x0 = __byte_perm(p, 0x64646464u, 0x4140u);  // [a_k, 0x64, b_k, 0x64]
    const uint32_t x1 = __byte_perm(p, 0x64646464u, 0x4342u);  // [a_k-1, 0x64, b_k-1, 0x64]
    const __half2 off = __halves2half2(__float2half(1152.f), __float2half(1152.f));
    const __half2 h0 = __hsub2(*reinterpret_cast<const __half2*>(&x0), off);
    const __half2 h1 = __hsub2(*reinterpret_cast<const __half2*>(&x1), off);
    dt = *reinterpret_cast<const uint32_t*>(&h0);
    dt1 = *reinterpret_cast<const uint32_t*>(&h1);
}

// the 8 digits (top first) of one entry as FP16, in one 16-byte row: pairs (t, t + 1) from
// one byte permute each (bytes i and i - 1 of a word, interleaved with the exponent byte
// 0x64), 1152 subtracted
__device__ __forceinline__ void digit_row8(uint32_t wl, uint32_t wh, uint4& v) {
    const __half2 off = __halves2half2(__float2half(1152.f), __float2half(1152.f));
    uint32_t x[4] = {__byte_perm(wh, 0x64646464u, 0x4243u), __byte_perm(wh, 0x64646464u, 0x4041u),
                     __byte_perm(wl, 0x64646464u, 0x4243u), __byte_perm(wl, 0x64646464u, 0x4041u)};
    uint32_t r[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const __half2 h = __hsub2(*reinterpret_cast<const __half2*>(&x[i]), off);
        r[i] = *reinterpret_cast<const uint32_t*>(&h);
    }
    v = make_uint4(r[0], r[1], r[2], r[3]);
}

// the 8 digit pairs (top first) of two rows of one column from their biased words
__device__ __forceinline__ void digits8(uint32_t l0, uint32_t h0, uint32_t l1, uint32_t h1, uint32_t (&d)[oz::kDigits]) {
    digit_pairs2<0>(h0, h1, d[0], d[1]);
    digit_pairs2<2>(h0, h1, d[2], d[3]);
    digit_pairs2<4>(l0, l1, d[4], d[5]);
    digit_pairs2<6>(l0, l1, d[6], d[7]);
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

// the same bounded wait with a short sleep between polls (the MMA-issue thread, which
// otherwise polls for the whole time the split warps fill a stage)
__device__ __forceinline__ bool oz_wait_sleep(uint32_t bar, uint32_t parity, long limit) {
    uint32_t done = 0;
    for (long it = 0; it < limit; ++it) {
        asm volatile("{\n.reg .pred P;\nmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\nselp.b32 %0, 1, 0, P;\n}"
                     : "=r"(done)
                     : "r"(bar), "r"(parity)
                     : "memory");
        if (done) break;
        __nanosleep(32);
    }
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

// The digit-pair sums of one drained tile: TMEM lane (warp quarter, lane) is the V digit
// ta of column a; its column tb BST + b holds the sum against digit tb of Y column b, read
// 16 at a time (columns with b >= KB hold nothing kept). Each exact FP32 integer S is added
// into acc[b] with weight 256^(kCut - tb); the thread's contribution is acc >> 8 ta (every
// kept term has kCut - tb >= ta, so that shift is exact).
template <int KB, int BST, int NC>
__device__ __forceinline__ void drain_tile(uint32_t taddr, int ta, int tmin, oz::i128 (&acc)[KB]) {
#pragma unroll
    for (int c0 = 0; c0 < NC; c0 += 16) {
        if (c0 >= (oz::kCut + 1 - tmin) * BST) break;     // warp-uniform (tmin: the warp's smallest ta)
        uint32_t r[16];
        tmem_ld<16>(taddr + (uint32_t)c0, r);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int col = c0 + j, tb = col / BST, b = col % BST;
            if (col < NC && b < KB && tb < oz::kDigits && tb <= oz::kCut - ta) {
                const int S = __float2int_rn(__uint_as_float(r[j]));
                acc[b] += (oz::i128)S << (8 * (oz::kCut - tb));
            }
        }
    }
}

// ZS: the symmetric 9-column pass V^T V of the s-step block at s = 8 (the z mode below,
// one column octet per warp). Its rows come into shared memory by TMA bulk copies (a
// producer warp keeps kZRawSlots stages of the 9 columns in flight) and the split warps
// read them from there; its B operand is its A tile (V = Y: the same digits in the same
// rows), so a digit stage is one tile and four of them fit. The other forms load their
// entries straight into registers one stage ahead.
constexpr int kZRawSlots = 8;                 // stages of raw rows in flight (ZS)
template <int G, int KB>
struct ZRaw {
    static constexpr int kCol = OzCfg<G, KB>::kRows + 8;   // doubles between columns: 960 B, half a bank row off
    static constexpr int kSlot = 9 * kCol * 8;             // bytes per slot: the 9 columns of one stage
    // digit stages: the A tile only (V^T V: the B operand is the same tile)
    static constexpr int kNS = 4;
    static constexpr int kSmem = kNS * OzCfg<G, KB>::kTile + kZRawSlots * kSlot;
    static_assert(kSmem <= 200 * 1024, "shared memory (static use besides)");
};
template <int G, int KB, bool ZS>
__global__ void __launch_bounds__(OzCfg<G, KB>::kThreads + (ZS ? 32 : 0), 1)
    gram_oz_kernel(int64_t n, const double* __restrict__ V, int64_t ldv, int ka, const unsigned* __restrict__ vmax,
                   const double* __restrict__ Y, int64_t ldy, const unsigned* __restrict__ ymax, Scratch sc, Epi epi,
                   int gate, long spin, int sym, int vw, uint64_t* __restrict__ wout, int64_t ldw, int nw) {
    using C = OzCfg<G, KB>;
    static_assert(!ZS || (G == 0 && KB == 9 && C::kSplitWarps == 14), "z mode shape");
    constexpr int BST = C::kBst;
    constexpr int kItems = ZS ? 1 : (G == 0 ? 2 : 4 * G) + (KB + 7) / 8;   // column octets per split warp and stage
    constexpr int PD = 1;                                          // stages of register loads in flight
    static_assert(C::kStagesPerChunk % PD == 0, "a chunk ends in the ring's last slot");
    constexpr int NT = C::kThreads + (ZS ? 32 : 0);                // + the producer warp (ZS)
    constexpr int RS = ZS ? kZRawSlots : 1;
    using R = ZRaw<0, 9>;
    constexpr int NS = ZS ? R::kNS : C::kNStages, NG = C::kGroups, CP = C::kColsPer;
    constexpr int STG = ZS ? C::kTile : C::kStage;   // bytes per digit stage
    constexpr int SBO = C::kSbo;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[NS], empty[NS], tfull[2], tempty[2], rfull[RS], rempty[RS];
    __shared__ uint32_t tmem_base;
    __shared__ volatile int failed;
    __shared__ bool last;
    __shared__ uint32_t ex[kMaxCols + kMaxS + 1];
    __shared__ double res[kMaxCols * (kMaxS + 1)];
    if (!gate_open(epi.st, gate)) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int c = tid; c < ka + KB; c += NT) ex[c] = oz::bound_exponent(c < ka ? vmax[c] : ymax[c - ka]);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                     "r"(C::kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        failed = 0;
        for (int b = 0; b < NS; ++b) {
            bar_init(&full[b], C::kSplitWarps);
            bar_init(&empty[b], 1);
        }
        for (int b = 0; b < 2; ++b) {
            bar_init(&tfull[b], 1);
            bar_init(&tempty[b], G == 0 ? 4 : kDrainWarps);   // the warps that drain (see drains)
        }
        if (ZS)
            for (int b = 0; b < RS; ++b) {
                bar_init(&rfull[b], 1);
                bar_init(&rempty[b], C::kSplitWarps);
            }
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base, sbase = smem_addr(smem);
    const int64_t nst = (n + C::kRows - 1) / C::kRows;
    const int64_t s0 = nst * blockIdx.x / gridDim.x, s1 = nst * (blockIdx.x + 1) / gridDim.x;
    const int64_t nstages = s1 - s0;

    // drain role: G >= 1: split warps 0..7, TMEM lane quarter q, V digit ta, column g 32 +
    // lane; G = 0: split warps 0..3, lane quarter q holds digits 2q and 2q + 1 of 16 columns
    const int q = warp & 3;
    const int ta = G == 0 ? 2 * q + (lane >> 4) : 4 * ((warp >> 2) & 1) + q;
    const int tmin = G == 0 ? 2 * q : ta;
    const int al_ = G == 0 ? (lane & 15) : lane;   // column within its group
    const bool drains = warp < (G == 0 ? 4 : kDrainWarps);
    oz::i128 acc[NG][KB];
#pragma unroll
    for (int g = 0; g < NG; ++g)
#pragma unroll
        for (int b = 0; b < KB; ++b) acc[g][b] = 0;

    if (warp == C::kSplitWarps) {
        // ---------------------------------------------------------------- MMA warp
        if (lane == 0) {
            int n_empty[NS] = {}, n_tfull[2] = {0, 0};
            for (unsigned gs = 0; gs < (unsigned)nstages && !failed; ++gs) {
                const int sb = (int)(gs % NS);
                const int chunk = (int)(gs / C::kStagesPerChunk), sic = (int)(gs % C::kStagesPerChunk);
                const int tb = chunk & 1;
                if (sic == 0 && chunk >= 2 &&   // the accumulators of chunk - 2 are drained
                    !oz_wait_sleep(smem_addr(&tempty[tb]), (uint32_t)(((chunk >> 1) - 1) & 1), spin)) {
                    failed = 1;
                    break;
                }
                if (!oz_wait_sleep(smem_addr(&full[sb]), (uint32_t)((gs / NS) & 1), spin)) {
                    failed = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t so = sbase + (uint32_t)(sb * STG);
                const uint32_t dt = tmem + (uint32_t)(tb * C::kBuf);
                if (G == 0) {   // one tile: all digit pairs of 16 columns against the B digits
#pragma unroll
                    for (int ks = 0; ks < C::kRows / 16; ++ks)
                        mma_f16(dt, op_desc<SBO>(so + (uint32_t)(ks * 256)),
                                op_desc<SBO>(so + (uint32_t)((ZS ? 0 : C::kTile) + ks * 256)), oz_idesc(C::kN0),
                                (sic > 0 || ks > 0) ? 1u : 0u);
                }
#pragma unroll
                for (int g = 0; g < G; ++g)
#pragma unroll
                    for (int ks = 0; ks < C::kRows / 16; ++ks) {
                        const uint32_t accf = (sic > 0 || ks > 0) ? 1u : 0u;
                        const uint32_t a0 = so + (uint32_t)(2 * g * C::kTile + ks * 256);
                        const uint64_t db = op_desc<SBO>(so + (uint32_t)(2 * G * C::kTile + ks * 256));
                        mma_f16(dt + (uint32_t)(g * C::kGroupCols), op_desc<SBO>(a0), db, oz_idesc(C::kN0), accf);
                        mma_f16(dt + (uint32_t)(g * C::kGroupCols + C::kN0), op_desc<SBO>(a0 + C::kTile), db, oz_idesc(kN1),
                                accf);
                    }
                mma_commit(&empty[sb]);
                ++n_empty[sb];
                if (sic == C::kStagesPerChunk - 1 || gs + 1 == (unsigned)nstages) {
                    mma_commit(&tfull[tb]);
                    ++n_tfull[tb];
                }
            }
            // every commit has landed before the CTA leaves (no arrive is left pending)
            for (int b = 0; b < NS; ++b)
                if (n_empty[b]) oz_wait(smem_addr(&empty[b]), (uint32_t)((n_empty[b] - 1) & 1), kOzSpin);
            for (int b = 0; b < 2; ++b)
                if (n_tfull[b]) oz_wait(smem_addr(&tfull[b]), (uint32_t)((n_tfull[b] - 1) & 1), kOzSpin);
        }
        __syncwarp();
    } else if (ZS && warp == C::kSplitWarps + 1) {
        // ---------------------------------------------------------------- producer warp (ZS)
        // stage gs: rows r0 .. r0 + 111 of the 9 columns into raw slot gs % RS, one bulk copy
        // per column (an even row count: a last odd row is read by its split lane directly)
        if (lane == 0) {
            int64_t issued = 0;
            for (int64_t gs = 0; gs < nstages && !failed; ++gs) {
                const int slot = (int)(gs % RS);
                if (gs >= RS && !oz_wait_sleep(smem_addr(&rempty[slot]), (uint32_t)(((gs / RS) - 1) & 1), spin)) {
                    failed = 1;
                    break;
                }
                const int64_t r0 = (s0 + gs) * C::kRows, left = n - r0;
                const uint32_t bytes = (uint32_t)(left >= C::kRows ? C::kRows : (left & ~1ll)) * 8u;
                const uint32_t bar = smem_addr(&rfull[slot]);
                const uint32_t dst = sbase + (uint32_t)(NS * STG + slot * R::kSlot);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(9u * bytes)
                             : "memory");
                if (bytes)
                    for (int c = 0; c < 9; ++c)
                        asm volatile(
                            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                            ::"r"(dst + (uint32_t)(c * R::kCol * 8)), "l"(V + (int64_t)c * ldv + r0), "r"(bytes),
                            "r"(bar)
                            : "memory");
                issued = gs + 1;
            }
            // every copy has landed before the CTA goes on (the split warps waited for all of
            // them unless they stopped early)
            for (int64_t gs = issued > RS ? issued - RS : 0; gs < issued; ++gs)
                oz_wait(smem_addr(&rfull[gs % RS]), (uint32_t)((gs / RS) & 1), kOzSpin);
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------------------- split warps
        // item j: column octet j (V octets first, then Y octets) of this warp's K group of 8
        // rows; lane: column c8 of the octet, rows kk and kk + 1 of the stage
        // sym (V = Y): the V columns only, each digit stored into A and B
        // zmode (the 9-column V^T V of the s-step block, s = 8): columns 0..7 as one octet in
        // every warp, and column 8 as one item of 28 row pairs in each of warps 2 and 3 (the
        // two sub-partitions with three split warps), instead of a second octet with one
        // column in use in every warp; its stores meet bank conflicts, the issue slots are fewer
        const bool zmode = ZS;   // (chosen at launch: sym, ka = KB = 9)
        const int noct_v = zmode ? 1 : (ka + 7) >> 3, noct = noct_v + (sym ? 0 : (KB + 7) / 8);
        const int c8 = lane >> 2, kk = warp * 8 + (lane & 3) * 2;
        const bool zw = zmode && (warp == 2 || warp == 3);            // warp-uniform
        const int zrow = (warp - 2) * 56 + 2 * lane;                   // stage row of a z lane
        const bool zl = zw && lane < 28;
        const double* zp = Y + 8 * ldy + s0 * C::kRows + (zl ? zrow : 0);
        const uint32_t ze = ex[ka + (KB > 8 ? 8 : 0)];
        // per item: the entry (row kk of this CTA's first stage) and whether it is 16-byte
        // aligned (kk and the stage height are even, so that holds for every stage)
        // per item: the entry in row kk of this CTA's first stage (a column past ka or kb reads
        // column 0 of its operand instead, so every lane loads, and its digits are stored
        // where no kept sum reads them), its bound exponent and its shared-memory offsets
        const double* cp[kItems];
        uint32_t ce[kItems];
        uint32_t aoff[kItems], boff[kItems];   // byte offsets of digit 0 in A and in B (none: ~0u)
        int bcol[kItems];
        bool cv[kItems];
        bool al = true;                        // every item's entries 16-byte aligned
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            const bool isv = j < noct_v;
            const int c = isv ? j * 8 + c8 : (j - noct_v) * 8 + c8;
            cv[j] = j < noct && c < (isv ? ka : KB);
            const int cl = cv[j] ? c : 0;
            cp[j] = (isv ? V + (int64_t)cl * ldv : Y + (int64_t)cl * ldy) + s0 * C::kRows + kk;
            al = al && ((uintptr_t)cp[j] & 15) == 0;
            ce[j] = ex[isv ? cl : ka + cl];
            // B: digit t of column c in row t BST + c (C::kFastB: the octet's unused columns land
            // in rows no drain reads); otherwise (BST = 9) the row is formed per digit
            if (isv) {
                aoff[j] = G == 0 ? op_off<SBO>(c, kk) : (uint32_t)((c >> 5) * 2 * C::kTile) + op_off<SBO>(c & 31, kk);
                boff[j] = sym ? (uint32_t)(C::kAT * C::kTile) + op_off<SBO>(c, kk) : ~0u;
            } else {
                aoff[j] = ~0u;
                boff[j] = (uint32_t)(C::kAT * C::kTile) + (C::kFastB ? op_off<SBO>(c, kk) : 0u);
            }
            bcol[j] = c;
        }
        al = __all_sync(0xffffffffu, al);   // (the z column is aligned with column 0, in every warp's test)
        auto zload = [&](int64_t st, double2& z) {
            z = make_double2(0.0, 0.0);
            if (!zl) return;
            const int64_t r = (s0 + st) * C::kRows + zrow;
            if ((s0 + st + 1) * C::kRows <= n && al) {
                z = __ldg(reinterpret_cast<const double2*>(zp + st * C::kRows));
            } else {
                if (r < n) z.x = __ldg(zp + st * C::kRows);
                if (r + 1 < n) z.y = __ldg(zp + st * C::kRows + 1);
            }
        };
        auto load = [&](int64_t st, double2 (&buf)[kItems]) {
            const int64_t off = st * C::kRows, r = (s0 + st) * C::kRows + kk;
            const bool whole = (s0 + st + 1) * C::kRows <= n;   // warp-uniform: no row past n
            if (whole && al) {
#pragma unroll
                for (int j = 0; j < kItems; ++j)
                    if (j < noct) buf[j] = __ldg(reinterpret_cast<const double2*>(cp[j] + off));
            } else {
#pragma unroll
                for (int j = 0; j < kItems; ++j) {
                    buf[j] = make_double2(0.0, 0.0);
                    if (j < noct) {
                        const double* p = cp[j] + off;
                        if (r < n) buf[j].x = __ldg(p);
                        if (r + 1 < n) buf[j].y = __ldg(p + 1);
                    }
                }
            }
        };
        // the chunk's exact sums out of tensor memory into the 128-bit accumulators
        // (only the draining warps wait for the chunk's sums; the others go on splitting the
        // next chunk's stages into the other accumulator buffer)
        auto drain_chunk = [&](int chunk) -> bool {
            if (!drains) return true;
            const int tb = chunk & 1;
            if (!oz_wait(smem_addr(&tfull[tb]), (uint32_t)((chunk >> 1) & 1), spin)) return false;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t tb0 = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(tb * C::kBuf);
            if (drains) {
                if (G == 0) {
                    drain_tile<KB, BST, C::kN0>(tb0, ta, tmin, acc[0]);
                } else {
#pragma unroll
                    for (int g = 0; g < NG; ++g) {
                        if (ta < 4) drain_tile<KB, BST, C::kN0>(tb0 + (uint32_t)(g * C::kGroupCols), ta, ta, acc[g]);
                        else drain_tile<KB, BST, kN1>(tb0 + (uint32_t)(g * C::kGroupCols + C::kN0), ta, ta, acc[g]);
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) bar_arrive(&tempty[tb]);
            return true;
        };
        // A ring of PD stages of loads in registers: stage gs + PD is requested as stage gs
        // is taken out of its slot, so PD stages of loads are in flight per warp. The slot
        // index is static (the loop is unrolled by PD): a register move would wait for its load.
        double2 ring[PD][kItems], zring[PD];
#pragma unroll
        for (int u = 0; u < PD; ++u) {
            zring[u] = make_double2(0.0, 0.0);
#pragma unroll
            for (int j = 0; j < kItems; ++j) ring[u][j] = make_double2(0.0, 0.0);
            if (!ZS && (int64_t)u < nstages) {
                load(u, ring[u]);
                if (zw) zload(u, zring[u]);
            }
        }
        bool stop = false;
        for (unsigned gs0 = 0; gs0 < (unsigned)nstages && !stop; gs0 += PD) {
#pragma unroll
          for (int u = 0; u < PD; ++u) {
            const unsigned gs = gs0 + (unsigned)u;
            if (gs >= (unsigned)nstages || failed) {
                stop = true;
                break;
            }
            double2 cur[kItems], zcur = zring[u];
            if constexpr (ZS) {
                // this lane's entries from the raw slot: column c8, rows kk and kk + 1; column 8,
                // rows zrow and zrow + 1 (z lanes); rows past n are 0
                const int slot = (int)(gs % RS);
                if (!oz_wait(smem_addr(&rfull[slot]), (uint32_t)((gs / RS) & 1), spin)) {
                    failed = 1;
                    stop = true;
                    break;
                }
                const double* raw = reinterpret_cast<const double*>(smem + NS * STG + slot * R::kSlot);
                const int64_t r0 = (s0 + (int64_t)gs) * C::kRows, left = n - r0;
                const int copied = (int)(left >= C::kRows ? C::kRows : (left & ~1ll));
                cur[0] = make_double2(0.0, 0.0);
                if (kk < copied) cur[0] = *reinterpret_cast<const double2*>(raw + c8 * R::kCol + kk);
                else if (kk < left) cur[0].x = __ldg(V + (int64_t)c8 * ldv + r0 + kk);
                zcur = make_double2(0.0, 0.0);
                if (zl) {
                    if (zrow < copied) zcur = *reinterpret_cast<const double2*>(raw + 8 * R::kCol + zrow);
                    else if (zrow < left) zcur.x = __ldg(V + 8 * ldv + r0 + zrow);
                }
                __syncwarp();
                if (lane == 0) bar_arrive(&rempty[slot]);
            } else {
#pragma unroll
                for (int j = 0; j < kItems; ++j) cur[j] = ring[u][j];
                if (gs + PD < (unsigned)nstages) {
                    load(gs + PD, ring[u]);
                    if (zw) zload(gs + PD, zring[u]);
                }
            }

            const int sb = (int)(gs % NS);
            if (gs >= NS && !oz_wait(smem_addr(&empty[sb]), (uint32_t)(((gs / NS) - 1) & 1), spin)) {
                failed = 1;
                stop = true;
                break;
            }
            unsigned char* sp = smem + sb * STG;
#pragma unroll
            for (int j = 0; j < kItems; ++j) {
                if (j < noct) {   // warp-uniform
                    const bool isv = j < noct_v;
                    const uint64_t b0 = (uint64_t)__double_as_longlong(cur[j].x);
                    const uint64_t b1 = (uint64_t)__double_as_longlong(cur[j].y);
                    uint32_t l0, h0, l1, h1;
                    if (isv && vw) {   // warp-uniform: V holds the biased fixed-point words already
                        l0 = (uint32_t)b0;
                        h0 = (uint32_t)(b0 >> 32);
                        l1 = (uint32_t)b1;
                        h1 = (uint32_t)(b1 >> 32);
                    } else {
                        oz::fixed_biased_words((uint32_t)b0, (uint32_t)(b0 >> 32), ce[j], l0, h0);
                        oz::fixed_biased_words((uint32_t)b1, (uint32_t)(b1 >> 32), ce[j], l1, h1);
                    }
                    if (isv && wout) {   // keep the words of the first nw V columns (warp-uniform test)
                        const int c = j * 8 + c8;
                        const int64_t r = (s0 + (int64_t)gs) * C::kRows + kk;
                        if (cv[j] && c < nw) {
                            uint64_t* wp = wout + (int64_t)c * ldw + r;
                            if (r + 1 < n) *reinterpret_cast<uint4*>(wp) = make_uint4(l0, h0, l1, h1);
                            else if (r < n) *reinterpret_cast<uint2*>(wp) = make_uint2(l0, h0);
                        }
                    }
                    uint32_t d[oz::kDigits];
                    digits8(l0, h0, l1, h1, d);
                    if (isv) {   // unused columns of an octet land in unused A rows
                        unsigned char* base = sp + aoff[j];
                        if (G == 0) {   // row t 16 + c of the one tile
#pragma unroll
                            for (int t = 0; t < oz::kDigits; ++t)
                                *reinterpret_cast<uint32_t*>(base + t * 2 * SBO) = d[t];
                        } else {        // tile 2 (c / 32) + t / 4, row (t % 4) 32 + c % 32
#pragma unroll
                            for (int t = 0; t < oz::kDigits; ++t)
                                *reinterpret_cast<uint32_t*>(base + (t >> 2) * C::kTile + (t & 3) * 4 * SBO) = d[t];
                        }
                        if (sym && !ZS) {   // warp-uniform; sym implies G = 0, so C::kFastB (ZS: B is A)
                            unsigned char* bb = sp + boff[j];
#pragma unroll
                            for (int t = 0; t < oz::kDigits; ++t)
                                *reinterpret_cast<uint32_t*>(bb + (uint32_t)(t * (BST / 8)) * SBO) = d[t];
                        }
                    } else if (C::kFastB) {
                        unsigned char* bb = sp + boff[j];
#pragma unroll
                        for (int t = 0; t < oz::kDigits; ++t)
                            *reinterpret_cast<uint32_t*>(bb + (uint32_t)(t * (BST / 8)) * SBO) = d[t];
                    } else {           // BST = KB = 9: unused columns go to the spare rows 72..79
                        unsigned char* bb = sp + boff[j];
#pragma unroll
                        for (int t = 0; t < oz::kDigits; ++t) {
                            const int row = cv[j] ? t * BST + bcol[j] : 8 * BST + (bcol[j] & 7);
                            *reinterpret_cast<uint32_t*>(bb + op_off<SBO>(row, kk)) = d[t];
                        }
                    }
                }
            }
            if (zw) {   // column 8 of this stage's rows zrow, zrow + 1: A row t 16 + 8 and B row t BST + 8
                const uint64_t b0 = (uint64_t)__double_as_longlong(zcur.x);
                const uint64_t b1 = (uint64_t)__double_as_longlong(zcur.y);
                uint32_t l0, h0, l1, h1;
                oz::fixed_biased_words((uint32_t)b0, (uint32_t)(b0 >> 32), ze, l0, h0);
                oz::fixed_biased_words((uint32_t)b1, (uint32_t)(b1 >> 32), ze, l1, h1);
                uint32_t d[oz::kDigits];
                digits8(l0, h0, l1, h1, d);
                if (zl) {
#pragma unroll
                    for (int t = 0; t < oz::kDigits; ++t) {
                        *reinterpret_cast<uint32_t*>(sp + op_off<SBO>(t * 16 + 8, zrow)) = d[t];
                        if (!ZS)
                            *reinterpret_cast<uint32_t*>(sp + C::kAT * C::kTile + op_off<SBO>(t * BST + 8, zrow)) = d[t];
                    }
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) bar_arrive(&full[sb]);
            // drain at the end of each chunk (kStagesPerChunk is a multiple of PD, so a chunk
            // ends in the last slot); with PD > 1 a last, partial chunk is drained after the loop
            const int sic = (int)(gs % C::kStagesPerChunk);
            if ((PD == 1 || u == PD - 1) &&
                (sic == C::kStagesPerChunk - 1 || (PD == 1 && gs + 1 == (unsigned)nstages)) &&
                !drain_chunk((int)(gs / C::kStagesPerChunk))) {
                failed = 1;
                stop = true;
                break;
            }
          }
        }
        if (PD > 1 && !failed && nstages > 0 && nstages % C::kStagesPerChunk != 0 &&
            !drain_chunk((int)((nstages - 1) / C::kStagesPerChunk)))
            failed = 1;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::kCols));
    if (failed && tid == 0) atomicExch(sc.counter + 1, 1u);

    // the CTA's exact partial sums: per (digit ta, column a, column b) in shared memory (the
    // stage buffers are free), summed over the digits, then added
    // into the 128-bit accumulators: atomicAdd of the low words, whose old value gives the
    // carry, then of the high words (addition of integers is exact and order-free)
    oz::i128* part = reinterpret_cast<oz::i128*>(smem);   // [8 digits][NG CP columns][KB]
    if (drains)
#pragma unroll
        for (int g = 0; g < NG; ++g)
#pragma unroll
            for (int b = 0; b < KB; ++b) part[(ta * NG * CP + g * CP + al_) * KB + b] = acc[g][b] >> (8 * ta);
    __syncthreads();
    for (int e = tid; e < ka * KB; e += NT) {
        const int a = e % ka, b = e / ka;
        oz::i128 s = 0;
        for (int k = 0; k < oz::kDigits; ++k) s += part[(k * NG * CP + a) * KB + b];
        const unsigned long long lo = (unsigned long long)(uint64_t)s;
        const unsigned long long hi = (unsigned long long)(uint64_t)((oz::u128)s >> 64);
        const unsigned long long old = atomicAdd(sc.acc + 2 * e, lo);
        atomicAdd(sc.acc + 2 * e + 1, hi + ((old + lo < old) ? 1ull : 0ull));
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) last = atomicAdd(sc.counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    // last CTA: one rounding per entry, then the accumulators go back to zero for the next launch
    const bool err = ((volatile unsigned*)sc.counter)[1] != 0u;
    for (int e = tid; e < ka * KB; e += NT) {
        const uint64_t lo = __ldcg(sc.acc + 2 * e), hi = __ldcg(sc.acc + 2 * e + 1);
        sc.acc[2 * e] = 0ull;
        sc.acc[2 * e + 1] = 0ull;
        const oz::i128 s = (oz::i128)(((oz::u128)hi << 64) | (oz::u128)lo);
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

// the tensor-core Gram pass keeps no per-CTA partials (its exact sums go to Scratch::acc)
int oz_partials_doubles() { return 0; }

void launch_colmax(int64_t n, const double* X, int64_t ld, int ncols, unsigned* out, cudaStream_t stream) {
    if (n <= 0 || ncols <= 0) return;
    const int per_col = std::max(1, std::min(grid_for(n, 4 * device_sms()), (4 * device_sms() + ncols - 1) / ncols));
    colmax_kernel<<<dim3(per_col, ncols), kThreads, 0, stream>>>(n, X, ld, out);
}

namespace {
template <int G, int KB>
void launch_oz(int64_t n, const double* V, int64_t ldv, int ka, const unsigned* vmax, const double* Y, int64_t ldy,
               const unsigned* ymax, Scratch sc, const Epi& epi, int gate, cudaStream_t stream, long spin, int sym,
               int vw, uint64_t* wout, int64_t ldw, int nw) {
    using C = OzCfg<G, KB>;
    constexpr bool kZ = G == 0 && KB == 9 && C::kSplitWarps == 14;   // the z-mode form exists
    static bool attr[64][2] = {};     // once per device and form
    int dev = 0;
    cudaGetDevice(&dev);
    // the z-mode form: V^T V of 9 columns whose starts are 16-byte aligned (bulk copies)
    const bool z = kZ && sym && ka == 9 && ((uintptr_t)V & 15) == 0 && (ldv & 1) == 0;
    if (dev < 0 || dev >= 64 || !attr[dev][z]) {
        if (z) cudaFuncSetAttribute(gram_oz_kernel<G, KB, kZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    ZRaw<0, 9>::kSmem);
        else cudaFuncSetAttribute(gram_oz_kernel<G, KB, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem);
        if (dev >= 0 && dev < 64) attr[dev][z] = true;
    }
    const int64_t nst = (n + C::kRows - 1) / C::kRows;
    int grid = device_sms();
    if (grid > nst) grid = (int)std::max<int64_t>(nst, 1);
    if (z)
        gram_oz_kernel<G, KB, kZ><<<grid, C::kThreads + 32, ZRaw<0, 9>::kSmem, stream>>>(
            n, V, ldv, ka, vmax, Y, ldy, ymax, sc, epi, gate, spin, sym, vw, wout, ldw, nw);
    else
        gram_oz_kernel<G, KB, false><<<grid, C::kThreads, C::kSmem, stream>>>(n, V, ldv, ka, vmax, Y, ldy, ymax, sc,
                                                                               epi, gate, spin, sym, vw, wout, ldw, nw);
}
}  // namespace

long g_oz_spin = kOzSpin;

bool launch_gram_oz(int64_t n, const double* V, int64_t ldv, int ka, const unsigned* vmax, const double* Y,
                    int64_t ldy, int kb, const unsigned* ymax, Scratch sc, const Epi& epi, int gate,
                    cudaStream_t stream, int vw, uint64_t* wout, int64_t ldw, int nw) {
    if (ka < 1 || ka > kMaxCols || kb < 1 || kb > kMaxS + 1 || n < 1 || n > ((int64_t)1 << 27) || !sc.acc) return false;
    if (((uintptr_t)V & 7) || ((uintptr_t)Y & 7)) return false;
    const int sym = (V == Y && ldv == ldy && ka == kb && !vw) ? 1 : 0;   // V^T V: split each column once
    // kept words: 16-byte stores of row pairs (even leading dimension, aligned panel)
    if (wout && (((uintptr_t)wout & 15) || (ldw & 1) || ldw < n || vw)) return false;
    switch (kb) {
#define SSTEP_OZ_CASE(KB)                                                                                       \
    case KB:                                                                                                    \
        if (ka <= 16) launch_oz<0, KB>(n, V, ldv, ka, vmax, Y, ldy, ymax, sc, epi, gate, stream, g_oz_spin, sym, vw, \
                                       wout, ldw, nw);                                                          \
        else if (ka <= 32) launch_oz<1, KB>(n, V, ldv, ka, vmax, Y, ldy, ymax, sc, epi, gate, stream, g_oz_spin, sym, \
                                            vw, wout, ldw, nw);                                                 \
        else launch_oz<2, KB>(n, V, ldv, ka, vmax, Y, ldy, ymax, sc, epi, gate, stream, g_oz_spin, sym, vw, wout, \
                              ldw, nw);                                                                         \
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

// ================================================================== block update on the tensor cores
// Yhat[:, j] = Y[:, j] - V T[:, j] for j0 <= j < j0 + KBO, in place (Alg. 4.1 step 7; the
// Gram matrix of the result is the tensor-core Gram pass's next launch). Every V column a
// is in 61-bit fixed point relative to its bound (q 2^(ea - kFrac)); T is folded with those
// scales, T'[a][j] = 2^(ea - kFrac) T[a][j], so V_ra T_aj = q_ra T'_aj, and every column j
// of T' is in fixed point relative to its own bound: T'_aj = p_aj 2^(Fj - kFrac). Then
// P_rj = 2^(Fj - kFrac) sum_a q_ra p_aj, an exact integer sum of digit products. The A
// operand holds V's digit planes (M = 128 rows, K = digit plane x column), the B operand a
// banded arrangement of T's digits: row (j, d), K position (ta, a) holds digit d - ta of
// T'_aj (zero outside 0..7), so one MMA over the whole K gives, for every output j and
// digit diagonal d = ta + tb <= 8, the exact FP32 sum over the digit pairs of that
// diagonal (at most 8 x 32 products of 2^14). The epilogue combines the 9 diagonals into
// a 128-bit integer (Horner in 256), rounds P once and forms Y - P in FP64.
namespace sstep {
namespace {

// warps 0..15 split tile t and then run the epilogue of tile t - 1 (warps w, w + 4, w + 8 and
// w + 12 share tensor-memory lane quarter w % 4 and take a quarter of the outputs each); warp
// 16 issues the MMAs
constexpr int kUpSplitWarps = 16, kUpMmaWarp = 16;
constexpr int kUpThreads = (kUpSplitWarps + 1) * 32;

constexpr int kUpRows = 128;                      // rows per tile (MMA M)
constexpr int kUpDiags = oz::kCut + 1;            // kept digit diagonals
constexpr uint32_t kUpBuf = 128;                  // tensor-memory columns per accumulator buffer

// B rows: the outputs in groups of H = ceil(KBO / 4), one group per warp of a tensor-memory
// lane quarter; group g takes rows (accumulator columns) 32 g .. 32 g + 9 H - 1, output
// j = g H + i at 32 g + 9 i + d (d the diagonal, fastest). Every group starts on the same
// boundary, so one epilogue serves all four warps of a quarter (the MMA's N grows to 32
// per group; the tensor pipe has room).
__host__ __device__ constexpr int up_h(int kbo) { return (kbo + 3) / 4; }
__host__ __device__ constexpr int up_n(int kbo) { return 32 * ((kbo + up_h(kbo) - 1) / up_h(kbo)); }
__host__ __device__ constexpr int up_row(int kbo, int j) { return 32 * (j / up_h(kbo)) + kUpDiags * (j % up_h(kbo)); }

template <int KAP, int KBO>
struct UpCfg {
    static constexpr int kK = oz::kDigits * KAP;  // K of one row: 8 digit planes of KAP columns
    static constexpr int kSbo = KAP * 128;        // bytes between 8-row groups
    static constexpr int kN = up_n(KBO);          // MMA N
    static constexpr int kA = kUpRows * kK * 2;   // one A buffer (FP16)
    static constexpr int kB = kN * kK * 2;        // B: kN rows
    static constexpr int kSmem = 2 * kA + kB;
    static_assert(kN <= (int)kUpBuf && kUpDiags * up_h(KBO) <= 32, "accumulator buffer");
    static_assert(kSmem + 4096 <= 227 * 1024, "shared memory");
};

template <int KAP, int KBO>
__global__ void __launch_bounds__(kUpThreads, 1)
    update_oz_kernel(int64_t n, const double* __restrict__ V, int64_t ldv, int ka, const unsigned* __restrict__ vmax,
                     double* Y, int64_t ldy, int j0, const double* __restrict__ T, int ldt, unsigned* bout,
                     unsigned* bout2, int nb2, const unsigned* bcopy_src, unsigned* bcopy_dst, const SolverState* st,
                     int gate, long spin, unsigned* err, int vw) {
    using C = UpCfg<KAP, KBO>;
    constexpr int SBO = C::kSbo;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[2], empty[2], tfull[2], tempty[2];
    __shared__ uint32_t tmem_base;
    __shared__ volatile int failed;
    __shared__ uint32_t exv[32];
    __shared__ unsigned fmax[KBO];
    __shared__ int fexp[KBO];
    static_assert(KBO <= 16, "the B operand has 16 rows");
    __shared__ int nonfinite;
    __shared__ double tp[32 * KBO];
    if (!gate_open(st, gate)) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* Abuf = smem;
    unsigned char* Bop = smem + 2 * C::kA;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                     "r"(2 * kUpBuf));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        failed = 0;
        nonfinite = 0;
        for (int b = 0; b < 2; ++b) {
            bar_init(&full[b], kUpSplitWarps);
            bar_init(&empty[b], 1);
            bar_init(&tfull[b], 1);
            bar_init(&tempty[b], kUpSplitWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
        if (bcopy_dst && blockIdx.x == 0) *bcopy_dst = *bcopy_src;   // the unchanged column's bound
    }
    if (tid < 32) exv[tid] = tid < ka ? oz::bound_exponent(vmax[tid]) : 0u;
    if (tid < KBO) fmax[tid] = 0u;
    // zero both A buffers and B: columns KAP > ka and the padded output rows stay zero
    for (int i = tid; i < C::kSmem / 16; i += kUpThreads) reinterpret_cast<uint4*>(smem)[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    // T' = 2^(ea - kFrac) T and the bound of each of its columns
    for (int e = tid; e < ka * KBO; e += kUpThreads) {
        const int a = e % ka, j = e / ka;
        const double t = T[a + (int64_t)(j0 + j) * ldt];
        const uint32_t ea = exv[a];
        if (ea == oz::kNonFinite || !isfinite(t)) nonfinite = 1;
        const double v = ea == 0 ? 0.0 : ldexp(t, (int)ea - oz::kFrac);
        tp[e] = v;
        atomicMax(&fmax[j], oz::abs_hiword((uint32_t)((unsigned long long)__double_as_longlong(v) >> 32)));
    }
    __syncthreads();
    if (tid < KBO) fexp[tid] = (int)oz::bound_exponent(fmax[tid]);
    __syncthreads();
    // B: row (j, d), K = 8 a + ta (column a of V, its digit ta): digit d - ta of T'_aj where
    // 0 <= d - ta <= 7, zero elsewhere, so one MMA over all of K sums each digit diagonal d
    for (int e = tid; e < ka * KBO; e += kUpThreads) {
        const int a = e % ka, j = e / ka;
        const uint64_t bits = (uint64_t)__double_as_longlong(tp[e]);
        const uint64_t w = oz::fixed_biased((uint32_t)bits, (uint32_t)(bits >> 32), (uint32_t)fexp[j]);
#pragma unroll
        for (int tb = 0; tb < oz::kDigits; ++tb) {
            const __half e16 = __int2half_rn(oz::digit(w, tb));
#pragma unroll
            for (int ta = 0; ta < oz::kDigits; ++ta)
                if (ta + tb <= oz::kCut)
                    *reinterpret_cast<__half*>(Bop + op_off<SBO>(up_row(KBO, j) + ta + tb, 8 * a + ta)) = e16;
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base, sbase = smem_addr(smem);
    const int64_t ntiles = (n + kUpRows - 1) / kUpRows;
    const int64_t t0 = ntiles * blockIdx.x / gridDim.x, t1 = ntiles * (blockIdx.x + 1) / gridDim.x;
    const int64_t nt = t1 - t0;

    if (warp == kUpMmaWarp) {
        // ---------------------------------------------------------------- MMA warp
        if (lane == 0) {
            int n_empty[2] = {0, 0}, n_tfull[2] = {0, 0};
            for (int64_t lt = 0; lt < nt && !failed; ++lt) {
                const int b = (int)(lt & 1);
                if (lt >= 2 && !oz_wait_sleep(smem_addr(&tempty[b]), (uint32_t)(((lt >> 1) - 1) & 1), spin)) {
                    failed = 1;
                    break;
                }
                if (!oz_wait_sleep(smem_addr(&full[b]), (uint32_t)((lt >> 1) & 1), spin)) {
                    failed = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t ab = sbase + (uint32_t)(b * C::kA), bb = sbase + (uint32_t)(2 * C::kA);
                const uint32_t dt = tmem + (uint32_t)b * kUpBuf;
                const int nks = (ka + 1) >> 1;   // K steps of 16 = two columns; the rest is zero in B
#pragma unroll
                for (int ks = 0; ks < C::kK / 16; ++ks)
                    if (ks < nks)
                        mma_f16(dt, op_desc<SBO>(ab + (uint32_t)(ks * 256)), op_desc<SBO>(bb + (uint32_t)(ks * 256)),
                                oz_idesc(C::kN), ks > 0 ? 1u : 0u);
                mma_commit(&empty[b]);
                ++n_empty[b];
                mma_commit(&tfull[b]);
                ++n_tfull[b];
            }
            for (int b = 0; b < 2; ++b)
                if (n_empty[b]) oz_wait(smem_addr(&empty[b]), (uint32_t)((n_empty[b] - 1) & 1), kOzSpin);
            for (int b = 0; b < 2; ++b)
                if (n_tfull[b]) oz_wait(smem_addr(&tfull[b]), (uint32_t)((n_tfull[b] - 1) & 1), kOzSpin);
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------------------- split + epilogue warps
        // split: warp w owns rows 8 w .. 8 w + 7 of every tile; item i holds columns 4 i .. 4 i + 3,
        // lane: row 8 w + (lane & 7) of column 4 i + (lane >> 3). With K = 8 a + t, the 8 digits
        // of one entry are one 16-byte row of a core matrix: one store per entry. Columns past
        // ka read column 0 (finite digits against B's zeros); items past them are skipped and
        // stay zero from the initial clear.
        constexpr int kIt = KAP / 4;
        const int rr = warp * 8 + (lane & 7), csub = lane >> 3;
        const int nit = (ka + 3) >> 2;   // items with a column < ka (warp-uniform)
        const double* pa[kIt];
        uint32_t ea[kIt];
        // byte offset of the entry's digit row in an A buffer: item i adds 4 columns of 128 B
        const uint32_t soff0 = op_off<SBO>(rr, 8 * csub);
#pragma unroll
        for (int i = 0; i < kIt; ++i) {
            const int a = 4 * i + csub, ac = a < ka ? a : 0;
            pa[i] = V + (int64_t)ac * ldv + t0 * kUpRows + rr;
            ea[i] = exv[ac];
        }
        // epilogue: rows 32 q + lane of a tile; warp group g = warp / 4 takes the outputs
        // g H .. g H + H - 1, whose accumulators start at column 32 g (one code path for all)
        constexpr int H = (KBO + 3) / 4;
        const int q = warp & 3, g = warp >> 2;
        unsigned bm[H];
#pragma unroll
        for (int j = 0; j < H; ++j) bm[j] = 0;
        auto load = [&](int64_t lt, double (&buf)[kIt]) {
            const int64_t off = lt * kUpRows;
            const bool in = (t0 + lt) * kUpRows + rr < n;
#pragma unroll
            for (int i = 0; i < kIt; ++i)
                if (i < nit) buf[i] = in ? __ldg(pa[i] + off) : 0.0;
        };
        // this thread's Y entries of tile lt (loaded a whole split ahead of their use)
        double yv[H];
        auto load_y = [&](int64_t lt) {
            const int64_t r = (t0 + lt) * kUpRows + q * 32 + lane;
#pragma unroll
            for (int j = 0; j < H; ++j) {
                const int jj = g * H + j;
                yv[j] = (r < n && jj < KBO) ? Y[(int64_t)(j0 + jj) * ldy + r] : 0.0;
            }
        };
        // epilogue of tile lt: Yhat = Y - P for this thread's row and outputs
        auto epilogue = [&](int64_t lt) -> bool {
            const int jo = g * H;   // this warp's outputs jo .. jo + H - 1, columns 32 g + 9 i + d
            const int b = (int)(lt & 1);
            const int64_t r = (t0 + lt) * kUpRows + q * 32 + lane;
            if (!oz_wait(smem_addr(&tfull[b]), (uint32_t)((lt >> 1) & 1), spin)) return false;
            asm volatile("tcgen05.fence::after_thread_sync;");
            // Q = sum_d S_d 256^(8 - d) = Qh 2^32 + Ql: Horner in 64 bits over the diagonals
            // 0..4 (Qh < 2^54) and 5..8 (Ql < 2^47), then one 128-bit step
            // Each S is an exact integer with |S| <= 2^22, so S + 1.5 2^23 is exact and its FP32
            // bits are 0x4B400000 + S: the sums run over those bits (FP32 add, integer Horner)
            // and the constant they add is taken off at the end.
            constexpr unsigned kMagic = 0x4B400000u;
            unsigned long long Qh[H], Ql[H];
#pragma unroll
            for (int j = 0; j < H; ++j) Qh[j] = Ql[j] = 0;
            // the group's 32 accumulator columns from 32 g (output jo + i, diagonal d at 9 i + d)
            constexpr int NR = 32;
            uint32_t rv[NR];
            if (jo < KBO) {   // warp-uniform (a warp past the last group has no outputs)
                const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)b * kUpBuf + (uint32_t)(32 * g);
                tmem_ld<NR>(ta, rv);
            }
#pragma unroll
            for (int d = 0; d < kUpDiags; ++d) {
#pragma unroll
                for (int j = 0; j < H; ++j) {
                    const unsigned mS = jo + j < KBO
                                            ? (unsigned)__float_as_int(__uint_as_float(rv[kUpDiags * j + d]) + 12582912.0f)
                                            : kMagic;
                    if (d < 5) Qh[j] = Qh[j] * 256 + mS;
                    else Ql[j] = Ql[j] * 256 + mS;
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) bar_arrive(&tempty[b]);
            if (r < n) {
#pragma unroll
                for (int j = 0; j < H; ++j) {
                    if (jo + j < KBO) {
                        const long long qh = (long long)(Qh[j] - (unsigned long long)kMagic * 0x0101010101ull);
                        const long long ql = (long long)(Ql[j] - (unsigned long long)kMagic * 0x01010101ull);
                        const oz::i128 Q = ((oz::i128)qh << 32) + (oz::i128)ql;
                        const int fj = fexp[jo + j];
                        const double P = (nonfinite || fj == (int)oz::kNonFinite)
                                             ? __longlong_as_double(0x7FF8000000000000ll)
                                             : oz::i128_to_double_int(Q, 8 * (2 * (oz::kDigits - 1) - oz::kCut) + fj -
                                                                             oz::kFrac);
                        const double yh = yv[j] - P;
                        Y[(int64_t)(j0 + jo + j) * ldy + r] = yh;
                        bm[j] = max(bm[j],
                                    oz::abs_hiword((uint32_t)((unsigned long long)__double_as_longlong(yh) >> 32)));
                    }
                }
            }
            return true;
        };
        auto run_epilogue = [&](int64_t lt) -> bool { return epilogue(lt); };
        double cur[kIt];
        if (nt > 0) load(0, cur);
        for (int64_t lt = 0; lt < nt; ++lt) {
            if (failed) break;
            double nxt[kIt];
            if (lt + 1 < nt) load(lt + 1, nxt);

            if (lt >= 1) load_y(lt - 1);   // consumed by the epilogue after this split
            const int b = (int)(lt & 1);
            if (lt >= 2 && !oz_wait(smem_addr(&empty[b]), (uint32_t)(((lt >> 1) - 1) & 1), spin)) {
                failed = 1;
                break;
            }
            unsigned char* ap = Abuf + b * C::kA;
#pragma unroll
            for (int i = 0; i < kIt; ++i) {
                if (i < nit) {   // warp-uniform
                    const uint64_t bits = (uint64_t)__double_as_longlong(cur[i]);
                    uint32_t wl = (uint32_t)bits, wh = (uint32_t)(bits >> 32);   // vw: the words already
                    if (!vw) oz::fixed_biased_words((uint32_t)bits, (uint32_t)(bits >> 32), ea[i], wl, wh);
                    uint4 v;
                    digit_row8(wl, wh, v);
                    *reinterpret_cast<uint4*>(ap + soff0 + i * 4 * 128) = v;
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) bar_arrive(&full[b]);
#pragma unroll
            for (int i = 0; i < kIt; ++i) cur[i] = nxt[i];
            if (lt >= 1 && !run_epilogue(lt - 1)) {   // the previous tile, while this tile's MMAs run
                failed = 1;
                break;
            }
        }
        if (!failed && nt > 0) {
            load_y(nt - 1);
            if (!run_epilogue(nt - 1)) failed = 1;
        }
#pragma unroll
        for (int j = 0; j < H; ++j) {
            const int jj = g * H + j;
            const unsigned m = __reduce_max_sync(0xffffffffu, bm[j]);
            if (lane == 0 && m && jj < KBO) {
                if (bout) atomicMax(bout + jj, m);
                if (bout2 && jj < nb2) atomicMax(bout2 + jj, m);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kUpBuf));
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

template <int KAP, int KBO>
void launch_up(int64_t n, const double* V, int64_t ldv, int ka, const unsigned* vmax, double* Y, int64_t ldy, int j0,
               const double* T, int ldt, unsigned* bout, unsigned* bout2, int nb2, const unsigned* bsrc,
               unsigned* bdst, const SolverState* st, int gate, cudaStream_t stream, unsigned* err, int vw) {
    using C = UpCfg<KAP, KBO>;
    static bool attr[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attr[dev]) {
        cudaFuncSetAttribute(update_oz_kernel<KAP, KBO>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem);
        if (dev >= 0 && dev < 64) attr[dev] = true;
    }
    const int64_t ntiles = (n + kUpRows - 1) / kUpRows;
    int grid = device_sms();
    if (grid > ntiles) grid = (int)std::max<int64_t>(ntiles, 1);
    update_oz_kernel<KAP, KBO><<<grid, kUpThreads, C::kSmem, stream>>>(n, V, ldv, ka, vmax, Y, ldy, j0, T, ldt, bout,
                                                                        bout2, nb2, bsrc, bdst, st, gate, g_oz_spin,
                                                                        err, vw);
}

}  // namespace

bool launch_update_oz(int64_t n, const double* V, int64_t ldv, int ka, const unsigned* vmax, double* Y, int64_t ldy,
                      int j0, int kbo, const double* T, int ldt, unsigned* bout, unsigned* bout2, int nb2,
                      const unsigned* bcopy_src, unsigned* bcopy_dst, const SolverState* st, int gate,
                      cudaStream_t stream, unsigned* err, int vw) {
    if (ka < 1 || ka > 32 || kbo < 1 || kbo > kMaxS + 1 || n < 1 || n > ((int64_t)1 << 27)) return false;
    const bool k16 = ka <= 16;
    switch (kbo) {
#define SSTEP_UP_CASE(KBO)                                                                                      \
    case KBO:                                                                                                   \
        if (k16) launch_up<16, KBO>(n, V, ldv, ka, vmax, Y, ldy, j0, T, ldt, bout, bout2, nb2, bcopy_src,       \
                                    bcopy_dst, st, gate, stream, err, vw);                                      \
        else launch_up<32, KBO>(n, V, ldv, ka, vmax, Y, ldy, j0, T, ldt, bout, bout2, nb2, bcopy_src,           \
                                bcopy_dst, st, gate, stream, err, vw);                                          \
        return true;
        SSTEP_UP_CASE(1)
        SSTEP_UP_CASE(2)
        SSTEP_UP_CASE(3)
        SSTEP_UP_CASE(4)
        SSTEP_UP_CASE(5)
        SSTEP_UP_CASE(6)
        SSTEP_UP_CASE(7)
        SSTEP_UP_CASE(8)
        SSTEP_UP_CASE(9)
#undef SSTEP_UP_CASE
        default: return false;
    }
}

}  // namespace sstep
