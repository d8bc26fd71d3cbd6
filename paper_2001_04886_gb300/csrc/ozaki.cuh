// Exact fixed-point digit arithmetic for FP64 inner products on the tensor cores.
//
// The Gram pass of the s-step block (Sec. 1: the 2s inner products computed at once;
// Alg. 4.1 steps 4-5) is a tall-skinny contraction C = V^T Y. GB300 issues two FP64
// FMAs per clock per SM, so this file represents FP64 columns exactly enough in small
// integers that the FP16 tensor cores can do the contraction with no rounding at all
// (the error-free splitting of Ozaki, Ogita, Oishi and Rump, "Error-free transformations
// of matrix multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 59, 2012, in its fixed-point form):
//
//   * every column has a power-of-two bound: ex_max, the largest biased exponent of its
//     entries, so |x| < 2^(ex_max - 1022) for every entry x;
//   * x is written as the integer q = trunc(x 2^(1083 - ex_max)), |q| < 2^61 (61-bit fixed
//     point relative to the column bound: the error is below 2^-61 of the bound);
//   * q = sum_{i=0..7} d_i 256^i with balanced digits d_i in [-128, 127]: the bytes of
//     w = q + 0x8080808080808080 minus 128 (the top digit d_7 lies in [-32, 32]);
//   * a digit is an integer of at most 8 bits, exact in FP16, and a product of two digits
//     is at most 2^14, so the FP32 accumulation of the tensor cores is exact for up to
//     1024 rows (2^24); sums of more rows are drained into 128-bit integers;
//   * of the 64 digit pairs, the 45 with t_a + t_b <= 8 (t = 7 - i counts from the top) are
//     kept; per row the dropped ones weigh less than 2^-65 of the product of the column
//     bounds (the truncation of x and y to q costs up to 2^-61 of each bound). The bounds
//     can exceed most entries of a column by far (one large entry among small ones), so
//     both terms are kept well below FP64's unit roundoff per row.
//
// Every sum is then an exact integer, independent of the order of the rows and of the
// grid, and the result is rounded to FP64 once. The functions here are plain integer
// arithmetic and compile for the host as well (the CPU tests run them).
#pragma once

#include <math.h>
#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define OZ_HD __host__ __device__ __forceinline__
#else
#define OZ_HD inline
#endif

namespace sstep {
namespace oz {

constexpr int kDigits = 8;                          // balanced base-256 digits per value
constexpr int kCut = 8;                             // keep digit pairs with t_a + t_b <= kCut
constexpr uint64_t kBias = 0x8080808080808080ull;   // 128 in each of the 8 digit bytes
constexpr int kFrac = 1083;                         // x = q 2^(ex_max - kFrac)
constexpr int kChunkRows = 1024;                  // rows per exact FP32 accumulation
constexpr uint32_t kNonFinite = 0x7FF;            // ex_max of a column holding Inf or NaN

// The column bound record of one entry: the high word of |x|. Its maximum over a column
// (an unsigned max: the exponent field sits above the mantissa bits) gives ex_max.
OZ_HD uint32_t abs_hiword(uint32_t hi) { return hi & 0x7FFFFFFFu; }
OZ_HD uint32_t bound_exponent(uint32_t max_hiword) { return max_hiword >> 20; }

// w = q + kBias for the entry (lo, hi) of a column with bound exponent ex_max: the 53-bit
// significand moved up 8 bits and down by the entry's distance to the bound (entries
// with a zero exponent field, zero and subnormal, count as 0; so do entries more than 63
// binades below the bound).
OZ_HD uint64_t fixed_biased(uint32_t lo, uint32_t hi, uint32_t ex_max) {
    const uint32_t ex = (hi >> 20) & 0x7FFu;
    const uint32_t sh = ex_max - ex;
    const uint64_t m = ((uint64_t)((hi & 0xFFFFFu) | 0x100000u) << 32) | lo;
    const uint64_t q = (ex == 0 || sh > 63u) ? 0ull : ((m << 8) >> sh);
    const uint64_t s = (uint64_t)(int64_t)((int32_t)hi >> 31);   // all ones for a negative entry
    return (q ^ s) + kBias + (s & 1ull);                          // two's complement sign, then the bias
}

// Funnel shifts on 32-bit words: the low word of (hi:lo) >> min(sh, 32), and the high
// word of (hi:lo) << sh for sh < 32 (one instruction each on the device)
OZ_HD uint32_t fshr_clamp(uint32_t lo, uint32_t hi, uint32_t sh) {
#ifdef __CUDA_ARCH__
    return __funnelshift_rc(lo, hi, sh);
#else
    const uint64_t v = ((uint64_t)hi << 32) | lo;
    return (uint32_t)(v >> (sh < 32u ? sh : 32u));
#endif
}
OZ_HD uint32_t fshl(uint32_t lo, uint32_t hi, uint32_t sh) {
#ifdef __CUDA_ARCH__
    return __funnelshift_l(lo, hi, sh);
#else
    const uint64_t v = ((uint64_t)hi << 32) | lo;
    return (uint32_t)((v << (sh & 31u)) >> 32);
#endif
}

// fixed_biased in 32-bit words (the kernels' form): the same w = q + kBias, returned as
// its low and high words. The significand moved up 8 bits is (h:l); it moves down by
// sh = ex_max - ex in two clamped steps of at most 32 (sh = 64 for a zero exponent field,
// which leaves 0); a negative entry is complemented into the bias add (w = (q ^ s) + kBias
// + (s & 1) with s the sign mask), one 32-bit add with carry per word.
OZ_HD void fixed_biased_words(uint32_t lo, uint32_t hi, uint32_t ex_max, uint32_t& wlo, uint32_t& whi) {
    const uint32_t ex = (hi >> 20) & 0x7FFu;
    const uint32_t sh = ex ? ex_max - ex : 64u;
    const uint32_t mh = (hi & 0xFFFFFu) | 0x100000u;
    uint32_t h = fshl(lo, mh, 8u), l = lo << 8;
    const uint32_t s1 = sh < 32u ? sh : 32u, s2 = sh - s1;
    l = fshr_clamp(l, h, s1);
    h = fshr_clamp(h, 0u, s1);
    l = fshr_clamp(l, h, s2);
    h = fshr_clamp(h, 0u, s2);
    const uint32_t sm = (uint32_t)((int32_t)hi >> 31);   // all ones for a negative entry
    const uint64_t lo_sum = (uint64_t)(l ^ sm) + 0x80808080u + (sm & 1u);
    wlo = (uint32_t)lo_sum;
    whi = (h ^ sm) + 0x80808080u + (uint32_t)(lo_sum >> 32);
}

// digit t (0 = top) of a biased word
OZ_HD int digit(uint64_t w, int t) { return (int)((w >> (8 * (kDigits - 1 - t))) & 0xFFu) - 128; }

// weight exponent (in bytes) of the pair (t_a, t_b) after the common factor 256^(14 - kCut)
OZ_HD int pair_shift_bytes(int ta, int tb) { return kCut - ta - tb; }

// x = q 2^(ex_max - kFrac) and the pair (t_a, t_b) weighs 256^(14 - t_a - t_b): a Gram entry
// is C_ab = T 2^scale_exp with T the sum of the kept digit-pair sums S_(ta,tb) 256^(kCut - ta - tb)
OZ_HD int gram_scale_exp(uint32_t ea, uint32_t eb) {
    return (int)ea + (int)eb - 2 * kFrac + 8 * (2 * (kDigits - 1) - kCut);
}

typedef __int128 i128;
typedef unsigned __int128 u128;

OZ_HD int clz64(uint64_t v) {
#ifdef __CUDA_ARCH__
    return __clzll((long long)v);
#else
    return v ? __builtin_clzll(v) : 64;
#endif
}

// round v 2^e2 to the nearest double (ties to even), one rounding; 0 for v = 0
OZ_HD double i128_to_double(i128 v, int e2) {
    if (v == 0) return 0.0;
    const bool neg = v < 0;
    u128 u = neg ? (u128)0 - (u128)v : (u128)v;
    const uint64_t hi = (uint64_t)(u >> 64), lo = (uint64_t)u;
    const int lz = hi ? clz64(hi) : 64 + clz64(lo);
    u <<= lz;                                            // top bit at position 127
    uint64_t top = (uint64_t)(u >> 64);
    top |= ((uint64_t)u != 0ull) ? 1ull : 0ull;          // sticky bit: the u64 -> f64 rounding stays exact
    const double d = (double)top;                        // rounds to 53 bits
    const double r = ldexp(d, 64 - lz + e2);
    return neg ? -r : r;
}

// The same rounding with integer operations only (no FP64 instruction): normalise, round
// the top 53 bits to nearest even with a sticky bit, and assemble sign, exponent and
// significand. Results outside the normal range fall back to i128_to_double.
OZ_HD double i128_to_double_int(i128 v, int e2) {
    if (v == 0) return 0.0;
    const uint64_t sign = v < 0 ? 0x8000000000000000ull : 0ull;
    u128 u = v < 0 ? (u128)0 - (u128)v : (u128)v;
    const uint64_t hi = (uint64_t)(u >> 64), lo = (uint64_t)u;
    const int lz = hi ? clz64(hi) : 64 + clz64(lo);
    u <<= lz;
    const uint64_t top = (uint64_t)(u >> 64);
    const bool sticky = (uint64_t)u != 0ull;
    uint64_t m = top >> 11;                       // 53 bits, the leading one at bit 52
    const uint64_t r = top & 0x7FFull;
    if (r > 0x400ull || (r == 0x400ull && (sticky || (m & 1ull)))) ++m;
    int ex = 127 - lz + e2 + 1023;                // the value is m 2^(127 - lz + e2 - 52)
    if (m >> 53) {                                // rounding carried into bit 53
        m >>= 1;
        ++ex;
    }
    if (ex <= 0 || ex >= 2047) return i128_to_double(v, e2);
    const uint64_t bits = sign | ((uint64_t)ex << 52) | (m & 0xFFFFFFFFFFFFFull);
    double d;
    memcpy(&d, &bits, 8);
    return d;
}

}  // namespace oz
}  // namespace sstep
