// Host emulation of the tensor-core Gram pass (test infrastructure).
//
// Compiles the library's fixed-point helpers (csrc/ozaki.cuh) for the host and runs the
// same arithmetic as the kernel with plain integer loops: column bounds, the 53-bit
// fixed-point value of every entry, its seven balanced digits, the digit pairs kept, the
// exact 128-bit sums and the one rounding. Every sum is an exact integer, so the kernel's
// result must equal this emulation bit for bit.
#include <stdint.h>
#include <string.h>

#include "ozaki.cuh"

using namespace sstep::oz;

static uint32_t column_bound(const double* x, int64_t n) {
    uint32_t m = 0;
    for (int64_t i = 0; i < n; ++i) {
        uint64_t b;
        memcpy(&b, x + i, 8);
        const uint32_t h = abs_hiword((uint32_t)(b >> 32));
        if (h > m) m = h;
    }
    return bound_exponent(m);
}

static uint64_t biased(double x, uint32_t ex) {
    uint64_t b;
    memcpy(&b, &x, 8);
    return fixed_biased((uint32_t)b, (uint32_t)(b >> 32), ex);
}

extern "C" {

// bound exponent of a column
uint32_t oz_bound(const double* x, int64_t n) { return column_bound(x, n); }

// the seven digits (top first) of each entry for a given bound exponent
void oz_digits(const double* x, int64_t n, uint32_t ex, int* digits) {
    for (int64_t i = 0; i < n; ++i) {
        const uint64_t w = biased(x[i], ex);
        for (int t = 0; t < kDigits; ++t) digits[i * kDigits + t] = digit(w, t);
    }
}

// C = V^T Y (V: n x ka, Y: n x kb, both column-major with leading dimension n; C: ka x kb
// column-major) keeping the digit pairs with t_a + t_b <= cut (the library keeps kCut)
void oz_gram(int64_t n, const double* V, int ka, const double* Y, int kb, int cut, double* C) {
    for (int a = 0; a < ka; ++a) {
        const uint32_t ea = column_bound(V + a * n, n);
        for (int b = 0; b < kb; ++b) {
            const uint32_t eb = column_bound(Y + b * n, n);
            i128 T = 0;
            for (int64_t r = 0; r < n; ++r) {
                const uint64_t wa = biased(V[a * n + r], ea), wb = biased(Y[b * n + r], eb);
                for (int ta = 0; ta < kDigits; ++ta)
                    for (int tb = 0; tb < kDigits; ++tb) {
                        if (ta + tb > cut) continue;
                        const int sh = 8 * (kCut - ta - tb);
                        const i128 p = (i128)((int64_t)digit(wa, ta) * digit(wb, tb));
                        T += sh >= 0 ? p << sh : p >> (-sh);   // cut > kCut: finer pairs, truncated
                    }
            }
            C[a + b * ka] = (ea == kNonFinite || eb == kNonFinite) ? __builtin_nan("") : i128_to_double(T, gram_scale_exp(ea, eb));
        }
    }
}
}

extern "C" {
// the 64-bit and the 32-bit-word forms of the biased fixed-point word of each entry
void oz_biased_both(const double* x, int64_t n, uint32_t ex, uint64_t* out) {
    for (int64_t i = 0; i < n; ++i) {
        uint64_t b;
        memcpy(&b, x + i, 8);
        out[2 * i] = fixed_biased((uint32_t)b, (uint32_t)(b >> 32), ex);
        uint32_t wl, wh;
        fixed_biased_words((uint32_t)b, (uint32_t)(b >> 32), ex, wl, wh);
        out[2 * i + 1] = ((uint64_t)wh << 32) | wl;
    }
}

// both roundings of v 2^e2 for v = hi 2^64 + lo (two's complement): the FP64 reference and
// the integer-only one the kernels use
void oz_round_both(uint64_t hi, uint64_t lo, int e2, double* out) {
    const i128 v = (i128)(((u128)hi << 64) | (u128)lo);
    out[0] = i128_to_double(v, e2);
    out[1] = i128_to_double_int(v, e2);
}
}
