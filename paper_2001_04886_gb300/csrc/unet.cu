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
#include <vector>

#include "../../include/sstep.h"

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

// dW[co][ci][k] = sum_{b,y,x} g[b,co,y,x] in[b,ci,y+ky-1,x+kx-1], one CTA per (ci, co):
// each thread sums its pixels, then a fixed-order CTA reduction.
__global__ void __launch_bounds__(kT) conv3x3_wgrad_kernel(const float* __restrict__ in, int Cin,
                                                           const float* __restrict__ g, int Cout, int B, int H, int Wd,
                                                           float* __restrict__ dW) {
    const int ci = blockIdx.x, co = blockIdx.y;
    const int64_t plane = (int64_t)H * Wd, npix = (int64_t)B * plane;
    float acc[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[k] = 0.f;
    for (int64_t p = threadIdx.x; p < npix; p += kT) {
        const int b = (int)(p / plane);
        const int64_t rem = p - (int64_t)b * plane;
        const int y = (int)(rem / Wd), x = (int)(rem - (int64_t)y * Wd);
        const float gv = g[((int64_t)b * Cout + co) * plane + rem];
        const float* src = in + ((int64_t)b * Cin + ci) * plane;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const int yy = y + k / 3 - 1, xx = x + k % 3 - 1;
            const float v = (yy >= 0 && yy < H && xx >= 0 && xx < Wd) ? src[(int64_t)yy * Wd + xx] : 0.f;
            acc[k] = fmaf(gv, v, acc[k]);
        }
    }
    __shared__ float red[kT / 32][9];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        float t = acc[k];
        for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
        if (lane == 0) red[warp][k] = t;
    }
    __syncthreads();
    if (threadIdx.x < 9) {
        float t = 0.f;
        for (int w = 0; w < kT / 32; ++w) t += red[w][threadIdx.x];
        dW[((int64_t)co * Cin + ci) * 9 + threadIdx.x] = t;
    }
}

// db[c] = sum_{b,y,x} g[b,c,y,x]   (one CTA per channel)
__global__ void __launch_bounds__(kT) bias_grad_kernel(const float* __restrict__ g, int C, int B, int64_t plane,
                                                       float* __restrict__ db) {
    const int c = blockIdx.x;
    float t = 0.f;
    for (int64_t p = threadIdx.x; p < (int64_t)B * plane; p += kT) {
        const int b = (int)(p / plane);
        t += g[((int64_t)b * C + c) * plane + (p - (int64_t)b * plane)];
    }
    __shared__ float red[kT / 32];
    for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < kT / 32; ++w) s += red[w];
        db[c] = s;
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
__global__ void conv1x1_wgrad_kernel(const float* __restrict__ g, const float* __restrict__ in, int C, int B,
                                     int64_t plane, float* __restrict__ dW) {
    const int c = blockIdx.x;
    float t = 0.f;
    for (int64_t p = threadIdx.x; p < (int64_t)B * plane; p += kT) {
        const int b = (int)(p / plane);
        t = fmaf(g[p], in[((int64_t)b * C + c) * plane + (p - (int64_t)b * plane)], t);
    }
    __shared__ float red[kT / 32];
    for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < kT / 32; ++w) s += red[w];
        dW[c] = s;
    }
}

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
    return (int)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
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
        conv1x1_wgrad_kernel<<<c.cin, kT, 0, s>>>(g, in, c.cin, B, plane, dW);
        bias_grad_kernel<<<1, kT, 0, s>>>(g, 1, B, plane, db);
        if (din) conv1x1_dgrad_kernel<WT><<<blocks_for(B * plane), kT, 0, s>>>(g, c.cin, W, din, B, plane);
        return;
    }
    conv3x3_wgrad_kernel<<<dim3(c.cin, c.cout), kT, 0, s>>>(in, c.cin, g, c.cout, B, H, Wd, dW);
    bias_grad_kernel<<<c.cout, kT, 0, s>>>(g, c.cout, B, plane, db);
    if (din) {
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
