// Shared device-side definitions of the s-step library (FP64 path).
//
// Everything here is plain CUDA C++ for sm_103a. The operator is the
// (2d+1)-point stencil of Sec. 1 / Sec. 5; the reductions implement the
// "simultaneous inner products" of Sec. 1 as one grid pass with a fixed-order
// second stage, so every result is bitwise reproducible run to run.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sstep.h"

namespace sstep {

constexpr int kThreads = 256;          // threads per CTA of every streaming kernel
constexpr int kWarps = kThreads / 32;
constexpr int kMaxS = SSTEP_MAX_S;
constexpr int kMaxM = SSTEP_MAX_M;
constexpr int kMaxCols = SSTEP_MAX_COLS;

// ------------------------------------------------------------------ operator
// Row p: a0 u_p + sum_d (am_d u_{p-e_d} + ap_d u_{p+e_d}), zero outside the grid.
struct StencilDesc {
    int dim;
    int nx, ny, nz;
    int64_t n;
    int variable;            // 0: constant coefficients in c[], 1: per-point fields in f[]
    double c[7];             // a0, am_x, ap_x, am_y, ap_y, am_z, ap_z
    const double* f[7];      // same order, device arrays of n (variable == 1)
    // the same coefficients split into float pairs (hi + lo = c to 48 bits) for the
    // mixed-precision kernels, so no kernel converts FP64 constants on the slow pipe
    float ch[7], cl[7];
    const float2* fdf[7];    // variable coefficients as float pairs (variable == 1)
};

__device__ __forceinline__ double coef(const StencilDesc& A, int q, int64_t p) {
    return A.variable ? __ldg(A.f[q] + p) : A.c[q];
}

// (A v)_p, summed centre, x-, x+, y-, y+, z-, z+ with fused multiply-adds.
__device__ __forceinline__ double stencil_row(const StencilDesc& A, const double* __restrict__ v,
                                              int64_t p, int x, int y, int z) {
    double acc = coef(A, 0, p) * __ldg(v + p);
    if (x > 0) acc = fma(coef(A, 1, p), __ldg(v + p - 1), acc);
    if (x < A.nx - 1) acc = fma(coef(A, 2, p), __ldg(v + p + 1), acc);
    if (y > 0) acc = fma(coef(A, 3, p), __ldg(v + p - A.nx), acc);
    if (y < A.ny - 1) acc = fma(coef(A, 4, p), __ldg(v + p + A.nx), acc);
    if (A.dim == 3) {
        const int64_t pl = (int64_t)A.nx * A.ny;
        if (z > 0) acc = fma(coef(A, 5, p), __ldg(v + p - pl), acc);
        if (z < A.nz - 1) acc = fma(coef(A, 6, p), __ldg(v + p + pl), acc);
    }
    return acc;
}

// ------------------------------------------------------------------ solver state
// Lives in device memory; scalars first so the host can copy the header alone.
struct SolverState {
    // ---- header (copied to the host once per cycle / batch)
    int active;        // 1 while the solve runs
    int building;      // 1 while the current cycle still adds blocks (GMRES) / steps (Omin)
    int status;        // sstep_status
    int cycles;
    int iters;
    int matvecs;
    int K;             // basis columns in the current cycle's least-squares problem
    int hist_len;
    int confirm;       // Orthomin: the updated residual reached tol; recompute explicitly
    int pad_;
    double relres;     // last explicit relres
    double est;        // last least-squares estimate / updated residual (relative)
    // ---- parameters
    int s, m, k, nb;
    int max_cycles, max_iters, hist_cap, pad2_;
    double nf, tol, sigma;
    // ---- per-cycle scalars
    double beta;       // ||r0||
    double vscale;     // 1 / norm of the pending raw start vector
    double nu;         // ||u|| of the last block (GMRES) / hn (standard GMRES)
    // ---- small arrays (device pointers into the workspace)
    double* L;         // GMRES: nb blocks of s x s upper Cholesky factors (col-major, ld s)
    double* T;         // projection coefficients, m x (s+1) col-major (ld m); Omin: B blocks
    double* S;         // s
    double* G;         // (m+1) x m Hessenberg G, col-major (ld m+1)
    double* R;         // (m+1) x m Givens-reduced L G
    double* gc;        // m rotation cosines
    double* gs;        // m rotation sines
    double* g;         // m+1 right-hand side
    double* y;         // m least-squares solution
    double* hist;      // hist_cap residual history entries
    double* C;         // reduced Gram output (up to kMaxCols x (kMaxS+1))
    double* a;         // Omin: s step coefficients
    double* theta;     // s shifts of the Newton basis (zero: the monomial powers)
};

// ------------------------------------------------------------------ reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    return v;
}

// Reduce NV per-thread values over the CTA into red[0..NV) (shared), fixed order.
template <int NV>
__device__ __forceinline__ void block_reduce(double (&acc)[NV], double* red /* kWarps*NV shared */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        double t = warp_sum(acc[v]);
        if (lane == 0) red[warp * NV + v] = t;
    }
    __syncthreads();
    for (int v = threadIdx.x; v < NV; v += blockDim.x) {
        double t = 0.0;
        for (int w = 0; w < kWarps; ++w) t += red[w * NV + v];
        red[kWarps * NV + v] = t;   // result area after the per-warp sums
    }
    __syncthreads();
}

// Publish this CTA's partial vector and decide whether it is the last CTA of
// the grid to arrive. Returns true in every thread of the last CTA, which then
// reads all partials (in CTA order) for the deterministic second stage.
__device__ __forceinline__ bool publish_partial(const double* red, int nv, double* partials,
                                                unsigned* counter) {
    __shared__ bool last;
    const int cta = blockIdx.x + blockIdx.y * gridDim.x;
    for (int v = threadIdx.x; v < nv; v += blockDim.x) partials[(int64_t)cta * nv + v] = red[v];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned total = gridDim.x * gridDim.y;
        last = (atomicAdd(counter, 1u) == total - 1);
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

__device__ __forceinline__ double ld_cg(const double* p) { return __ldcg(p); }

// ------------------------------------------------------------------ launch helpers
int device_sms();   // multiprocessors of the current device, queried once per device (ozaki.cu)

inline int grid_for(int64_t n, int max_ctas) {
    int64_t need = (n + kThreads - 1) / kThreads;
    if (need < 1) need = 1;
    return (int)(need < max_ctas ? need : max_ctas);
}

}  // namespace sstep
