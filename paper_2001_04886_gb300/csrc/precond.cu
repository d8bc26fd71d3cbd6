// ILU(0) in red-black ordering as a right preconditioner of s-step GMRES.
//
// Red points have x + y + z even. Every stencil neighbour of a point has the other
// colour, so with the red points first A = [[D_r, E], [F, D_b]] (D_r, D_b diagonal) and
// ILU(0) (no fill beyond the sparsity of A) is L = [[I, 0], [F D_r^-1, I]],
// U = [[D_r, E], [0, D~_b]] with D~_b = D_b - diag(F D_r^-1 E). M^-1 v is two parallel
// half-sweeps: black points w_b = (v_b - sum_r A[b, r] v_r / a0_r) / d~_b, then red points
// w_r = (v_r - sum_b A[r, b] w_b) / a0_r. (The paper preconditions with ILU(0) in the
// natural ordering, whose triangular solves run in 3N - 2 sequential hyperplanes.)
#include "kernels.cuh"

namespace sstep {

namespace {

// neighbour q in 1..6 (x-, x+, y-, y+, z-, z+) of point (x, y, z): its index, or -1 outside
__device__ __forceinline__ int64_t nbr(const StencilDesc& A, int64_t p, int x, int y, int z, int q) {
    switch (q) {
        case 1: return x > 0 ? p - 1 : -1;
        case 2: return x < A.nx - 1 ? p + 1 : -1;
        case 3: return y > 0 ? p - A.nx : -1;
        case 4: return y < A.ny - 1 ? p + A.nx : -1;
        case 5: return (A.dim == 3 && z > 0) ? p - (int64_t)A.nx * A.ny : -1;
        default: return (A.dim == 3 && z < A.nz - 1) ? p + (int64_t)A.nx * A.ny : -1;
    }
}

__device__ __forceinline__ int opposite(int q) { return q + ((q & 1) ? 1 : -1); }   // 1<->2, 3<->4, 5<->6

__device__ __forceinline__ void xyz(const StencilDesc& A, int64_t p, int& x, int& y, int& z) {
    const int64_t pl = (int64_t)A.nx * A.ny;
    z = (int)(p / pl);
    const int64_t q = p - (int64_t)z * pl;
    y = (int)(q / A.nx);
    x = (int)(q - (int64_t)y * A.nx);
}

}  // namespace

// The reciprocal pivots: 1 / d~_b at black points, d~_b = a0_b - sum_r A[b, r] A[r, b] / a0_r,
// and 1 / a0_r at red points (the sweeps then multiply instead of divide: an FP64
// division costs many FP64 FMAs on this part)
__global__ void __launch_bounds__(kThreads) rbilu_setup_kernel(StencilDesc A, double* __restrict__ dt) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < A.n; p += stride) {
        int x, y, z;
        xyz(A, p, x, y, z);
        double d = coef(A, 0, p);
        if ((x + y + z) & 1) {
            for (int q = 1; q <= 2 * A.dim; ++q) {
                const int64_t r = nbr(A, p, x, y, z, q);
                if (r >= 0) d -= coef(A, q, p) * coef(A, opposite(q), r) / coef(A, 0, r);
            }
        }
        dt[p] = 1.0 / d;
    }
}

// black points: w_b = (v_b - sum_r A[b, r] v_r / a0_r) / d~_b, with rp = the reciprocal pivots
__global__ void __launch_bounds__(kThreads) rbilu_black_kernel(StencilDesc A, const double* __restrict__ rp,
                                                               const double* __restrict__ v, double* __restrict__ w,
                                                               const SolverState* st, int gate) {
    if (!gate_open(st, gate)) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < A.n; p += stride) {
        int x, y, z;
        xyz(A, p, x, y, z);
        if (!((x + y + z) & 1)) continue;
        double t = __ldg(v + p);
        for (int q = 1; q <= 2 * A.dim; ++q) {
            const int64_t r = nbr(A, p, x, y, z, q);
            if (r >= 0) t = fma(-coef(A, q, p), __ldg(v + r) * __ldg(rp + r), t);
        }
        w[p] = t * __ldg(rp + p);
    }
}

// red points: w_r = (v_r - sum_b A[r, b] w_b) / a0_r (w holds the black results)
__global__ void __launch_bounds__(kThreads) rbilu_red_kernel(StencilDesc A, const double* __restrict__ rp,
                                                             const double* __restrict__ v, double* w,
                                                             const SolverState* st, int gate) {
    if (!gate_open(st, gate)) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < A.n; p += stride) {
        int x, y, z;
        xyz(A, p, x, y, z);
        if ((x + y + z) & 1) continue;
        double t = __ldg(v + p);
        for (int q = 1; q <= 2 * A.dim; ++q) {
            const int64_t b = nbr(A, p, x, y, z, q);
            if (b >= 0) t = fma(-coef(A, q, p), w[b], t);
        }
        w[p] = t * __ldg(rp + p);
    }
}

// dst = *dscale * src (the scaled start vector of a block), gated
__global__ void __launch_bounds__(kThreads) scale_copy_kernel(const double* __restrict__ src, double* __restrict__ dst,
                                                              int64_t n, const double* dscale, const SolverState* st,
                                                              int gate) {
    if (!gate_open(st, gate)) return;
    const double f = *dscale;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) dst[p] = f * src[p];
}

// x += d, gated
__global__ void __launch_bounds__(kThreads) add_kernel(double* __restrict__ x, const double* __restrict__ d, int64_t n,
                                                       const SolverState* st, int gate) {
    if (!gate_open(st, gate)) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) x[p] += d[p];
}

void launch_rbilu_setup(const StencilDesc& A, double* dt, cudaStream_t s) {
    rbilu_setup_kernel<<<grid_for(A.n, 8 * device_sms()), kThreads, 0, s>>>(A, dt);
}

void launch_rbilu_apply(const StencilDesc& A, const double* dt, const double* v, double* w, const SolverState* st,
                        int gate, cudaStream_t s) {
    const int grid = grid_for(A.n, 8 * device_sms());
    rbilu_black_kernel<<<grid, kThreads, 0, s>>>(A, dt, v, w, st, gate);
    rbilu_red_kernel<<<grid, kThreads, 0, s>>>(A, dt, v, w, st, gate);
}

void launch_scale_copy(const double* src, double* dst, int64_t n, const double* dscale, const SolverState* st,
                       int gate, cudaStream_t s) {
    scale_copy_kernel<<<grid_for(n, 8 * device_sms()), kThreads, 0, s>>>(src, dst, n, dscale, st, gate);
}

void launch_add(double* x, const double* d, int64_t n, const SolverState* st, int gate, cudaStream_t s) {
    add_kernel<<<grid_for(n, 8 * device_sms()), kThreads, 0, s>>>(x, d, n, st, gate);
}

}  // namespace sstep
