// Damped Jacobi sweeps on the stencil operator (textbook relaxation, e.g. Saad,
// "Iterative Methods for Sparse Linear Systems", Sec. 4.1): one sweep is
//     y = x + omega (f - A x) / a0,
// with a0 the diagonal (coefficient 0) of the row. The learned initial guess is
// post-smoothed with a few sweeps before the residual test that accepts or rejects
// it: the sweeps damp the rough error components that the h^2-scaled operator
// amplifies most, and leave the smooth part of the prediction in place.
#include "smooth.cuh"

namespace sstep {

__global__ void __launch_bounds__(kThreads) jacobi_kernel(StencilDesc A, const double* __restrict__ f,
                                                          const double* __restrict__ x, double* __restrict__ y,
                                                          double omega) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t pl = (int64_t)A.nx * A.ny;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < A.n; p += stride) {
        const int z = (int)(p / pl);
        const int64_t q = p - (int64_t)z * pl;
        const int yy = (int)(q / A.nx);
        const int xx = (int)(q - (int64_t)yy * A.nx);
        const double r = __ldg(f + p) - stencil_row(A, x, p, xx, yy, z);
        y[p] = fma(omega, r / coef(A, 0, p), __ldg(x + p));
    }
}

void launch_jacobi(const StencilDesc& A, const double* f, const double* x, double* y, double omega,
                   cudaStream_t stream) {
    const int grid = grid_for(A.n, 8 * device_sms());
    jacobi_kernel<<<grid, kThreads, 0, stream>>>(A, f, x, y, omega);
}

// The same sweep for many systems at once: blockIdx.y picks the system, the CTAs along
// x stride over its points. src/dst alternate between x and work per sweep (flip).
__global__ void __launch_bounds__(kThreads) jacobi_batched_kernel(const SmoothSys* __restrict__ sys, double omega,
                                                                  int flip) {
    const SmoothSys& S = sys[blockIdx.y];
    const StencilDesc& A = S.A;
    const double* x = flip ? S.work : S.x;
    double* y = flip ? S.x : S.work;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t pl = (int64_t)A.nx * A.ny;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < A.n; p += stride) {
        const int z = (int)(p / pl);
        const int64_t q = p - (int64_t)z * pl;
        const int yy = (int)(q / A.nx);
        const int xx = (int)(q - (int64_t)yy * A.nx);
        const double r = __ldg(S.f + p) - stencil_row(A, x, p, xx, yy, z);
        y[p] = fma(omega, r / coef(A, 0, p), __ldg(x + p));
    }
}

__global__ void copy_back_kernel(const SmoothSys* __restrict__ sys) {
    const SmoothSys& S = sys[blockIdx.y];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < S.A.n; p += stride) S.x[p] = S.work[p];
}

// sys: device array of nsys descriptors; nmax: the largest n
int launch_jacobi_batched(const SmoothSys* sys, int nsys, int64_t nmax, int sweeps, double omega,
                          cudaStream_t stream) {
    if (nsys < 1 || nsys > 65535) return -1;
    int gx = (int)((nmax + kThreads - 1) / kThreads);
    const int cap = (8 * device_sms() + nsys - 1) / nsys;   // about one wave over all systems
    gx = gx < 1 ? 1 : (gx > cap ? (cap < 1 ? 1 : cap) : gx);
    for (int t = 0; t < sweeps; ++t)
        jacobi_batched_kernel<<<dim3(gx, nsys), kThreads, 0, stream>>>(sys, omega, t & 1);
    if (sweeps & 1) copy_back_kernel<<<dim3(gx, nsys), kThreads, 0, stream>>>(sys);
    return 0;
}

}  // namespace sstep
