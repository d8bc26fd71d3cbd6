// Damped Jacobi sweeps on the stencil operator (textbook relaxation, e.g. Saad,
// "Iterative Methods for Sparse Linear Systems", Sec. 4.1): one sweep is
//     y = x + omega (f - A x) / a0,
// with a0 the diagonal (coefficient 0) of the row. The learned initial guess is
// post-smoothed with a few sweeps before the residual test that accepts or rejects
// it: the sweeps damp the rough error components that the h^2-scaled operator
// amplifies most, and leave the smooth part of the prediction in place.
#include "common.cuh"

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
    const int grid = grid_for(A.n, 152 * 8);
    jacobi_kernel<<<grid, kThreads, 0, stream>>>(A, f, x, y, omega);
}

}  // namespace sstep
