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

// ================================================================== ILU(0), natural ordering
// The paper's preconditioner (Sec. 5). With no fill outside A's sparsity, L U = A on it:
// U = diag(d) + A's upper part, L = I + L_k[p] at (p, p - e_k) with L_k[p] = A[p, p - e_k] /
// d[p - e_k], and d[p] = A[p,p] - sum_k A[p, p - e_k] A[p - e_k, p] / d[p - e_k]. Each factor
// entry and each substitution step at p needs only the points p - e_k (forward) or p + e_k
// (backward), which lie on the neighbouring hyperplane x + y + z = c -/+ 1, so every sweep is
// a chain of 2N - 1 (2-D) or 3N - 2 (3-D) hyperplanes of independent points: the
// vectorisable form the paper cites. One CTA walks the chain with a barrier between
// hyperplanes (its own global writes are visible to all its threads after the barrier).
// The arithmetic is the oracle's, term by term in its order (x, y, z), with every product,
// quotient and difference rounded on its own (no contraction), so the factors and M^-1 v
// are the oracle's bit for bit.
namespace {

constexpr int kNiluThreads = 1024;

// f(p, x, y, z) for every grid point with x + y + z = c, spread over the CTA's threads
template <int DIM, typename F>
__device__ __forceinline__ void for_plane(const StencilDesc& A, int c, F&& f) {
    if (DIM == 2) {
        const int lo = max(0, c - (A.ny - 1)), hi = min(c, A.nx - 1);
        for (int x = lo + (int)threadIdx.x; x <= hi; x += (int)blockDim.x) {
            const int y = c - x;
            f((int64_t)y * A.nx + x, x, y, 0);
        }
    } else {
        const int klo = max(0, c - (A.nx - 1) - (A.ny - 1)), khi = min(c, A.nz - 1);
        const int64_t cnt = khi >= klo ? (int64_t)(khi - klo + 1) * A.ny : 0;
        for (int64_t t = threadIdx.x; t < cnt; t += blockDim.x) {
            const int z = klo + (int)(t / A.ny), y = (int)(t % A.ny), x = c - y - z;
            if (x >= 0 && x < A.nx) f(((int64_t)z * A.ny + y) * A.nx + x, x, y, z);
        }
    }
}

template <int DIM>
__device__ __forceinline__ int last_plane(const StencilDesc& A) {
    return (A.nx - 1) + (A.ny - 1) + (DIM == 3 ? A.nz - 1 : 0);
}

// the factors: f[0] = d (pivots), f[1 + k] = L_k (zero where p - e_k is outside the grid)
template <int DIM>
__global__ void __launch_bounds__(kNiluThreads) nilu_setup_kernel(StencilDesc A, double* f) {
    double* d = f;
    double* Lx = f + A.n;
    double* Ly = f + 2 * A.n;
    double* Lz = f + 3 * A.n;
    const int64_t sy = A.nx, sz = (int64_t)A.nx * A.ny;
    const int cmax = last_plane<DIM>(A);
    for (int c = 0; c <= cmax; ++c) {
        for_plane<DIM>(A, c, [&](int64_t p, int x, int y, int z) {
            double dp = coef(A, 0, p);
            if (x > 0) dp = __dsub_rn(dp, __ddiv_rn(__dmul_rn(coef(A, 1, p), coef(A, 2, p - 1)), d[p - 1]));
            if (y > 0) dp = __dsub_rn(dp, __ddiv_rn(__dmul_rn(coef(A, 3, p), coef(A, 4, p - sy)), d[p - sy]));
            if (DIM == 3 && z > 0)
                dp = __dsub_rn(dp, __ddiv_rn(__dmul_rn(coef(A, 5, p), coef(A, 6, p - sz)), d[p - sz]));
            d[p] = dp;
            Lx[p] = x > 0 ? __ddiv_rn(coef(A, 1, p), d[p - 1]) : 0.0;
            Ly[p] = y > 0 ? __ddiv_rn(coef(A, 3, p), d[p - sy]) : 0.0;
            if (DIM == 3) Lz[p] = z > 0 ? __ddiv_rn(coef(A, 5, p), d[p - sz]) : 0.0;
        });
        __syncthreads();
    }
}

// w = M^-1 v: forward y = L^-1 v into w hyperplane by hyperplane, then backward
// z = U^-1 y in place (z at p overwrites y at p; the backward step at p reads y[p] and
// the z of hyperplane c + 1)
template <int DIM>
__global__ void __launch_bounds__(kNiluThreads) nilu_apply_kernel(StencilDesc A, const double* f, const double* v,
                                                                  double* w, const SolverState* st, int gate) {
    if (!gate_open(st, gate)) return;
    const double* d = f;
    const double* Lx = f + A.n;
    const double* Ly = f + 2 * A.n;
    const double* Lz = f + 3 * A.n;
    const int64_t sy = A.nx, sz = (int64_t)A.nx * A.ny;
    const int cmax = last_plane<DIM>(A);
    for (int c = 0; c <= cmax; ++c) {
        for_plane<DIM>(A, c, [&](int64_t p, int x, int y, int z) {
            double t = v[p];
            if (x > 0) t = __dsub_rn(t, __dmul_rn(__ldg(Lx + p), w[p - 1]));
            if (y > 0) t = __dsub_rn(t, __dmul_rn(__ldg(Ly + p), w[p - sy]));
            if (DIM == 3 && z > 0) t = __dsub_rn(t, __dmul_rn(__ldg(Lz + p), w[p - sz]));
            w[p] = t;
        });
        __syncthreads();
    }
    for (int c = cmax; c >= 0; --c) {
        for_plane<DIM>(A, c, [&](int64_t p, int x, int y, int z) {
            double t = w[p];
            if (x < A.nx - 1) t = __dsub_rn(t, __dmul_rn(coef(A, 2, p), w[p + 1]));
            if (y < A.ny - 1) t = __dsub_rn(t, __dmul_rn(coef(A, 4, p), w[p + sy]));
            if (DIM == 3 && z < A.nz - 1) t = __dsub_rn(t, __dmul_rn(coef(A, 6, p), w[p + sz]));
            w[p] = __ddiv_rn(t, __ldg(d + p));
        });
        __syncthreads();
    }
}

// 2-D, nx <= kNiluThreads: thread x owns grid column x and meets its points in order of
// y on the successive hyperplanes (forward: y = c - x rising; backward: falling). The
// neighbour along y is its own previous result (a register); the neighbour along x is
// the previous hyperplane's result of thread x -/+ 1, passed through a double-buffered
// shared row. The operands that do not depend on the recurrence (v, L, the upper
// coefficients, the pivots, y for the backward sweep) are fetched one hyperplane ahead
// and prefetched into L1 eight ahead. Same operations, same order as nilu_apply_kernel.
__global__ void __launch_bounds__(kNiluThreads) nilu_apply2d_kernel(StencilDesc A, const double* f, const double* v,
                                                                    double* w, const SolverState* st, int gate) {
    if (!gate_open(st, gate)) return;
    __shared__ double row[2][kNiluThreads];
    const double* d = f;
    const double* Lx = f + A.n;
    const double* Ly = f + 2 * A.n;
    const int x = (int)threadIdx.x, nx = A.nx, ny = A.ny;
    const bool on = x < nx;
    const int cmax = nx - 1 + ny - 1;
    constexpr int kAhead = 8;
    // forward: y = L^-1 v
    double prev = 0.0, nv = 0.0, nlx = 0.0, nly = 0.0;
    auto fetch_f = [&](int c) {
        const int yy = c - x;
        if (on && yy >= 0 && yy < ny) {
            const int64_t p = (int64_t)yy * nx + x;
            nv = v[p];
            nlx = __ldg(Lx + p);
            nly = __ldg(Ly + p);
        }
        const int ya = yy + kAhead;
        if (on && ya >= 0 && ya < ny) {
            const int64_t pa = (int64_t)ya * nx + x;
            asm volatile("prefetch.global.L1 [%0];" ::"l"(v + pa));
            asm volatile("prefetch.global.L1 [%0];" ::"l"(Lx + pa));
            asm volatile("prefetch.global.L1 [%0];" ::"l"(Ly + pa));
        }
    };
    fetch_f(0);
    for (int c = 0; c <= cmax; ++c) {
        const double cv = nv, clx = nlx, cly = nly;
        const int yy = c - x;
        const bool act = on && yy >= 0 && yy < ny;
        fetch_f(c + 1);
        if (act) {
            double t = cv;
            if (x > 0) t = __dsub_rn(t, __dmul_rn(clx, row[(c - 1) & 1][x - 1]));
            if (yy > 0) t = __dsub_rn(t, __dmul_rn(cly, prev));
            w[(int64_t)yy * nx + x] = t;
            row[c & 1][x] = t;
            prev = t;
        }
        __syncthreads();
    }
    // backward: z = U^-1 y in place
    double ny_ = 0.0, nux = 0.0, nuy = 0.0, nd = 0.0;
    auto fetch_b = [&](int c) {
        const int yy = c - x;
        if (on && yy >= 0 && yy < ny) {
            const int64_t p = (int64_t)yy * nx + x;
            ny_ = w[p];
            nux = coef(A, 2, p);
            nuy = coef(A, 4, p);
            nd = __ldg(d + p);
        }
    };
    fetch_b(cmax);
    prev = 0.0;
    for (int c = cmax; c >= 0; --c) {
        const double cy = ny_, cux = nux, cuy = nuy, cd = nd;
        const int yy = c - x;
        const bool act = on && yy >= 0 && yy < ny;
        fetch_b(c - 1);
        if (act) {
            double t = cy;
            if (x < nx - 1) t = __dsub_rn(t, __dmul_rn(cux, row[(c + 1) & 1][x + 1]));
            if (yy < ny - 1) t = __dsub_rn(t, __dmul_rn(cuy, prev));
            t = __ddiv_rn(t, cd);
            w[(int64_t)yy * nx + x] = t;
            row[c & 1][x] = t;
            prev = t;
        }
        __syncthreads();
    }
}

}  // namespace

void launch_nilu_setup(const StencilDesc& A, double* f, cudaStream_t s) {
    if (A.dim == 3) nilu_setup_kernel<3><<<1, kNiluThreads, 0, s>>>(A, f);
    else nilu_setup_kernel<2><<<1, kNiluThreads, 0, s>>>(A, f);
}

void launch_nilu_apply(const StencilDesc& A, const double* f, const double* v, double* w, const SolverState* st,
                       int gate, cudaStream_t s) {
    if (A.dim == 3) nilu_apply_kernel<3><<<1, kNiluThreads, 0, s>>>(A, f, v, w, st, gate);
    else if (A.nx <= kNiluThreads) nilu_apply2d_kernel<<<1, kNiluThreads, 0, s>>>(A, f, v, w, st, gate);
    else nilu_apply_kernel<2><<<1, kNiluThreads, 0, s>>>(A, f, v, w, st, gate);
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
