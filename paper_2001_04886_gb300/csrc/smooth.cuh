// Damped Jacobi smoothing of many systems at once (smooth.cu): one descriptor per system.
#pragma once

#include "common.cuh"

namespace sstep {

struct SmoothSys {
    StencilDesc A;
    const double* f;
    double* x;       // read and overwritten
    double* work;    // scratch of n doubles
};

// `sweeps` sweeps x <- x + omega (f - A x) / a0 for every system; sys: device array of
// nsys (<= 65535) descriptors; nmax: the largest n. Returns -1 on bad arguments.
int launch_jacobi_batched(const SmoothSys* sys, int nsys, int64_t nmax, int sweeps, double omega,
                          cudaStream_t stream);

}  // namespace sstep
