// Kernel declarations and launch-argument structs of the FP64 path.
#pragma once

#include "common.cuh"

namespace sstep {

// What the last CTA of a reduction does with the reduced values.
enum EpiMode : int {
    EPI_NONE = 0,       // write the reduced matrix to `out` only
    EPI_NF,             // ||f||^2 -> st->nf
    EPI_FINAL,          // ||f - A x||^2 -> st->relres (no decisions)
    EPI_RESTART,        // GMRES restart (Alg. 4.2 step 5 / Alg. 2.2 start)
    EPI_GM_T,           // s-step GMRES Scalar2: T_i = W_i^{-1} C_i
    EPI_GM_W,           // s-step GMRES Scalar1: W_k = L^T L, S = W_k^{-1} V_k^T z
    EPI_GM_NU,          // s-step GMRES: nu, columns of G (eq. 4-5), Givens on L G (eq. 9)
    EPI_ST_H,           // GMRES: h_{i,j} (Alg. 2.2 step 1)
    EPI_ST_NORM,        // GMRES: h_{j+1,j} (step 3), Givens (eq. 2)
    EPI_OM_RESTART,     // Orthomin: explicit residual at a (re)start
    EPI_OM_R,           // Orthomin: updated residual after step 4
    EPI_OM_B,           // Orthomin Scalar2: B_j = -W_j^{-1} C_j
    EPI_OM_W            // Orthomin Scalar1: W_{i+1} = L^T L, a = W^{-1} m
};

// Kernels run only while a flag of the solver state is set.
enum Gate : int { GATE_NONE = 0, GATE_ACTIVE = 1, GATE_BUILDING = 2 };

struct Epi {
    int mode = EPI_NONE;
    SolverState* st = nullptr;
    double* out = nullptr;   // EPI_NONE: reduced result (column-major, ld = ldo)
    int ldo = 0;
    int o = 0;               // GMRES: first column of the block / step index j
    int lastblock = 0;       // GMRES: this block or step ends the cycle
    int slot = 0;            // Orthomin: slot of the new direction block
    int nwin = 0;            // Orthomin: blocks in the window
    int win[kMaxCols];       // Orthomin: window slots, oldest first
    int ortho = 0;           // Orthomin: A^T A-orthonormal blocks; the Gram pass has the
                             // A R block last (win[nwin]) and T holds its factor F after B
};

struct Scratch {
    double* partials;        // per-CTA partial results
    unsigned* counter;       // arrival counter (zero between launches); [1]: error flag
    unsigned long long* acc = nullptr;   // exact 128-bit sums of the tensor-core Gram pass
                                         // (kOzAccWords words, zero between launches)
};
constexpr int kOzAccWords = 2 * SSTEP_MAX_COLS * (SSTEP_MAX_S + 1);

__device__ __forceinline__ bool gate_open(const SolverState* st, int gate) {
    if (gate == GATE_NONE) return true;
    if (gate == GATE_ACTIVE) return ((volatile const int*)st)[0] != 0;
    return ((volatile const int*)st)[1] != 0;
}

// ------------------------------------------------------------------ launchers (kernels.cu)
// y = fy * (A v), w = fw * v (if w); fy and fw are multiplied by *dscale when dscale is set.
// y = fy (A v - shift u) with u = v unless given; w = fw v when w is set (shift: the
// Newton basis, 0 otherwise; u: the unpreconditioned power when v = M^-1 u)
// ybnd / wbnd (may be null): atomicMax of the high word of |y_p| / |w_p| over the sweep
// (the column bound of the tensor-core Gram pass; the slots must start at 0).
void launch_stencil(const StencilDesc& A, const double* v, double fy, double* y, double fw, double* w,
                    const double* dscale, const SolverState* st, int gate, cudaStream_t stream, double shift = 0.0,
                    const double* u = nullptr, unsigned* ybnd = nullptr, unsigned* wbnd = nullptr,
                    unsigned* ybnd2 = nullptr, unsigned* wbnd2 = nullptr);

// r = f - A x (x may be null: r = f); out (may be null) receives r; reduces ||r||^2.
void launch_residual(const StencilDesc& A, const double* f, const double* x, double* out, Scratch sc,
                     const Epi& epi, int gate, cudaStream_t stream);

// C = V^T Y (ka x kb), V columns at V + i*ldv (win_s > 0: blocks of win_s columns at
// the panel slots epi.win[]), Y columns at Y + j*ldy.
void launch_gram(int64_t n, const double* V, int64_t ldv, int ka, const double* Y, int64_t ldy, int kb,
                 int win_s, Scratch sc, const Epi& epi, int gate, cudaStream_t stream);

// Yout[:, j] = Yin[:, j] + sgn * V T[:, j] for j >= j0 (columns j < j0 copied as is only
// when Yout != Yin); with gram, reduces Yout^T Yout (kb x kb). ka < 0: ka = st->K and
// T = st->y (the least-squares solution).
// bnd (may be null): bnd[j - j0] receives the column bound (atomicMax of the high word of
// |Yout[:, j]|) of the output columns j0 <= j < bnd_hi.
void launch_update(int64_t n, const double* V, int64_t ldv, int ka, const double* Yin, int64_t ldy,
                   double* Yout, int64_t ldo, int kb, int j0, const double* T, int ldt, double sgn,
                   bool gram, Scratch sc, const Epi& epi, int gate, cudaStream_t stream, unsigned* bnd = nullptr,
                   int bnd_hi = 0);

// ------------------------------------------------------------------ tensor-core Gram pass (ozaki.cu)
// C = V^T Y as launch_gram (contiguous V columns), computed exactly in 61-bit fixed point on
// the tensor cores and rounded once; vmax[ka] / ymax[kb] are the column bounds (largest high
// word of |x| per column, launch_colmax or the producing kernel). Returns false, launching
// nothing, for shapes it does not take (ka > 64, kb > 9, n > 2^27, V or Y not 8-byte
// aligned, no Scratch::acc). A bounded wait that runs out gives NaN entries.
// vw = 1: V holds, in place of each FP64 entry, its biased fixed-point word (the
// fixed_biased value for the column's bound vmax), as kept by an earlier pass. wout: keep
// the words of V's first nw columns there (leading dimension ldw, even; 16-byte aligned),
// for later passes to read with vw = 1.
bool launch_gram_oz(int64_t n, const double* V, int64_t ldv, int ka, const unsigned* vmax, const double* Y,
                    int64_t ldy, int kb, const unsigned* ymax, Scratch sc, const Epi& epi, int gate,
                    cudaStream_t stream, int vw = 0, uint64_t* wout = nullptr, int64_t ldw = 0, int nw = 0);
// Yhat[:, j] = Y[:, j] - V T[:, j], j0 <= j < j0 + kbo, in place, on the tensor cores (exact
// 61-bit fixed-point products, one rounding of V T, then the FP64 difference); vmax: the
// bounds of the ka V columns. bout[j - j0] (and bout2[j - j0] for j - j0 < nb2) receive the
// bounds of the outputs; *bcopy_dst = *bcopy_src (may be null). Returns false, launching
// nothing, for ka > 32 or kbo > 9. A bounded wait that runs out sets st->status to
// SSTEP_ERR_TIMEOUT (ends the solve) and *err (either may be null).
bool launch_update_oz(int64_t n, const double* V, int64_t ldv, int ka, const unsigned* vmax, double* Y, int64_t ldy,
                      int j0, int kbo, const double* T, int ldt, unsigned* bout, unsigned* bout2, int nb2,
                      const unsigned* bcopy_src, unsigned* bcopy_dst, const SolverState* st, int gate,
                      cudaStream_t stream, unsigned* err = nullptr, int vw = 0);   // vw: as launch_gram_oz
// Fused matrix powers of the FP64 s-step block (powers.cu): Y[:, 0] = d u, Y[:, j] = sigma
// (A - theta[j-1] I) Y[:, j-1], j = 1..s, d = *dscale, in one launch whose start-vector
// tiles come in by TMA; the same columns as s separate launch_stencil sweeps, bit for bit.
// b1[j], b2[j] (either may be null): column-bound records of column j. Returns false,
// launching nothing, unless the coefficients are constant, s is 2, 4 or 8, nx is even and
// u is 16-byte aligned (or the driver has no tensor-map encoder). A bounded wait that runs
// out sets st->status to SSTEP_ERR_TIMEOUT and *err.
bool launch_powers_fused(const StencilDesc& A, const double* u, double sigma, const double* dscale, double* Y,
                         int64_t ldy, int s, const double* theta, unsigned* const* b1, unsigned* const* b2,
                         const SolverState* st, int gate, cudaStream_t stream, unsigned* err = nullptr);
// out[c] = column bound of column c (out must be zeroed first)
void launch_colmax(int64_t n, const double* X, int64_t ld, int ncols, unsigned* out, cudaStream_t stream);
int oz_partials_doubles();      // per-CTA partials of the tensor-core Gram pass (none: sums go to Scratch::acc)
int device_sms();               // multiprocessors of the current device
extern long g_oz_spin;          // mbarrier poll limit of the tensor-core Gram pass

// Orthomin: x += P a, r -= AP a (a = st->a), reduces ||r||^2.
void launch_omin_xr(int64_t n, const double* P, const double* AP, int64_t ld, int s, double* x, double* r,
                    Scratch sc, const Epi& epi, int gate, cudaStream_t stream);

// Orthomin: P_new = R + sum_w P_w B_w, AP_new = AR + sum_w AP_w B_w with R = [r, sigma AR_1..];
// reduces W = AP_new^T AP_new and m = AP_new^T r.
void launch_omin_pupdate(int64_t n, const double* r, const double* AR, const double* Ppanel,
                         const double* APpanel, int64_t ld, int s, double sigma, Scratch sc, const Epi& epi,
                         int gate, cudaStream_t stream);

// One CTA: y = R^{-1} g over the first st->K columns (back substitution).
void launch_lsq_solve(SolverState* st, int gate, cudaStream_t stream);

int max_partials_doubles();          // partials of every reduction kernel (workspace size)
int fp64_gram_partials_doubles();    // partials of the FP64 Gram kernel alone

// out = [a0 | am_x | ap_x | am_y | ap_y] (5 arrays of n) for -Lap u + beta (u_x + u_y):
// a0 = 4, am = -1 - beta h/2, ap = -1 + beta h/2
void launch_convdiff_fields(const double* beta, double h, int64_t n, double* out, cudaStream_t stream);
// red-black ILU(0) right preconditioner (precond.cu): setup of the reciprocal pivots
// (1/d~ at black points, 1/a0 at red points), w = M^-1 v (w != v),
// dst = *dscale src, x += d
void launch_rbilu_setup(const StencilDesc& A, double* dt, cudaStream_t s);
void launch_rbilu_apply(const StencilDesc& A, const double* dt, const double* v, double* w, const SolverState* st,
                        int gate, cudaStream_t s);
// ILU(0) in the natural ordering (precond.cu): the factors f = [d | L_x | L_y | L_z] ((dim + 1)
// arrays of n; 2-D: three) by one hyperplane sweep, and w = M^-1 v (w != v) by two
void launch_nilu_setup(const StencilDesc& A, double* f, cudaStream_t s);
void launch_nilu_apply(const StencilDesc& A, const double* f, const double* v, double* w, const SolverState* st,
                       int gate, cudaStream_t s);
void launch_scale_copy(const double* src, double* dst, int64_t n, const double* dscale, const SolverState* st,
                       int gate, cudaStream_t s);
void launch_add(double* x, const double* d, int64_t n, const SolverState* st, int gate, cudaStream_t s);
// damped Jacobi sweep y = x + omega (f - A x) / a0 (smooth.cu)
void launch_jacobi(const StencilDesc& A, const double* f, const double* x, double* y, double omega,
                   cudaStream_t stream);

}  // namespace sstep

namespace sstep {

// ------------------------------------------------------------------ mixed-precision basis (kernels_mp.cu)
// PREC_DF64: basis stored as float pairs (hi, lo) and processed in double-float
// arithmetic on the FP32 pipe. PREC_FP32: basis stored and processed in FP32,
// with every inner product accumulated in double-float. Right-hand side,
// iterate and explicit residuals stay FP64; so does all scalar work.
enum Prec : int { PREC_FP64 = 0, PREC_DF64 = 1, PREC_FP32 = 2 };

inline size_t prec_bytes(int prec) { return prec == PREC_FP32 ? 4 : 8; }

template <int P>
void mp_launch_stencil(const StencilDesc& A, const void* v, double fy, void* y, double fw, void* w,
                       const double* dscale, const SolverState* st, int gate, cudaStream_t stream,
                       double shift = 0.0);
template <int P>
void mp_launch_residual(const StencilDesc& A, const double* f, const double* x, void* out, Scratch sc,
                        const Epi& epi, int gate, cudaStream_t stream);
template <int P>
void mp_launch_gram(int64_t n, const void* V, int64_t ldv, int ka, const void* Y, int64_t ldy, int kb,
                    Scratch sc, const Epi& epi, int gate, cudaStream_t stream);
template <int P>
void mp_launch_update(int64_t n, const void* V, int64_t ldv, int ka, const void* Yin, int64_t ldy, void* Yout,
                      int64_t ldo, int kb, int j0, const double* T, int ldt, double sgn, bool gram, Scratch sc,
                      const Epi& epi, int gate, cudaStream_t stream);
// dst[p] = src[p] split into a float pair (variable coefficients for the mixed-precision kernels)
void launch_split_fields(const double* src, float2* dst, int64_t n, cudaStream_t stream);

// Y[:,0] = (*dscale) u, Y[:,j] = sigma A Y[:,j-1], j = 1..s, in one launch (constant
// coefficients, s in {2, 4, 8}); returns false (nothing launched) otherwise.
template <int P>
bool mp_launch_powers_fused(const StencilDesc& A, const void* u, void* Y, int64_t ldy, int s, double sigma,
                            const double* dscale, const SolverState* st, int gate, cudaStream_t stream);

// x += V y over the current cycle's st->K columns (y = st->y)
template <int P>
void mp_launch_axpy(int64_t n, const void* V, int64_t ldv, double* x, const Epi& epi, int gate,
                    cudaStream_t stream);

}  // namespace sstep

namespace sstep {
// ------------------------------------------------------------------ batched persistent solver (batched.cu)
// one system of a batch: its operator, right-hand side, iterate, basis panel and state
struct BatchSys {
    StencilDesc A;
    const double* f;
    double* x;
    double* U;           // m+2 columns of ld entries (double, or float for the FP32 basis): basis, raw start vector
    SolverState* st;     // state copy 0; copy g (cooperative solves) at st + g * st_stride bytes
    int64_t ld;
    int64_t st_stride;
};
constexpr int kBatchCopies = 8;   // state copies per system: the largest cluster
size_t batched_scratch_bytes(int threads);
// the persistent kernel; cluster = CTAs per cluster (1..8), systems with n >= nbig are
// solved cooperatively by a whole cluster. batched_grid: the grid for about `ctas` CTAs
// with no more clusters than can be resident at once (-1: the configuration cannot run).
// f32: the FP32-basis form (double-float sums, FP64 residual, x and scalar work).
int batched_grid(int s, int threads, int ctas, int cluster, bool f32);
int launch_batched(const BatchSys* sys, const int* order, int nsys, unsigned* queue, int s, int threads, int grid,
                   int cluster, int64_t nbig, bool f32, cudaStream_t stream);
// copies the initial state images src[i * kBatchCopies + g] into every state copy
void launch_batch_init(const SolverState* src, const BatchSys* sys, int nsys, cudaStream_t stream);
}  // namespace sstep
