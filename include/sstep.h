/*
 * sstep.h - C ABI of the GB300 s-step Orthomin / s-step GMRES library.
 *
 * Method: A. T. Chronopoulos and S. K. Kim, "s-Step Orthomin and GMRES
 * implemented on parallel computers" (1990). Section numbers, algorithms and
 * equations below refer to that paper.
 *
 * Conventions for every entry point:
 *   - All vector pointers are DEVICE pointers on the current CUDA device unless
 *     a comment says "host". Vectors are contiguous float64 arrays of n values
 *     in grid order (x fastest, then y, then z).
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *     stream. Work is stream-ordered. Kernel-level entry points return after
 *     enqueueing; solvers synchronise `stream` (see each solver).
 *   - The caller owns every pointer it passes. Matrix handles own their
 *     coefficient copies and their solver workspace.
 *   - Every call returns an sstep_status (0 = success). Nothing aborts and no
 *     C++ exception crosses the ABI. Argument errors return SSTEP_ERR_ARG before
 *     any work is enqueued.
 *   - A handle may run one solve at a time (its workspace is reused).
 *
 * Environment switches (read once per process, at the first solve; all default to the
 * fastest measured path):
 *   SSTEP_TC_GRAM=0       FP64 s-step GMRES forms its inner products and block updates
 *                         on the FP64 CUDA cores instead of the tensor cores (exact fixed
 *                         point); for comparisons.
 *   SSTEP_TC_WORDS=0      the tensor-core passes convert every basis column again instead
 *                         of reading the fixed-point words the block's Gram pass kept.
 *   SSTEP_FUSED_POWERS=1  the s powers of a block in one fused launch with s-deep halos
 *                         (FP64: start-vector tiles staged by TMA; the same columns bit for
 *                         bit); measured slower than the separate sweeps on GB300.
 */
#ifndef SSTEP_H
#define SSTEP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SSTEP_OK = 0,
    SSTEP_NOT_CONVERGED = 1,   /* max cycles / iterations reached; x holds the last iterate */
    SSTEP_ERR_ARG = -1,        /* invalid argument (null pointer, size, s, m, k out of range) */
    SSTEP_ERR_CUDA = -2,       /* a CUDA runtime call failed */
    SSTEP_ERR_OOM = -3,        /* device allocation failed */
    SSTEP_ERR_BREAKDOWN = -4,  /* non-positive Cholesky pivot in a Gram block W (Scalar1/Scalar2) */
    SSTEP_ERR_NAN = -5,        /* a residual norm became NaN or Inf */
    SSTEP_ERR_TIMEOUT = -6     /* a bounded device-side wait (tensor-core pipeline) ran out */
} sstep_status;

typedef struct sstep_matrix_s* sstep_matrix;

/* ------------------------------------------------------------------ operator
 * The operator of Sec. 1 / Sec. 5: a (2*dim+1)-point stencil on an
 * nx x ny [x nz] grid of interior unknowns with homogeneous Dirichlet
 * boundaries (neighbours outside the grid are zero). Row p is
 *   (A u)_p = a0 u_p + sum_d ( am_d u_{p-e_d} + ap_d u_{p+e_d} ),
 * summed in the order centre, x-, x+, y-, y+, z-, z+.
 */

/* Constant coefficients. shape = {nx, ny, nz} (nz ignored when dim == 2).
 * coef (host) = {a0, am_x, ap_x, am_y, ap_y[, am_z, ap_z]}. */
int stencil_matrix_create(sstep_matrix* out, int dim, const int64_t shape[3], const double* coef);

/* Variable coefficients: fields (host array of 2*dim+1 DEVICE pointers, each n
 * values, same order as coef). The library copies the fields. */
int stencil_matrix_create_fields(sstep_matrix* out, int dim, const int64_t shape[3],
                                 const double* const* fields, void* stream);

/* The h^2-scaled centred convection-diffusion operator of -Lap u + beta . grad u
 * on the unit square/cube (Sec. 5, eq. 10 with constant coefficients): all sides
 * equal N, h = 1/(N+1), c_d = beta_d h / 2, a0 = 2 dim, am_d = -1 - c_d,
 * ap_d = -1 + c_d. beta (host) holds dim values. */
int stencil_matrix_create_convdiff(sstep_matrix* out, int dim, const int64_t shape[3], const double* beta);

/* The 2-D operator of -Lap u + beta(x, y) (u_x + u_y) on an N x N interior grid
 * (non-conservative form): row p has a0 = 4 and am_d = -1 - c_p, ap_d = -1 + c_p with
 * c_p = beta_p h / 2, h = 1/(N+1). beta_field: DEVICE array of N*N values (copied;
 * the coefficient fields are computed on the device). */
int stencil_matrix_create_convdiff_variable(sstep_matrix* out, int64_t N, const double* beta_field, void* stream);

int stencil_matrix_destroy(sstep_matrix A);

/* n (number of unknowns) and ||A||_inf (max absolute row sum). Host outputs. */
int stencil_matrix_info(sstep_matrix A, int64_t* n, double* norm_inf);

/* w = M^-1 v for the red-black ILU(0) of A (the preconditioner of SSTEP_PRECOND_RBILU0;
 * its factor diagonal is built on first use and kept with A). v, w: DEVICE arrays of n,
 * distinct. Stream-ordered. */
int stencil_matrix_rbilu0_apply(sstep_matrix A, const double* v, double* w, void* stream);

/* w = M^-1 v for ILU(0) of A in the natural ordering (Sec. 5: the paper's right
 * preconditioner; the preconditioner of SSTEP_PRECOND_ILU0). With no fill outside A's
 * sparsity, L U = A there: U = diag(d) + the upper part of A, L = I + A[p, p - e_k] / d[p - e_k]
 * below it, d[p] = A[p,p] - sum_k A[p, p - e_k] A[p - e_k, p] / d[p - e_k]. The factors
 * ((dim + 1) n doubles) are built on first use and kept with A. Both substitutions run as
 * sweeps over the hyperplanes x + y (+ z) = c, one CTA with a barrier between hyperplanes
 * (2N - 1 of them in 2-D, 3N - 2 in 3-D), every operation rounded as written, so the
 * result is that of the plain point-by-point substitutions in the natural order. v, w:
 * DEVICE arrays of n, distinct. Stream-ordered. */
int stencil_matrix_ilu0_apply(sstep_matrix A, const double* v, double* w, void* stream);

/* The Newton-basis shifts theta_1..theta_s of the last s-step GMRES solve on A with
 * basis = SSTEP_BASIS_NEWTON (HOST output, up to cap values). Returns their number (0
 * when the last solve kept the monomial powers), or SSTEP_ERR_ARG. */
int sstep_last_shifts(sstep_matrix A, double* theta, int cap);

/* Caps the device workspace a solve may allocate (bytes; 0: no cap). A solve that needs
 * more returns SSTEP_ERR_OOM before touching the device: the allocation-failure path,
 * testable without a GPU. Process-global. */
int sstep_set_workspace_limit(int64_t bytes);

/* The shift computation on its own (host only, no GPU): theta[0..s) = the Leja-ordered
 * real parts of the eigenvalues of the K x K upper Hessenberg matrix G (HOST,
 * column-major, leading dimension ldg >= K), as the Newton basis uses them. Returns
 * SSTEP_ERR_BREAKDOWN if the QR iteration does not settle. */
int sstep_newton_shifts(const double* G, int ldg, int K, int s, double* theta);

/* y = A x (Sec. 1: one sweep over the grid). x and y must not overlap. */
int stencil_matrix_apply(sstep_matrix A, const double* x, double* y, void* stream);

/* Damped Jacobi smoothing (textbook relaxation, e.g. Saad, Iterative Methods for
 * Sparse Linear Systems, Sec. 4.1; not part of the s-step method): `sweeps` times
 * x <- x + omega (f - A x) / a0, a0 the diagonal of the row. Used to post-smooth a
 * learned initial guess. f, x, work: DEVICE arrays of n doubles, caller-owned; work is
 * scratch and must not alias x or f; x is read and overwritten. sweeps >= 0 (0: no-op),
 * 0 < omega < 2, else SSTEP_ERR_ARG. Stream-ordered, no synchronisation. */
int stencil_matrix_smooth(sstep_matrix A, const double* f, double* x, double* work, int sweeps, double omega,
                          void* stream);
/* The same for nsys (1..65535) systems in one launch per sweep: A, f, x, work are HOST
 * arrays of nsys handles / DEVICE pointers with the per-system conventions above.
 * Synchronises `stream` once (the descriptors are copied from the host). */
int stencil_matrix_smooth_batched(int nsys, const sstep_matrix* A, const double* const* f, double* const* x,
                                  double* const* work, int sweeps, double omega, void* stream);

/* ------------------------------------------------------------------ s-step block primitives
 * The three data-parallel steps of one s-step (Sec. 1, Alg. 3.1, Alg. 4.1),
 * exposed one by one. Column-major panels: column j of a panel P with leading
 * dimension ld starts at P + j*ld; ld >= n.
 */

/* Matrix powers (Alg. 3.1 R_i, Alg. 4.1 step 3):
 *   Y[:,0] = scale * v,  Y[:,j] = sigma * A Y[:,j-1]  for j = 1..s.
 * v must not overlap Y. 1 <= s <= SSTEP_MAX_S. */
int sstep_matrix_powers(sstep_matrix A, const double* v, double scale, double sigma, int s,
                        double* Y, int64_t ldy, void* stream);

/* Bytes of device workspace the Gram pass (sstep_gram or sstep_gram_tc) needs for ka x kb
 * outputs over n rows. */
int sstep_gram_workspace_size(int64_t n, int ka, int kb, size_t* bytes);

/* The simultaneous inner products of one s-step (Sec. 1; Alg. 4.1 steps 4-5;
 * Alg. 3.1 steps 1 and 6) as one tall-skinny Gram pass:
 *   C = V^T Y,  V: n x ka (ldv), Y: n x kb (ldy), C: ka x kb column-major (ldc >= ka), device.
 * work: device buffer of at least sstep_gram_workspace_size bytes, 256-byte aligned.
 * The reduction order is fixed, so results are bitwise reproducible.
 * 1 <= ka <= SSTEP_MAX_COLS, 1 <= kb <= SSTEP_MAX_S + 1. */
int sstep_gram(int64_t n, const double* V, int64_t ldv, int ka, const double* Y, int64_t ldy, int kb,
               double* C, int ldc, void* work, size_t work_bytes, void* stream);

/* The same inner products (Sec. 1; Alg. 4.1 steps 4-5) on the tensor cores, the Gram pass
 * the FP64 s-step GMRES uses. Every column is scaled by a power of two from its largest
 * entry and written as a 61-bit fixed-point integer of eight balanced 8-bit digits (an
 * Ozaki-Ogita-Oishi-Rump error-free splitting); the digit products run as FP16 MMAs whose
 * FP32 sums stay exact integers, the sums over rows are exact 128-bit integers, and each
 * entry of C is rounded to FP64 once. Error per entry before that rounding: at most
 * 2^-65 sum_rows(Bv By) + 2^-60 sum_rows(Bv |y| + |v| By), where Bv, By are the two
 * columns' power-of-two bounds (below 2 max|entry|) -- the digit pairs left out and the
 * truncation to 61 bits; subnormal entries count as zero. The result is independent of the
 * grid and of the order of the rows. A column holding Inf or NaN gives NaN in its row or
 * column of C.
 * Arguments, work and ranges as for sstep_gram; in addition n <= 2^27, else SSTEP_ERR_ARG. */
int sstep_gram_tc(int64_t n, const double* V, int64_t ldv, int ka, const double* Y, int64_t ldy, int kb,
                  double* C, int ldc, void* work, size_t work_bytes, void* stream);

/* Test hook: the number of polls of each bounded mbarrier wait in the tensor-core Gram
 * pass (process-global; 0: every wait runs out at once; < 0 restores the default 2^24).
 * A wait that runs out makes the results of that call NaN; the kernel still waits for
 * its tensor-core work in flight, frees its tensor memory and ends normally. */
int sstep_set_tc_wait_limit(long limit);

/* The same Gram pass as sstep_gram, for callers that cannot allocate device
 * memory when they call it: applications that fix their device-memory budget at
 * start-up and forbid later allocations, and plug-in hosts whose own allocator owns
 * all device memory, so that a library allocating behind their back would break
 * their accounting or fail. The paper has no counterpart; this is a property of the
 * library's interface, not of the method.
 *   - Allocates nothing: the scratch is a fixed 884,992-byte array in the library's
 *     device image (sized for devices of up to 192 multiprocessors), present on every
 *     GPU that loads the library until the process exits. ka <= SSTEP_MAX_COLS,
 *     kb <= SSTEP_MAX_S + 1 and at most 192 multiprocessors, else SSTEP_ERR_ARG.
 *   - The first call on each device looks up the array's device address (with that
 *     device current); make that first call before any stream capture begins. Later
 *     calls on a stream that is not being captured look the address up again, so a
 *     cudaDeviceReset in between is harmless.
 *   - Every call shares the one array per device, and its contents persist between
 *     calls: calls whose executions overlap on the GPU (other streams, other host
 *     threads) race and give wrong results. Serialise them on one stream.
 * Arguments and results as for sstep_gram. */
int sstep_gram_noalloc(int64_t n, const double* V, int64_t ldv, int ka, const double* Y, int64_t ldy, int kb,
                       double* C, int ldc, void* stream);

/* Block update (Alg. 4.1 step 7 with Scalar1's Gram; Alg. 3.1 steps 8-9 shape):
 *   Y <- Y - V T  (in place; V: n x ka, T: ka x kb column-major device, ldt >= ka),
 *   then Gout = Y^T Y (kb x kb, column-major, device) over the updated Y.
 * ka may be 0 (Gram only). V must not overlap Y. work as for sstep_gram(n, kb, kb). */
int sstep_block_update(int64_t n, const double* V, int64_t ldv, int ka, double* Y, int64_t ldy, int kb,
                       const double* T, int ldt, double* Gout, void* work, size_t work_bytes, void* stream);

/* The same block update on the tensor cores, as the FP64 s-step GMRES runs it: every V
 * column in 61-bit fixed point relative to its power-of-two bound, T folded with those
 * bounds and split the same way per column, the digit products summed exactly per digit
 * diagonal on the tensor cores, V T rounded to FP64 once per entry and subtracted from Y
 * in FP64; then Gout = Y^T Y by sstep_gram_tc. Error of V T per entry before its rounding:
 * at most 2^-65 sum_a(Bv_a Bt_j) + 2^-60 sum_a(Bv_a |t_aj| + |v_a| Bt_j) in the scaled
 * quantities (the bounds of sstep_gram_tc, for the products v_a t_aj). 0 <= ka <= 32,
 * 1 <= kb <= SSTEP_MAX_S + 1, n <= 2^27; work as for sstep_gram(n, 1, kb). A bounded
 * device wait that runs out leaves Y partly updated and Gout NaN. */
int sstep_block_update_tc(int64_t n, const double* V, int64_t ldv, int ka, double* Y, int64_t ldy, int kb,
                          const double* T, int ldt, double* Gout, void* work, size_t work_bytes, void* stream);

/* ------------------------------------------------------------------ solvers */
#define SSTEP_MAX_S 8        /* largest block size s on the GPU path */
#define SSTEP_MAX_M 64       /* largest Krylov dimension per cycle */
#define SSTEP_MAX_COLS 64    /* largest ka of the Gram pass */

typedef struct {
    int s;              /* block size (>= 1, <= SSTEP_MAX_S) */
    int m;              /* GMRES: Krylov dimension per cycle, a multiple of s (<= SSTEP_MAX_M) */
    int k;              /* Orthomin: number of previous direction blocks kept (>= 0) */
    double tol;         /* stop when ||f - A x|| / ||f|| <= tol (||f|| read as 1 when f = 0:
                           x = 0 solves, and from x0 = 0 the solve ends at its first residual) */
    int max_cycles;     /* GMRES: maximum restart cycles */
    int max_iters;      /* Orthomin: maximum (s-)steps */
    double sigma;       /* basis scale of the monomial powers; 0 => 1 / ||A||_inf */
    double* history;    /* HOST array receiving the residual history, or NULL */
    int history_cap;    /* capacity of history */
    int precision;      /* storage/arithmetic of the Krylov basis (GMRES solvers; Orthomin: FP64 only):
                           SSTEP_PREC_FP64: FP64;
                           SSTEP_PREC_DF64: double-float pairs (48-bit significand) on the FP32 pipe;
                           SSTEP_PREC_FP32: FP32 basis and powers, inner products accumulated in
                           double-float; with the FP64 restart residual this is FP32 iterative
                           refinement. f, x, residuals and all scalar work are FP64 in every mode. */
    int x0_guard;       /* 1: if ||f - A x0|| > ||f|| on entry, start from x0 = 0 instead (for
                           predicted initial guesses); 0: use x0 as given */
    int basis;          /* s-step GMRES (multi-kernel solver, every precision):
                           SSTEP_BASIS_MONOMIAL: y^{j+1} = sigma A y^j (Alg. 4.1 as printed);
                           SSTEP_BASIS_NEWTON: the first cycle is monomial; every later cycle uses
                           y^{j+1} = sigma (A - theta_j I) y^j with theta_1..theta_s the real parts
                           of the first cycle's Ritz values (eigenvalues of its Hessenberg G) in
                           Leja order. Same Krylov spaces, better-conditioned Gram blocks (Sec. 3
                           names such bases for large s). The batched solver is monomial only.
                           s-step Orthomin: SSTEP_BASIS_MONOMIAL (Alg. 3.1 as printed) or
                           SSTEP_BASIS_ORTHO: every direction block P_i (P_0 = R_0 and each
                           projected P_{i+1}) is made A^T A-orthonormal, the remedy Sec. 3 gives
                           for large s, so that W_i is the identity up to rounding; then
                           (k + 1) s <= SSTEP_MAX_COLS. Other values: SSTEP_ERR_ARG. */
    int precond;        /* s-step GMRES and s-step Orthomin, FP64 only (others: SSTEP_ERR_ARG):
                           SSTEP_PRECOND_NONE;
                           SSTEP_PRECOND_RBILU0: right preconditioning with ILU(0) in red-black
                           ordering (the sparsity pattern of A, d~_b = a0_b - sum_r A[b,r] A[r,b] /
                           a0_r); powers of A M^-1, x = x0 + M^-1 V y (Orthomin: the steps P a
                           accumulate and x += M^-1 of them before every explicit residual), true
                           restart residual; sigma defaults to 1.
                           SSTEP_PRECOND_ILU0: the same right preconditioning with ILU(0) in the
                           natural ordering (the paper's, Sec. 5; see stencil_matrix_ilu0_apply). */
} sstep_params;

#define SSTEP_BASIS_MONOMIAL 0
#define SSTEP_BASIS_NEWTON 1
#define SSTEP_BASIS_ORTHO 2

#define SSTEP_PRECOND_NONE 0
#define SSTEP_PRECOND_RBILU0 1
#define SSTEP_PRECOND_ILU0 2

#define SSTEP_PREC_FP64 0
#define SSTEP_PREC_DF64 1
#define SSTEP_PREC_FP32 2

typedef struct {
    int status;         /* sstep_status of the solve */
    int cycles;         /* GMRES restart cycles run (Orthomin: restarts from an explicit residual) */
    int iters;          /* Krylov steps (GMRES) or s-steps (Orthomin) */
    int matvecs;        /* products with A, including explicit residuals */
    int history_len;    /* entries written to params.history (<= history_cap) */
    double relres;      /* final explicit ||f - A x|| / ||f|| */
} sstep_result;

/* s-step GMRES (Alg. 4.2 over the s-step Arnoldi of Alg. 4.1, least squares of
 * eq. 6-9). Restart r = f - A x is explicit; per cycle m/s blocks of s products.
 * History: the explicit relres at every restart, then the least-squares estimate
 * after each step of every block; a cycle ends early once the estimate is <= tol.
 * x (device) is the initial guess on entry and the result on exit. Synchronises
 * `stream` once per cycle. */
int sstep_gmres_solve(sstep_matrix A, const double* f, double* x, const sstep_params* p,
                      sstep_result* res, void* stream);

/* Standard restarted GMRES(m) with classical Gram-Schmidt (Alg. 2.2, eq. 2-3):
 * the plain baseline of the same kernels' quality. p->s is ignored. */
int gmres_solve(sstep_matrix A, const double* f, double* x, const sstep_params* p,
                sstep_result* res, void* stream);

/* s-step Orthomin(k) (Alg. 3.1); s = 1 is Orthomin(k) (Alg. 2.1). The updated
 * residual is tested after each s-step; at tol it is recomputed explicitly and
 * the method restarts if the explicit residual is still above tol. History: the
 * explicit relres at (re)starts and the updated relres after each s-step.
 * With p->basis = SSTEP_BASIS_ORTHO the new block is orthonormalised in the A^T A
 * inner product by the triangular factor of its Gram matrix, predicted in the pass
 * that forms the window's inner products (W_new = A R^T A R - sum_j C_j^T W_j^-1 C_j)
 * and folded into the block update (no extra pass over the vectors); Scalar1/Scalar2
 * then solve with Gram blocks equal to the identity up to rounding. Where the
 * predicted Gram is not positive definite the block is left as formed. */
int sstep_omin_solve(sstep_matrix A, const double* f, double* x, const sstep_params* p,
                     sstep_result* res, void* stream);

/* ------------------------------------------------------------------ batched solves
 * Many independent systems solved by s-step GMRES (Alg. 4.1/4.2) together. A batch
 * handle plans the work once (workspace for every system, launch configuration)
 * and then solves any number of right-hand sides. Mode SSTEP_BATCH_PERSISTENT runs
 * the whole batch as one persistent kernel, replayed from a captured CUDA graph:
 * each CTA takes the next system from a work queue (largest first unless tuned
 * otherwise) and runs its entire solve with CTA-wide reductions. Mode
 * SSTEP_BATCH_PER_SYSTEM calls sstep_gmres_solve once per system (the comparison).
 * The handle keeps references to the matrices, which must outlive it.
 * p: s in {1, 2, 4, 8}, m <= 40 and a multiple of s; p->precision SSTEP_PREC_FP64 or
 * SSTEP_PREC_FP32 (the persistent kernel then keeps the basis in FP32, adds exact FP32
 * products in double-float and keeps the restart residual, x and the scalar work in
 * FP64: FP32 iterative refinement per system, as sstep_gmres_solve's FP32 mode, with
 * the same FP64 stopping test); monomial basis, no preconditioner; p->history is
 * ignored. */
#define SSTEP_BATCH_PERSISTENT 0
#define SSTEP_BATCH_PER_SYSTEM 1
typedef struct sstep_batch_s* sstep_batch;
int sstep_batch_create(sstep_batch* out, int nsys, const sstep_matrix* A, const sstep_params* p);
/* f, x: HOST arrays of nsys DEVICE pointers (x: initial guesses in, solutions out);
 * res: HOST array of nsys results. Synchronises `stream`. */
int sstep_batch_solve(sstep_batch B, const double* const* f, double* const* x, sstep_result* res, int mode,
                      void* stream);
/* Autotuner: times the persistent solve of the given batch under each candidate
 * launch configuration, keeps the fastest in the handle and reports it (host
 * outputs, may be NULL): threads per CTA, CTAs per SM, queue order (largest system
 * first or not), and the size classes: systems with n >= *coop_min_n are solved by
 * a thread-block cluster of *cluster CTAs together (cluster 1: every system by one
 * CTA), the rest by one CTA each. x is restored to its initial content after every
 * trial. */
int sstep_batch_tune(sstep_batch B, const double* const* f, double* const* x, int* threads, int* ctas_per_sm,
                     int* largest_first, int* cluster, int64_t* coop_min_n, void* stream);
/* Sets the launch configuration by hand (the values sstep_batch_tune chooses among):
 * threads in {32, 64, ..., 256}, ctas_per_sm >= 1, cluster in 1..8, coop_min_n >= 0
 * (systems with n >= coop_min_n are solved by a whole cluster when cluster > 1).
 * Configurations the device cannot run make sstep_batch_solve return SSTEP_ERR_ARG. */
int sstep_batch_configure(sstep_batch B, int threads, int ctas_per_sm, int largest_first, int cluster,
                          int64_t coop_min_n);
int sstep_batch_destroy(sstep_batch B);

const char* sstep_status_string(int status);

/* ------------------------------------------------------------------ learned initial guess
 * A 4-level convolutional U-Net mapping the channels (f, beta) of an H x W grid
 * (H, W multiples of 8) to an initial guess x0 for the solvers above. The paper has
 * no such component: it is a predictor whose output only enters as x0, and the
 * solver's own stopping test decides convergence. Weights are BF16 with an FP32
 * master copy (bf16_weights = 0 keeps FP32 weights, for gradient checks); every
 * product accumulates in FP32; activations are FP32, NCHW.
 * Layers (3x3, padding 1, ReLU): 2->16->16 | pool | 16->32->32 | pool | 32->64->64 |
 * pool | 64->64->64 | up, concat | 128->64->64 | up, concat | 96->32->32 | up,
 * concat | 48->16->16 | 1x1 16->1, then smooth_passes passes of the fixed filter
 * [1 2 1]/4 x [1 2 1]/4 (zero outside the grid). Pooling: 2x2 mean; upsampling: nearest.
 * Parameters: one flat FP32 vector, per layer W[co][ci][kh][kw] then b[co].
 * input: DEVICE (batch, 2, H, W) float32; output/target: DEVICE (batch, 1, H, W). */
typedef struct x0net_s* x0net;
int x0net_create(x0net* out, int H, int W, int batch_max, int bf16_weights, int smooth_passes);
int x0net_destroy(x0net X);
int x0net_num_params(x0net X, int64_t* n);
/* Adds w * mean((kappa A out - f_hat)^2) to the loss (w = 0: mean-squared error only), for
 * the operator the features encode: channel 0 = f_hat = f / s_f, channel 1 = beta / 20, A the
 * h^2-scaled operator of -Lap u + beta (u_x + u_y) on the H x W interior grid, h = 1/(H+1),
 * and out the solution divided by kappa s_f. The residual term penalises the rough error
 * components that A amplifies in ||f - A x0||. */
int x0net_set_residual_weight(x0net X, float w, float kappa);
/* params: host or device float32 array of x0net_num_params values; resets Adam */
int x0net_set_params(x0net X, const float* params, void* stream);
int x0net_get_params(x0net X, float* params, void* stream);
/* The training state: FP32 master weights, Adam's first and second moments (num_params
 * floats each, host or device pointers) and the Adam step count. get synchronises
 * `stream`; set also re-derives the BF16 weights. Saving the state after a step and
 * setting it on a fresh network resumes training bit for bit (every kernel of a step
 * reduces in a fixed order). */
int x0net_get_state(x0net X, float* params, float* m, float* v, int64_t* step, void* stream);
int x0net_set_state(x0net X, const float* params, const float* m, const float* v, int64_t step, void* stream);
int x0net_forward(x0net X, const float* input, float* output, int batch, void* stream);
/* The scalings of the learned form, on the device (the network works on O(1) data):
 *   x0net_features: for each of `batch` systems on an H x W grid (f, beta: DEVICE, batch x H x W
 *     doubles, system b at offset b H W), f_scale[b] = s_f = sqrt(mean f_b^2) (1 when f_b = 0;
 *     DEVICE, batch doubles) and input[b] = (f_b / s_f, beta_b / 20) as float32
 *     (DEVICE, (batch, 2, H, W)).
 *   x0net_targets: target[b] = x_b / (kappa s_f[b]) as float32 (training pairs), kappa =
 *     1 / (2 pi^2 h^2), h = 1 / (H + 1): the inverse of the smallest eigenvalue of the h^2-scaled
 *     Laplacian, so the targets are O(1) on any grid.
 *   x0net_predict: the forward pass and x0[b] = kappa s_f[b] out[b] (DEVICE, batch x H x W
 *     doubles): the initial guess the solver takes.
 * Stream-ordered; SSTEP_ERR_ARG for null pointers, sizes below 1 or batch > batch_max. */
int x0net_features(int H, int W, int batch, const double* f, const double* beta, float* input, double* f_scale,
                   void* stream);
int x0net_targets(int H, int W, int batch, const double* x, const double* f_scale, float* target, void* stream);
int x0net_predict(x0net X, const float* input, const double* f_scale, int batch, double* x0, void* stream);
/* loss = mean over batch*H*W of (out - target)^2 and its gradient with respect to
 * every parameter (host or device outputs; either may be NULL). Synchronises. */
int x0net_gradient(x0net X, const float* input, const float* target, int batch, float* loss, float* grads,
                   void* stream);
/* one Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the mean-squared loss;
 * loss_dev (DEVICE, may be NULL) receives the loss before the step. */
/* BF16 mode: run the 3x3 convolutions (forward and backward-data) on the tensor cores
 * (tcgen05 implicit GEMM, FP32 activations split into three BF16 parts, FP32 accumulation;
 * default on) or on the CUDA cores (on = 0). The FP32-weight mode always uses the CUDA
 * cores. */
int x0net_set_tensor_cores(x0net X, int on);
/* Synchronises `stream` and reports SSTEP_ERR_TIMEOUT if a tensor-core kernel's bounded
 * wait ran out since the last call (the flag is cleared; x0net_gradient reports it as
 * well). A timed-out kernel waits (bounded again) for its MMAs in flight, frees its
 * tensor memory and skips its output; the CUDA context stays usable. */
int x0net_status(x0net X, void* stream);
/* Polls per bounded wait of the tensor-core kernels before it counts as timed out
 * (negative: the default, 2^24). A test sets 0, so every first wait runs out at once,
 * to exercise the timeout path; the drain before freeing tensor memory always uses the
 * default limit. */
int x0net_set_wait_limit(x0net X, int64_t polls);
int x0net_train_step(x0net X, const float* input, const float* target, int batch, float lr, float* loss_dev,
                     void* stream);

/* ------------------------------------------------------------------ launch tracing
 * The library counts every kernel launch of the solvers per kernel kind. With
 * tracing on, it also brackets each launch with a pair of CUDA events recorded on
 * the launching stream and, at the end of each solve, adds the elapsed times per
 * kind (each pair costs about a microsecond of stream time). Process-global and
 * not thread-safe: meant for benchmarks and profiling. enable() resets the totals. */
int sstep_trace_enable(int on);
/* Only the kinds whose bit is set in kind_mask (bit k = kind k) get event pairs; the
 * others are still counted. Default: every kind. Lets a benchmark time one kernel kind
 * inside its timed region without bracketing every launch. */
int sstep_trace_select(unsigned kind_mask);
int sstep_trace_kinds(void);                       /* number of kernel kinds */
const char* sstep_trace_kind_name(int kind);       /* e.g. "gram", "block_update" */
int sstep_trace_read(int kind, double* total_ms, int64_t* launches);  /* host outputs */

#ifdef __cplusplus
}
#endif
#endif /* SSTEP_H */
