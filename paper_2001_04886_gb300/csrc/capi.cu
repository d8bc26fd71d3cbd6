// C ABI: matrix handles, kernel-level entry points and the solver drivers.
//
// The drivers only enqueue kernels and read back a small status header: every
// arithmetic step of the solvers runs on the device (kernels.cu). One host
// synchronisation per GMRES cycle, or per batch of Orthomin steps, decides
// whether to continue.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <complex>
#include <new>
#include <vector>

#include <chrono>

#include "kernels.cuh"
#include "smooth.cuh"

using namespace sstep;

struct sstep_matrix_s {
    StencilDesc A;
    std::vector<double> shifts;      // Newton-basis shifts of the last s-step GMRES solve (host)
    double* rbilu = nullptr;         // red-black ILU(0) reciprocal pivots (device, n), built on first use
    double* nilu = nullptr;          // natural-ordering ILU(0) factors (device, (dim + 1) n), built on first use
    double norm_inf = 0.0;
    double* fields = nullptr;        // owned copies of variable coefficients (7 x n)
    float2* fields_df = nullptr;     // the same as float pairs (mixed-precision kernels)
    // solver workspace, grown on demand
    char* ws = nullptr;
    size_t ws_bytes = 0;
    SolverState* hdr = nullptr;      // pinned host copy of the state
};

namespace {

constexpr size_t kAlign = 256;
// column bounds of the tensor-core passes: m + 1 basis columns, then s + 1 power columns
// per block, then s + 1 updated columns per block (m + 1 + 2 (m / s)(s + 1) <= 5 SSTEP_MAX_M + 1)
constexpr int kBndSlots = 8 * SSTEP_MAX_M;
inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }
inline int64_t col_ld(int64_t n) { return (n + 31) / 32 * 32; }   // 256-byte aligned columns

#define CUDA_TRY(expr)                                  \
    do {                                                \
        cudaError_t e_ = (expr);                        \
        if (e_ != cudaSuccess) return SSTEP_ERR_CUDA;   \
    } while (0)

int check_launch() { return cudaGetLastError() == cudaSuccess ? SSTEP_OK : SSTEP_ERR_CUDA; }

// ------------------------------------------------------------------ Newton-basis shifts
// Real parts of the eigenvalues of the K x K upper Hessenberg matrix held in G
// (column-major, leading dimension ld): single-shift QR steps in complex arithmetic
// (complex Givens rotations, Wilkinson shift = the eigenvalue of the trailing 2 x 2
// nearer its last diagonal entry, so complex pairs converge like real eigenvalues) on
// the active unreduced block, deflating where a subdiagonal entry is negligible next to
// its diagonal neighbours; every 10th step without deflation takes an exceptional
// shift. Returns false if the iteration does not settle within 100 K steps.
bool hessenberg_real_parts(const double* G, int ld, int K, std::vector<double>& out) {
    typedef std::complex<double> cplx;
    out.clear();
    std::vector<cplx> H((size_t)K * K, cplx(0.0, 0.0));   // row-major
    for (int j = 0; j < K; ++j)
        for (int i = 0; i <= std::min(j + 1, K - 1); ++i) H[(size_t)i * K + j] = G[i + (size_t)j * ld];
    auto h = [&](int i, int j) -> cplx& { return H[(size_t)i * K + j]; };
    const double eps = 2.220446049250313e-16;
    std::vector<double> cs(K);
    std::vector<cplx> sn(K);
    int hi = K - 1, steps = 0, stall = 0;
    while (hi >= 0) {
        if (hi == 0) {
            out.push_back(h(0, 0).real());
            break;
        }
        int lo = hi;
        while (lo > 0 && std::abs(h(lo, lo - 1)) > eps * (std::abs(h(lo, lo)) + std::abs(h(lo - 1, lo - 1)))) --lo;
        if (lo > 0) h(lo, lo - 1) = 0.0;
        if (lo == hi) {
            out.push_back(h(hi, hi).real());
            --hi;
            stall = 0;
            continue;
        }
        if (++steps > 100 * K) return false;
        const cplx a = h(hi - 1, hi - 1), b = h(hi - 1, hi), c = h(hi, hi - 1), d = h(hi, hi);
        const cplx half = 0.5 * (a - d), root = std::sqrt(half * half + b * c);
        const cplx r1 = 0.5 * (a + d) + root, r2 = 0.5 * (a + d) - root;
        cplx mu = std::abs(r1 - d) < std::abs(r2 - d) ? r1 : r2;
        if (++stall % 10 == 0) mu = d + 0.75 * std::abs(c);
        for (int i = lo; i <= hi; ++i) h(i, i) -= mu;
        for (int k = lo; k < hi; ++k) {   // Q^H (H - mu I) = R, rotation k on rows k, k+1
            const cplx x = h(k, k), y = h(k + 1, k);
            const double ax = std::abs(x), r = std::sqrt(ax * ax + std::norm(y));
            double cc = 1.0;
            cplx ss(0.0, 0.0);
            if (r > 0.0) {
                if (ax == 0.0) {
                    cc = 0.0;
                    ss = 1.0;
                } else {
                    cc = ax / r;
                    ss = (x / ax) * std::conj(y) / r;
                }
            }
            cs[k] = cc;
            sn[k] = ss;
            for (int j = k; j <= hi; ++j) {
                const cplx t1 = h(k, j), t2 = h(k + 1, j);
                h(k, j) = cc * t1 + ss * t2;
                h(k + 1, j) = -std::conj(ss) * t1 + cc * t2;
            }
        }
        for (int k = lo; k < hi; ++k) {   // R Q + mu I
            const double cc = cs[k];
            const cplx ss = sn[k];
            for (int i = lo; i <= std::min(k + 2, hi); ++i) {
                const cplx t1 = h(i, k), t2 = h(i, k + 1);
                h(i, k) = cc * t1 + std::conj(ss) * t2;
                h(i, k + 1) = -ss * t1 + cc * t2;
            }
        }
        for (int i = lo; i <= hi; ++i) h(i, i) += mu;
    }
    return (int)out.size() == K;
}

// The first `count` points of the Leja ordering of the (ascending) values: the largest in
// modulus first, then each next point maximises the sum of the logarithms of its
// distances to the points taken (ties go to the earlier value); points within
// 1e-10 max|v| of a taken one (the real parts of a complex pair) are skipped; the
// sequence repeats when the distinct values run out.
std::vector<double> leja_order(std::vector<double> v, int count) {
    std::sort(v.begin(), v.end());
    std::vector<double> seq;
    if (v.empty()) return std::vector<double>(count, 0.0);
    double vmax = 0.0;
    for (double t : v) vmax = std::max(vmax, fabs(t));
    const double tiny = 1e-10 * vmax;
    std::vector<char> used(v.size(), 0);
    size_t first = 0;
    for (size_t i = 1; i < v.size(); ++i)
        if (fabs(v[i]) > fabs(v[first])) first = i;
    used[first] = 1;
    seq.push_back(v[first]);
    for (;;) {
        int best = -1;
        double best_score = 0.0;
        for (size_t i = 0; i < v.size(); ++i) {
            if (used[i]) continue;
            double score = 0.0;
            bool zero = false;
            for (double t : seq) {
                const double dd = fabs(v[i] - t);
                if (dd <= tiny) {
                    zero = true;
                    break;
                }
                score += log(dd);
            }
            if (zero) continue;
            if (best < 0 || score > best_score) {
                best = (int)i;
                best_score = score;
            }
        }
        if (best < 0) break;
        used[best] = 1;
        seq.push_back(v[best]);
    }
    std::vector<double> out(count);
    for (int j = 0; j < count; ++j) out[j] = seq[j % seq.size()];
    return out;
}

// After the first cycle: the shifts from its Hessenberg G (device), written to the
// device state (st->theta) and returned; empty (monomial kept) if the QR does not settle.
std::vector<double> newton_shifts_from_device(const double* G_dev, int m, int K, int s, double* theta_dev,
                                              cudaStream_t stream) {
    std::vector<double> G((size_t)(m + 1) * m);
    if (K < 1 || cudaMemcpyAsync(G.data(), G_dev, sizeof(double) * G.size(), cudaMemcpyDeviceToHost, stream) !=
                     cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return {};
    std::vector<double> ev;
    if (!hessenberg_real_parts(G.data(), m + 1, K, ev)) return {};
    std::vector<double> th = leja_order(ev, s);
    if (cudaMemcpyAsync(theta_dev, th.data(), sizeof(double) * s, cudaMemcpyHostToDevice, stream) != cudaSuccess)
        return {};
    return th;
}

// The fused matrix-powers kernel (one launch for the s powers of a block) is off by
// default: on GB300 the 16.8 MB columns of a 128^3 solve stay in the 129 MB L2 between
// separate sweeps, so fusion saves only L2 reads while its tile halos recompute ~4x the
// points (measured slower). SSTEP_FUSED_POWERS=1 turns it on, in the mixed-precision solver
// and in the FP64 one (powers.cu; there the halos' extra multiply-adds fall on the FP64 pipe,
// which already bounds the separate sweeps).
// The Gram pass of the FP64 s-step GMRES runs on the tensor cores (exact fixed point,
// ozaki.cu) unless SSTEP_TC_GRAM=0 selects the FP64 CUDA-core kernel (for comparisons).
bool tc_gram_enabled() {
    static const bool on = [] {
        const char* v = getenv("SSTEP_TC_GRAM");
        return !(v && v[0] == '0');
    }();
    return on;
}

// The tensor-core passes read the basis from its kept fixed-point words (a second panel
// written by the Gram pass of each block) unless SSTEP_TC_WORDS=0 makes them convert the
// FP64 columns every time (for comparisons).
bool tc_words_enabled() {
    static const bool on = [] {
        const char* v = getenv("SSTEP_TC_WORDS");
        return !(v && v[0] == '0');
    }();
    return on;
}

bool fused_powers_enabled() {
    static const bool on = [] {
        const char* v = getenv("SSTEP_FUSED_POWERS");
        return v && v[0] == '1';
    }();
    return on;
}

// ------------------------------------------------------------------ launch tracing
// Every launch is counted; when tracing is on, a pair of CUDA events brackets each
// launch on its own stream and the elapsed times are summed per kernel kind at the
// end of the call that issued them.
enum Kind { K_STENCIL = 0, K_RESIDUAL, K_GRAM, K_UPDATE, K_NEXT, K_AXPY, K_OMIN_XR, K_OMIN_PUPDATE, K_LSQ, K_PRECOND,
            K_COUNT };
const char* const kKindNames[K_COUNT] = {"stencil_powers", "residual", "gram", "block_update", "next_vector",
                                         "basis_axpy", "omin_xr", "omin_pupdate", "lsq_solve", "precond"};
struct Tracer {
    bool on = false;
    unsigned mask = ~0u;          // kinds that get event pairs
    std::vector<cudaEvent_t> events;
    std::vector<int> kinds;       // kind of each recorded pair
    size_t used = 0;              // events in use (pairs * 2)
    double total_ms[K_COUNT] = {0};
    long long launches[K_COUNT] = {0};
};
Tracer g_trace;

int trace_begin(int kind, cudaStream_t s) {
    g_trace.launches[kind] += 1;
    if (!g_trace.on || !((g_trace.mask >> kind) & 1u)) return -1;
    if (g_trace.used + 2 > g_trace.events.size()) {
        for (int i = 0; i < 256; ++i) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return -1;
            g_trace.events.push_back(e);
        }
    }
    int idx = (int)g_trace.used;
    g_trace.used += 2;
    g_trace.kinds.push_back(kind);
    cudaEventRecord(g_trace.events[idx], s);
    return idx;
}

void trace_end(int idx, cudaStream_t s) {
    if (idx >= 0) cudaEventRecord(g_trace.events[idx + 1], s);
}

// Adds up the recorded pairs (their stream must have been synchronised).
void trace_collect() {
    for (size_t i = 0; i < g_trace.kinds.size(); ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, g_trace.events[2 * i], g_trace.events[2 * i + 1]) == cudaSuccess)
            g_trace.total_ms[g_trace.kinds[i]] += ms;
    }
    cudaGetLastError();
    g_trace.kinds.clear();
    g_trace.used = 0;
}

#define TRACED(kind, stream, call)                   \
    do {                                             \
        int tr_ = trace_begin((kind), (stream));     \
        call;                                        \
        trace_end(tr_, (stream));                    \
    } while (0)

// ||A||_inf of a constant stencil: per axis a row has both neighbours (side >= 3),
// exactly one of them (side 2) or none (side 1); axes are independent.
double row_norm_inf_const(const StencilDesc& A) {
    const int sz[3] = {A.nx, A.ny, A.nz};
    double t = fabs(A.c[0]);
    for (int d = 0; d < A.dim; ++d) {
        const double lo = fabs(A.c[1 + 2 * d]), hi = fabs(A.c[2 + 2 * d]);
        if (sz[d] >= 3) t += lo + hi;
        else if (sz[d] == 2) t += std::max(lo, hi);
    }
    return t;
}

// hi = c rounded to float, lo = the rest rounded to float: c = hi + lo to ~48 bits
void split_coefficients(StencilDesc& A) {
    for (int q = 0; q < 7; ++q) {
        A.ch[q] = (float)A.c[q];
        A.cl[q] = (float)(A.c[q] - (double)A.ch[q]);
    }
}

int make_desc(StencilDesc& A, int dim, const int64_t shape[3]) {
    if (dim != 2 && dim != 3) return SSTEP_ERR_ARG;
    if (!shape) return SSTEP_ERR_ARG;
    int64_t nx = shape[0], ny = shape[1], nz = dim == 3 ? shape[2] : 1;
    if (nx < 1 || ny < 1 || nz < 1) return SSTEP_ERR_ARG;
    int64_t n = nx * ny * nz;
    if (nx > (1 << 30) || ny > (1 << 30) || nz > (1 << 30) || n >= (int64_t)1 << 31) return SSTEP_ERR_ARG;
    memset(&A, 0, sizeof(A));
    A.dim = dim;
    A.nx = (int)nx;
    A.ny = (int)ny;
    A.nz = (int)nz;
    A.n = n;
    return SSTEP_OK;
}

// Device workspace of one solve. Small arrays first, then the columns.
struct Layout {
    size_t state, L, T, S, G, R, gc, gs, g, y, hist, C, a, theta, counter, bnd, ozacc, partials, cols;
    size_t total;
};

Layout plan(int64_t n, int ncols, int m, int hist_cap, size_t elem_bytes = sizeof(double)) {
    Layout l;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off = align_up(off + bytes);
        return at;
    };
    const int mm = std::max(m, 1);
    l.state = take(sizeof(SolverState));
    l.L = take(sizeof(double) * kMaxCols * kMaxS * 2);
    l.T = take(sizeof(double) * kMaxCols * (kMaxS + 1));
    l.S = take(sizeof(double) * kMaxCols);
    l.G = take(sizeof(double) * (mm + 1) * mm);
    l.R = take(sizeof(double) * (mm + 1) * mm);
    l.gc = take(sizeof(double) * mm);
    l.gs = take(sizeof(double) * mm);
    l.g = take(sizeof(double) * (mm + 1));
    l.y = take(sizeof(double) * kMaxCols);
    l.hist = take(sizeof(double) * std::max(hist_cap, 1));
    l.C = take(sizeof(double) * kMaxCols * (kMaxS + 1));
    l.a = take(sizeof(double) * kMaxCols);
    l.theta = take(sizeof(double) * kMaxS);
    l.counter = take(kAlign);
    l.bnd = take(sizeof(unsigned) * kBndSlots);
    l.ozacc = take(sizeof(unsigned long long) * kOzAccWords);
    l.partials = take(sizeof(double) * (size_t)max_partials_doubles());
    l.cols = take(elem_bytes * (size_t)col_ld(n) * ncols);
    l.total = off;
    return l;
}

// A cap on the solver workspace (0: none), for tests of the allocation-failure path.
int64_t g_workspace_limit = 0;

int ensure_workspace(sstep_matrix M, size_t bytes) {
    if (g_workspace_limit > 0 && (int64_t)bytes > g_workspace_limit) return SSTEP_ERR_OOM;
    if (!M->hdr) {
        if (cudaMallocHost((void**)&M->hdr, sizeof(SolverState)) != cudaSuccess) {
            M->hdr = nullptr;
            return SSTEP_ERR_OOM;
        }
    }
    if (M->ws_bytes >= bytes) return SSTEP_OK;
    if (M->ws) cudaFree(M->ws);
    M->ws = nullptr;
    M->ws_bytes = 0;
    if (cudaMalloc((void**)&M->ws, bytes) != cudaSuccess) {
        cudaGetLastError();
        return SSTEP_ERR_OOM;
    }
    M->ws_bytes = bytes;
    return SSTEP_OK;
}

// Host image of the state with its device pointers filled in.
SolverState init_state(const Layout& l, char* ws, const sstep_params* p, int s, int m, int k) {
    SolverState h;
    memset(&h, 0, sizeof(h));
    h.active = 1;
    h.building = 1;
    h.status = SSTEP_NOT_CONVERGED;
    h.s = s;
    h.m = m;
    h.k = k;
    h.nb = s > 0 ? m / s : 0;
    h.max_cycles = p->max_cycles;
    h.max_iters = p->max_iters;
    h.hist_cap = p->history ? p->history_cap : 0;
    h.tol = p->tol;
    h.L = (double*)(ws + l.L);
    h.T = (double*)(ws + l.T);
    h.S = (double*)(ws + l.S);
    h.G = (double*)(ws + l.G);
    h.R = (double*)(ws + l.R);
    h.gc = (double*)(ws + l.gc);
    h.gs = (double*)(ws + l.gs);
    h.g = (double*)(ws + l.g);
    h.y = (double*)(ws + l.y);
    h.hist = (double*)(ws + l.hist);
    h.C = (double*)(ws + l.C);
    h.a = (double*)(ws + l.a);
    h.theta = (double*)(ws + l.theta);
    return h;
}

int common_checks(sstep_matrix A, const double* f, double* x, const sstep_params* p, sstep_result* res) {
    if (!A || !f || !x || !p || !res) return SSTEP_ERR_ARG;
    if (!(p->tol > 0.0)) return SSTEP_ERR_ARG;
    if (p->history && p->history_cap < 0) return SSTEP_ERR_ARG;
    if (p->sigma < 0.0 || !isfinite(p->sigma)) return SSTEP_ERR_ARG;
    return SSTEP_OK;
}

// Copies the final state into res and the history into the caller's host array.
int finish(sstep_matrix M, const Layout& l, SolverState* st, const double* f, const double* x,
           const sstep_params* p, sstep_result* res, cudaStream_t stream) {
    Scratch sc{(double*)(M->ws + l.partials), (unsigned*)(M->ws + l.counter)};
    Epi e;
    e.mode = EPI_FINAL;
    e.st = st;
    TRACED(K_RESIDUAL, stream, launch_residual(M->A, f, x, nullptr, sc, e, GATE_NONE, stream));
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(M->hdr, st, sizeof(SolverState), cudaMemcpyDeviceToHost, stream));
    CUDA_TRY(cudaStreamSynchronize(stream));
    trace_collect();
    const SolverState& h = *M->hdr;
    res->status = h.status;
    res->cycles = h.cycles;
    res->iters = h.iters;
    res->matvecs = h.matvecs;
    res->relres = h.relres;
    int nh = std::min(h.hist_len, h.hist_cap);
    res->history_len = nh;
    if (p->history && nh > 0) {
        CUDA_TRY(cudaMemcpy(p->history, M->ws + l.hist, sizeof(double) * nh, cudaMemcpyDeviceToHost));
    }
    return SSTEP_OK;
}

int read_header(sstep_matrix M, SolverState* st, cudaStream_t stream) {
    CUDA_TRY(cudaMemcpyAsync(M->hdr, st, sizeof(SolverState), cudaMemcpyDeviceToHost, stream));
    CUDA_TRY(cudaStreamSynchronize(stream));
    return SSTEP_OK;
}

// x0_guard: when ||f - A x0|| > ||f|| (st->nf already set), start from x0 = 0
int apply_x0_guard(sstep_matrix M, const Layout& l, SolverState* st, const double* f, double* x,
                   cudaStream_t stream) {
    Scratch sc{(double*)(M->ws + l.partials), (unsigned*)(M->ws + l.counter)};
    Epi e;
    e.mode = EPI_FINAL;
    e.st = st;
    launch_residual(M->A, f, x, nullptr, sc, e, GATE_NONE, stream);
    CUDA_TRY(cudaGetLastError());
    int rc = read_header(M, st, stream);
    if (rc) return rc;
    if (!(M->hdr->relres <= 1.0)) CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * M->A.n, stream));
    return SSTEP_OK;
}


// ------------------------------------------------------------------ mixed-precision basis drivers
// The same kernel sequences as the FP64 drivers below, with the basis columns in
// the storage type of P (double-float pairs or FP32); f, x and all scalar work FP64.
template <int P>
int sstep_gmres_mp(sstep_matrix M, const double* f, double* x, const sstep_params* p, sstep_result* res,
                   cudaStream_t stream_) {
    int rc;
    const int s = p->s, m = p->m;
    const int64_t n = M->A.n, ld = col_ld(n);
    const size_t eb = prec_bytes(P);
    Layout l = plan(n, m + 2, m, p->history ? p->history_cap : 0, eb);
    if ((rc = ensure_workspace(M, l.total))) return rc;
    SolverState h = init_state(l, M->ws, p, s, m, 0);
    h.sigma = p->sigma > 0.0 ? p->sigma : 1.0 / M->norm_inf;
    SolverState* st = (SolverState*)(M->ws + l.state);
    char* U = M->ws + l.cols;
    auto col = [&](int j) { return (void*)(U + (size_t)j * ld * eb); };
    void* uraw = col(m + 1);
    Scratch sc{(double*)(M->ws + l.partials), (unsigned*)(M->ws + l.counter)};
    CUDA_TRY(cudaMemcpyAsync(st, &h, sizeof(h), cudaMemcpyHostToDevice, stream_));
    CUDA_TRY(cudaMemsetAsync(M->ws + l.counter, 0, kAlign, stream_));
    CUDA_TRY(cudaMemsetAsync(M->ws + l.G, 0, sizeof(double) * (m + 1) * m, stream_));
    CUDA_TRY(cudaMemsetAsync(M->ws + l.theta, 0, sizeof(double) * kMaxS, stream_));
    Epi e;
    e.st = st;
    e.mode = EPI_NF;
    TRACED(K_RESIDUAL, stream_, launch_residual(M->A, f, nullptr, nullptr, sc, e, GATE_NONE, stream_));
    if (p->x0_guard && (rc = apply_x0_guard(M, l, st, f, x, stream_))) return rc;
    const double sigma = h.sigma;
    const int nb = m / s;
    std::vector<double> theta(s, 0.0);   // Newton shifts (zero: monomial powers)
    bool shifted = false;
    M->shifts.clear();
    for (;;) {
        e = Epi();
        e.st = st;
        e.mode = EPI_RESTART;
        TRACED(K_RESIDUAL, stream_, mp_launch_residual<P>(M->A, f, x, uraw, sc, e, GATE_ACTIVE, stream_));
        for (int k = 0; k < nb; ++k) {
            const int o = k * s;
            // Alg. 4.1 step 3: the s powers, in one fused launch when enabled (SSTEP_FUSED_POWERS=1)
            bool fused = false;
            if (fused_powers_enabled() && !shifted)
                TRACED(K_STENCIL, stream_,
                       fused = mp_launch_powers_fused<P>(M->A, uraw, col(o), ld, s, sigma, &st->vscale, st,
                                                         GATE_BUILDING, stream_));
            if (!fused) {
                TRACED(K_STENCIL, stream_, mp_launch_stencil<P>(M->A, uraw, sigma, col(o + 1), 1.0, col(o),
                                                                &st->vscale, st, GATE_BUILDING, stream_, theta[0]));
                for (int j = 2; j <= s; ++j)
                    TRACED(K_STENCIL, stream_, mp_launch_stencil<P>(M->A, col(o + j - 1), sigma, col(o + j), 0.0,
                                                                    nullptr, nullptr, st, GATE_BUILDING, stream_,
                                                                    theta[j - 1]));
            }
            if (k > 0) {
                e = Epi();
                e.st = st;
                e.mode = EPI_GM_T;
                e.o = o;
                TRACED(K_GRAM, stream_, mp_launch_gram<P>(n, col(0), ld, o, col(o + 1), ld, s, sc, e, GATE_BUILDING,
                                                          stream_));
            }
            e = Epi();
            e.st = st;
            e.mode = EPI_GM_W;
            e.o = o;
            TRACED(K_UPDATE, stream_, mp_launch_update<P>(n, col(0), ld, o, col(o), ld, col(o), ld, s + 1, 1, h.T, m,
                                                          -1.0, true, sc, e, GATE_BUILDING, stream_));
            e = Epi();
            e.st = st;
            e.mode = EPI_GM_NU;
            e.o = o;
            e.lastblock = (k == nb - 1);
            TRACED(K_NEXT, stream_, mp_launch_update<P>(n, col(o), ld, s, col(o + s), ld, uraw, ld, 1, 0, h.S, s, -1.0,
                                                        true, sc, e, GATE_BUILDING, stream_));
        }
        TRACED(K_LSQ, stream_, launch_lsq_solve(st, GATE_ACTIVE, stream_));
        e = Epi();
        e.st = st;
        TRACED(K_AXPY, stream_, mp_launch_axpy<P>(n, col(0), ld, x, e, GATE_ACTIVE, stream_));
        CUDA_TRY(cudaGetLastError());
        if ((rc = read_header(M, st, stream_))) return rc;
        if (!M->hdr->active) break;
        if (p->basis == SSTEP_BASIS_NEWTON && !shifted) {   // shifts from the first cycle's Ritz values
            std::vector<double> th = newton_shifts_from_device(h.G, m, M->hdr->K, s, h.theta, stream_);
            if (!th.empty()) {
                theta = th;
                M->shifts = th;
            }
            shifted = true;
        }
    }
    return finish(M, l, st, f, x, p, res, stream_);
}

template <int P>
int gmres_mp(sstep_matrix M, const double* f, double* x, const sstep_params* p, sstep_result* res,
             cudaStream_t stream_) {
    int rc;
    const int m = p->m;
    const int64_t n = M->A.n, ld = col_ld(n);
    const size_t eb = prec_bytes(P);
    Layout l = plan(n, m + 3, m, p->history ? p->history_cap : 0, eb);
    if ((rc = ensure_workspace(M, l.total))) return rc;
    SolverState h = init_state(l, M->ws, p, 1, m, 0);
    h.sigma = 1.0;
    SolverState* st = (SolverState*)(M->ws + l.state);
    char* U = M->ws + l.cols;
    auto col = [&](int j) { return (void*)(U + (size_t)j * ld * eb); };
    void* wraw = col(m + 1);
    void* ybuf = col(m + 2);
    Scratch sc{(double*)(M->ws + l.partials), (unsigned*)(M->ws + l.counter)};
    CUDA_TRY(cudaMemcpyAsync(st, &h, sizeof(h), cudaMemcpyHostToDevice, stream_));
    CUDA_TRY(cudaMemsetAsync(M->ws + l.counter, 0, kAlign, stream_));
    CUDA_TRY(cudaMemsetAsync(M->ws + l.G, 0, sizeof(double) * (m + 1) * m, stream_));
    Epi e;
    e.st = st;
    e.mode = EPI_NF;
    TRACED(K_RESIDUAL, stream_, launch_residual(M->A, f, nullptr, nullptr, sc, e, GATE_NONE, stream_));
    if (p->x0_guard && (rc = apply_x0_guard(M, l, st, f, x, stream_))) return rc;
    for (;;) {
        e = Epi();
        e.st = st;
        e.mode = EPI_RESTART;
        TRACED(K_RESIDUAL, stream_, mp_launch_residual<P>(M->A, f, x, wraw, sc, e, GATE_ACTIVE, stream_));
        for (int j = 0; j < m; ++j) {
            TRACED(K_STENCIL, stream_, mp_launch_stencil<P>(M->A, wraw, 1.0, ybuf, 1.0, col(j), &st->vscale, st,
                                                            GATE_BUILDING, stream_));
            e = Epi();
            e.st = st;
            e.mode = EPI_ST_H;
            e.o = j;
            TRACED(K_GRAM, stream_, mp_launch_gram<P>(n, col(0), ld, j + 1, ybuf, ld, 1, sc, e, GATE_BUILDING, stream_));
            e = Epi();
            e.st = st;
            e.mode = EPI_ST_NORM;
            e.o = j;
            e.lastblock = (j == m - 1);
            TRACED(K_UPDATE, stream_, mp_launch_update<P>(n, col(0), ld, j + 1, ybuf, ld, wraw, ld, 1, 0,
                                                          h.G + (int64_t)j * (m + 1), m + 1, -1.0, true, sc, e,
                                                          GATE_BUILDING, stream_));
        }
        TRACED(K_LSQ, stream_, launch_lsq_solve(st, GATE_ACTIVE, stream_));
        e = Epi();
        e.st = st;
        TRACED(K_AXPY, stream_, mp_launch_axpy<P>(n, col(0), ld, x, e, GATE_ACTIVE, stream_));
        CUDA_TRY(cudaGetLastError());
        if ((rc = read_header(M, st, stream_))) return rc;
        if (!M->hdr->active) break;
    }
    return finish(M, l, st, f, x, p, res, stream_);
}


}  // namespace

// ------------------------------------------------------------------ batched solves
struct sstep_batch_s {
    int nsys = 0, s = 0, m = 0;
    sstep_params p{};
    std::vector<sstep_matrix> mats;
    std::vector<int> order_largest;      // system indices, largest n first
    char* ws = nullptr;                  // states, small arrays, basis panels
    size_t ws_bytes = 0;
    BatchSys* d_sys = nullptr;           // device descriptors
    int* d_order = nullptr;              // device copy of the queue order (largest first)
    unsigned* d_queue = nullptr;
    std::vector<BatchSys> h_sys;
    std::vector<SolverState> h_init;     // initial states, kBatchCopies per system
    SolverState* d_init = nullptr;       // the same on the device
    SolverState* h_states = nullptr;     // pinned copy back
    std::vector<size_t> state_off;
    // launch configuration (autotuned)
    int threads = 256, ctas_per_sm = 2, largest_first = 1, cluster = 1;
    int64_t nbig = 0;                    // systems with n >= nbig get a whole cluster
    cudaGraphExec_t graph = nullptr;
    int64_t graph_cfg[5] = {0, 0, 0, 0, 0};
};

namespace {

constexpr int kBatchMaxM = 40;

// Per-system state plus small arrays, laid out like plan() of one solve.
size_t batch_state_bytes(int m) {
    Layout l = plan(0, 0, m, 0);
    return align_up(l.partials);   // state .. counter (no partials, no columns)
}

SolverState batch_state(char* base, int m, int s, const sstep_params* p, double sigma) {
    Layout l = plan(0, 0, m, 0);
    sstep_params q = *p;
    q.history = nullptr;
    q.history_cap = 0;
    SolverState h = init_state(l, base, &q, s, m, 0);
    h.sigma = sigma;
    h.pad_ = p->x0_guard ? 1 : 0;   // the batched kernel reads the x0 guard here
    return h;
}

int batch_graph(sstep_batch B, cudaStream_t stream) {
    const int64_t cfg[5] = {B->threads, B->ctas_per_sm, B->largest_first, B->cluster, B->nbig};
    if (B->graph && memcmp(cfg, B->graph_cfg, sizeof(cfg)) == 0) return SSTEP_OK;
    if (B->graph) {
        cudaGraphExecDestroy(B->graph);
        B->graph = nullptr;
    }
    int dev = 0, sms = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const bool f32 = B->p.precision == SSTEP_PREC_FP32;
    const int grid = batched_grid(B->s, B->threads, sms * B->ctas_per_sm, B->cluster, f32);
    if (grid < 1) return SSTEP_ERR_ARG;
    cudaStream_t cap;
    CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t g;
    int rc = SSTEP_OK;
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = SSTEP_ERR_CUDA;
    if (!rc) {
        cudaMemsetAsync(B->d_queue, 0, sizeof(unsigned), cap);
        launch_batch_init(B->d_init, B->d_sys, B->nsys, cap);
        if (launch_batched(B->d_sys, B->largest_first ? B->d_order : nullptr, B->nsys, B->d_queue, B->s, B->threads,
                           grid, B->cluster, B->nbig, f32, cap))
            rc = SSTEP_ERR_ARG;
        if (cudaStreamEndCapture(cap, &g) != cudaSuccess) rc = SSTEP_ERR_CUDA;
    }
    if (!rc) {
        if (cudaGraphInstantiate(&B->graph, g, 0) != cudaSuccess) rc = SSTEP_ERR_CUDA;
        cudaGraphDestroy(g);
    }
    cudaStreamDestroy(cap);
    cudaGetLastError();
    if (!rc) memcpy(B->graph_cfg, cfg, sizeof(cfg));
    (void)stream;
    return rc;
}

int batch_run_persistent(sstep_batch B, const double* const* f, double* const* x, cudaStream_t stream) {
    for (int i = 0; i < B->nsys; ++i) {
        B->h_sys[i].f = f[i];
        B->h_sys[i].x = x[i];
    }
    CUDA_TRY(cudaMemcpyAsync(B->d_sys, B->h_sys.data(), sizeof(BatchSys) * B->nsys, cudaMemcpyHostToDevice, stream));
    int rc = batch_graph(B, stream);   // the graph resets the queue and every state copy, then solves
    if (rc) return rc;
    CUDA_TRY(cudaGraphLaunch(B->graph, stream));
    return SSTEP_OK;
}

}  // namespace

extern "C" {

int sstep_trace_enable(int on) {
    g_trace.on = on != 0;
    for (int k = 0; k < K_COUNT; ++k) {
        g_trace.total_ms[k] = 0.0;
        g_trace.launches[k] = 0;
    }
    g_trace.kinds.clear();
    g_trace.used = 0;
    return SSTEP_OK;
}

int sstep_trace_select(unsigned kind_mask) {
    g_trace.mask = kind_mask;
    return SSTEP_OK;
}

int sstep_trace_kinds(void) { return K_COUNT; }

const char* sstep_trace_kind_name(int kind) { return (kind >= 0 && kind < K_COUNT) ? kKindNames[kind] : ""; }

int sstep_trace_read(int kind, double* total_ms, int64_t* launches) {
    if (kind < 0 || kind >= K_COUNT) return SSTEP_ERR_ARG;
    if (total_ms) *total_ms = g_trace.total_ms[kind];
    if (launches) *launches = g_trace.launches[kind];
    return SSTEP_OK;
}

const char* sstep_status_string(int status) {
    switch (status) {
        case SSTEP_OK: return "ok";
        case SSTEP_NOT_CONVERGED: return "not converged";
        case SSTEP_ERR_ARG: return "invalid argument";
        case SSTEP_ERR_CUDA: return "CUDA error";
        case SSTEP_ERR_OOM: return "out of device memory";
        case SSTEP_ERR_BREAKDOWN: return "breakdown: non-positive Cholesky pivot in a Gram block";
        case SSTEP_ERR_NAN: return "residual is NaN or Inf";
        case SSTEP_ERR_TIMEOUT: return "a bounded device wait ran out";
        default: return "unknown status";
    }
}

int stencil_matrix_create(sstep_matrix* out, int dim, const int64_t shape[3], const double* coef) {
    if (!out || !coef) return SSTEP_ERR_ARG;
    *out = nullptr;
    StencilDesc A;
    int rc = make_desc(A, dim, shape);
    if (rc) return rc;
    for (int q = 0; q < 2 * dim + 1; ++q) {
        if (!isfinite(coef[q])) return SSTEP_ERR_ARG;
        A.c[q] = coef[q];
    }
    split_coefficients(A);
    sstep_matrix M = new (std::nothrow) sstep_matrix_s;
    if (!M) return SSTEP_ERR_OOM;
    M->A = A;
    M->norm_inf = row_norm_inf_const(A);
    *out = M;
    return SSTEP_OK;
}

int stencil_matrix_create_convdiff(sstep_matrix* out, int dim, const int64_t shape[3], const double* beta) {
    if (!out || !beta || !shape) return SSTEP_ERR_ARG;
    if (dim != 2 && dim != 3) return SSTEP_ERR_ARG;
    for (int d = 1; d < dim; ++d)
        if (shape[d] != shape[0]) return SSTEP_ERR_ARG;
    const double h = 1.0 / (double)(shape[0] + 1);
    double coef[7];
    coef[0] = 2.0 * dim;
    for (int d = 0; d < dim; ++d) {
        const double c = beta[d] * h / 2.0;
        coef[1 + 2 * d] = -1.0 - c;
        coef[2 + 2 * d] = -1.0 + c;
    }
    return stencil_matrix_create(out, dim, shape, coef);
}

int stencil_matrix_create_fields(sstep_matrix* out, int dim, const int64_t shape[3], const double* const* fields,
                                 void* stream) {
    if (!out || !fields) return SSTEP_ERR_ARG;
    *out = nullptr;
    StencilDesc A;
    int rc = make_desc(A, dim, shape);
    if (rc) return rc;
    const int nq = 2 * dim + 1;
    for (int q = 0; q < nq; ++q)
        if (!fields[q]) return SSTEP_ERR_ARG;
    sstep_matrix M = new (std::nothrow) sstep_matrix_s;
    if (!M) return SSTEP_ERR_OOM;
    if (cudaMalloc((void**)&M->fields, sizeof(double) * A.n * nq) != cudaSuccess) {
        cudaGetLastError();
        delete M;
        return SSTEP_ERR_OOM;
    }
    cudaStream_t s = (cudaStream_t)stream;
    for (int q = 0; q < nq; ++q) {
        if (cudaMemcpyAsync(M->fields + q * A.n, fields[q], sizeof(double) * A.n, cudaMemcpyDeviceToDevice, s) !=
            cudaSuccess) {
            cudaFree(M->fields);
            delete M;
            return SSTEP_ERR_CUDA;
        }
        A.f[q] = M->fields + q * A.n;
    }
    A.variable = 1;
    if (cudaMalloc((void**)&M->fields_df, sizeof(float2) * A.n * nq) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(M->fields);
        delete M;
        return SSTEP_ERR_OOM;
    }
    for (int q = 0; q < nq; ++q) {
        launch_split_fields(A.f[q], M->fields_df + q * A.n, A.n, s);
        A.fdf[q] = M->fields_df + q * A.n;
    }
    split_coefficients(A);
    M->A = A;
    // ||A||_inf: reduce on the host from a copy (creation-time only)
    std::vector<double> host((size_t)A.n * nq);
    if (cudaMemcpyAsync(host.data(), M->fields, sizeof(double) * A.n * nq, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaFree(M->fields);
        delete M;
        return SSTEP_ERR_CUDA;
    }
    double best = 0.0;
    for (int64_t p = 0; p < A.n; ++p) {
        int64_t x = p % A.nx, t = p / A.nx, y = t % A.ny, z = t / A.ny;
        double r = fabs(host[p]);
        if (x > 0) r += fabs(host[1 * A.n + p]);
        if (x < A.nx - 1) r += fabs(host[2 * A.n + p]);
        if (y > 0) r += fabs(host[3 * A.n + p]);
        if (y < A.ny - 1) r += fabs(host[4 * A.n + p]);
        if (dim == 3) {
            if (z > 0) r += fabs(host[5 * A.n + p]);
            if (z < A.nz - 1) r += fabs(host[6 * A.n + p]);
        }
        best = std::max(best, r);
    }
    M->norm_inf = best;
    *out = M;
    return SSTEP_OK;
}

int stencil_matrix_create_convdiff_variable(sstep_matrix* out, int64_t N, const double* beta_field, void* stream) {
    if (!out || !beta_field || N < 1 || N > 46340) return SSTEP_ERR_ARG;
    *out = nullptr;
    const int64_t n = N * N;
    double* tmp = nullptr;
    if (cudaMalloc((void**)&tmp, sizeof(double) * n * 5) != cudaSuccess) {
        cudaGetLastError();
        return SSTEP_ERR_OOM;
    }
    cudaStream_t s = (cudaStream_t)stream;
    launch_convdiff_fields(beta_field, 1.0 / (double)(N + 1), n, tmp, s);
    const double* f[5] = {tmp, tmp + n, tmp + 2 * n, tmp + 3 * n, tmp + 4 * n};
    const int64_t shape[3] = {N, N, 1};
    int rc = stencil_matrix_create_fields(out, 2, shape, f, stream);
    cudaStreamSynchronize(s);
    cudaFree(tmp);
    return rc;
}

int stencil_matrix_destroy(sstep_matrix M) {
    if (!M) return SSTEP_ERR_ARG;
    if (M->fields) cudaFree(M->fields);
    if (M->fields_df) cudaFree(M->fields_df);
    if (M->ws) cudaFree(M->ws);
    if (M->hdr) cudaFreeHost(M->hdr);
    if (M->rbilu) cudaFree(M->rbilu);
    if (M->nilu) cudaFree(M->nilu);
    delete M;
    return SSTEP_OK;
}

int stencil_matrix_info(sstep_matrix M, int64_t* n, double* norm_inf) {
    if (!M) return SSTEP_ERR_ARG;
    if (n) *n = M->A.n;
    if (norm_inf) *norm_inf = M->norm_inf;
    return SSTEP_OK;
}

int stencil_matrix_apply(sstep_matrix M, const double* x, double* y, void* stream) {
    if (!M || !x || !y) return SSTEP_ERR_ARG;
    launch_stencil(M->A, x, 1.0, y, 0.0, nullptr, nullptr, nullptr, GATE_NONE, (cudaStream_t)stream);
    return check_launch();
}

int stencil_matrix_smooth(sstep_matrix M, const double* f, double* x, double* work, int sweeps, double omega,
                          void* stream) {
    if (!M || sweeps < 0 || !(omega > 0.0 && omega < 2.0)) return SSTEP_ERR_ARG;
    if (sweeps == 0) return SSTEP_OK;
    if (!f || !x || !work || work == x || work == f) return SSTEP_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    double* src = x;
    double* dst = work;
    for (int t = 0; t < sweeps; ++t) {
        launch_jacobi(M->A, f, src, dst, omega, st);
        double* tmp = src;
        src = dst;
        dst = tmp;
    }
    if (src != x && cudaMemcpyAsync(x, src, sizeof(double) * (size_t)M->A.n, cudaMemcpyDeviceToDevice, st) !=
                        cudaSuccess)
        return SSTEP_ERR_CUDA;
    return check_launch();
}

int stencil_matrix_smooth_batched(int nsys, const sstep_matrix* A, const double* const* f, double* const* x,
                                  double* const* work, int sweeps, double omega, void* stream) {
    if (nsys < 1 || nsys > 65535 || !A || !f || !x || !work || sweeps < 0 || !(omega > 0.0 && omega < 2.0))
        return SSTEP_ERR_ARG;
    std::vector<SmoothSys> h(nsys);
    int64_t nmax = 1;
    for (int i = 0; i < nsys; ++i) {
        if (!A[i] || !f[i] || !x[i] || !work[i] || work[i] == x[i] || work[i] == f[i]) return SSTEP_ERR_ARG;
        h[i].A = A[i]->A;
        h[i].f = f[i];
        h[i].x = x[i];
        h[i].work = work[i];
        nmax = std::max<int64_t>(nmax, A[i]->A.n);
    }
    if (sweeps == 0) return SSTEP_OK;
    cudaStream_t st = (cudaStream_t)stream;
    SmoothSys* d = nullptr;
    if (cudaMallocAsync((void**)&d, sizeof(SmoothSys) * nsys, st) != cudaSuccess) return SSTEP_ERR_OOM;
    int rc = SSTEP_OK;
    if (cudaMemcpyAsync(d, h.data(), sizeof(SmoothSys) * nsys, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        launch_jacobi_batched(d, nsys, nmax, sweeps, omega, st) != 0)
        rc = SSTEP_ERR_CUDA;
    // the host array must outlive the copy: wait for it before h goes out of scope
    if (cudaStreamSynchronize(st) != cudaSuccess) rc = SSTEP_ERR_CUDA;
    cudaFreeAsync(d, st);
    if (rc == SSTEP_OK) rc = check_launch();
    return rc;
}

int sstep_set_workspace_limit(int64_t bytes) {
    if (bytes < 0) return SSTEP_ERR_ARG;
    g_workspace_limit = bytes;
    return SSTEP_OK;
}

int sstep_newton_shifts(const double* G, int ldg, int K, int s, double* theta) {
    if (!G || !theta || K < 1 || ldg < K || s < 1 || s > SSTEP_MAX_S) return SSTEP_ERR_ARG;
    std::vector<double> ev;
    if (!hessenberg_real_parts(G, ldg, K, ev)) return SSTEP_ERR_BREAKDOWN;
    const std::vector<double> th = leja_order(ev, s);
    for (int i = 0; i < s; ++i) theta[i] = th[i];
    return SSTEP_OK;
}

namespace {
// the factors of the right preconditioner `kind`, built on first use and kept with A
int ensure_precond(sstep_matrix M, int kind, cudaStream_t st) {
    if (kind == SSTEP_PRECOND_RBILU0 && !M->rbilu) {
        if (cudaMalloc((void**)&M->rbilu, sizeof(double) * M->A.n) != cudaSuccess) {
            cudaGetLastError();
            M->rbilu = nullptr;
            return SSTEP_ERR_OOM;
        }
        launch_rbilu_setup(M->A, M->rbilu, st);
    }
    if (kind == SSTEP_PRECOND_ILU0 && !M->nilu) {
        if (cudaMalloc((void**)&M->nilu, sizeof(double) * (M->A.dim + 1) * M->A.n) != cudaSuccess) {
            cudaGetLastError();
            M->nilu = nullptr;
            return SSTEP_ERR_OOM;
        }
        launch_nilu_setup(M->A, M->nilu, st);
    }
    return SSTEP_OK;
}

// w = M^-1 v for the preconditioner `kind` (its factors exist), gated like the solver's kernels
void precond_apply(sstep_matrix M, int kind, const double* v, double* w, const SolverState* st, int gate,
                   cudaStream_t s) {
    if (kind == SSTEP_PRECOND_ILU0) launch_nilu_apply(M->A, M->nilu, v, w, st, gate, s);
    else launch_rbilu_apply(M->A, M->rbilu, v, w, st, gate, s);
}
}  // namespace

int stencil_matrix_rbilu0_apply(sstep_matrix M, const double* v, double* w, void* stream) {
    if (!M || !v || !w || v == w) return SSTEP_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = ensure_precond(M, SSTEP_PRECOND_RBILU0, st);
    if (rc) return rc;
    precond_apply(M, SSTEP_PRECOND_RBILU0, v, w, nullptr, GATE_NONE, st);
    return check_launch();
}

int stencil_matrix_ilu0_apply(sstep_matrix M, const double* v, double* w, void* stream) {
    if (!M || !v || !w || v == w) return SSTEP_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = ensure_precond(M, SSTEP_PRECOND_ILU0, st);
    if (rc) return rc;
    precond_apply(M, SSTEP_PRECOND_ILU0, v, w, nullptr, GATE_NONE, st);
    return check_launch();
}

int sstep_last_shifts(sstep_matrix M, double* theta, int cap) {
    if (!M || cap < 0 || (cap > 0 && !theta)) return SSTEP_ERR_ARG;
    const int n = (int)M->shifts.size();
    for (int i = 0; i < n && i < cap; ++i) theta[i] = M->shifts[i];
    return n;
}

int sstep_matrix_powers(sstep_matrix M, const double* v, double scale, double sigma, int s, double* Y, int64_t ldy,
                        void* stream) {
    if (!M || !v || !Y || s < 1 || s > SSTEP_MAX_S || ldy < M->A.n) return SSTEP_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    launch_stencil(M->A, v, sigma * scale, Y + ldy, scale, Y, nullptr, nullptr, GATE_NONE, st);
    for (int j = 2; j <= s; ++j)
        launch_stencil(M->A, Y + (j - 1) * ldy, sigma, Y + j * ldy, 0.0, nullptr, nullptr, nullptr, GATE_NONE, st);
    return check_launch();
}

// work: the arrival counter and error flag (256 B), the partials, then the column bounds of
// the tensor-core pass (ka + kb <= 73 words: 512 B)
constexpr size_t kGramBndBytes = 2 * kAlign;
int sstep_gram_workspace_size(int64_t n, int ka, int kb, size_t* bytes) {
    if (!bytes || n < 0 || ka < 1 || ka > SSTEP_MAX_COLS || kb < 1 || kb > SSTEP_MAX_S + 1) return SSTEP_ERR_ARG;
    *bytes = kAlign + sizeof(double) * (size_t)max_partials_doubles() + kGramBndBytes;
    return SSTEP_OK;
}

int sstep_gram_tc(int64_t n, const double* V, int64_t ldv, int ka, const double* Y, int64_t ldy, int kb, double* C,
                  int ldc, void* work, size_t work_bytes, void* stream) {
    size_t need = 0;
    if (sstep_gram_workspace_size(n, ka, kb, &need)) return SSTEP_ERR_ARG;
    if (!V || !Y || !C || !work || work_bytes < need || ldv < n || ldy < n || ldc < ka) return SSTEP_ERR_ARG;
    if (((uintptr_t)work) % kAlign) return SSTEP_ERR_ARG;
    if (n > ((int64_t)1 << 27) || ((uintptr_t)V & 7) || ((uintptr_t)Y & 7)) return SSTEP_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (n == 0)
        return cudaMemset2DAsync(C, sizeof(double) * ldc, 0, sizeof(double) * ka, kb, st) == cudaSuccess ? SSTEP_OK
                                                                                                       : SSTEP_ERR_CUDA;
    Scratch sc{(double*)((char*)work + kAlign), (unsigned*)work};
    sc.acc = (unsigned long long*)sc.partials;   // the exact accumulators, in the partials area
    unsigned* bnd = (unsigned*)((char*)work + kAlign + sizeof(double) * (size_t)max_partials_doubles());
    CUDA_TRY(cudaMemsetAsync(work, 0, kAlign, st));
    CUDA_TRY(cudaMemsetAsync(sc.acc, 0, sizeof(unsigned long long) * kOzAccWords, st));
    CUDA_TRY(cudaMemsetAsync(bnd, 0, kGramBndBytes, st));
    launch_colmax(n, V, ldv, ka, bnd, st);
    launch_colmax(n, Y, ldy, kb, bnd + ka, st);
    Epi e;
    e.mode = EPI_NONE;
    e.out = C;
    e.ldo = ldc;
    if (!launch_gram_oz(n, V, ldv, ka, bnd, Y, ldy, kb, bnd + ka, sc, e, GATE_NONE, st)) return SSTEP_ERR_ARG;
    return check_launch();
}

// mbarrier poll limit of the tensor-core Gram pass (tests of its timeout path); < 0 restores the default
int sstep_set_tc_wait_limit(long limit) {
    static const long dflt = g_oz_spin;
    g_oz_spin = limit >= 0 ? limit : dflt;
    return SSTEP_OK;
}

int sstep_gram(int64_t n, const double* V, int64_t ldv, int ka, const double* Y, int64_t ldy, int kb, double* C,
               int ldc, void* work, size_t work_bytes, void* stream) {
    size_t need = 0;
    if (sstep_gram_workspace_size(n, ka, kb, &need)) return SSTEP_ERR_ARG;
    if (!V || !Y || !C || !work || work_bytes < need || ldv < n || ldy < n || ldc < ka) return SSTEP_ERR_ARG;
    if (((uintptr_t)work) % kAlign) return SSTEP_ERR_ARG;
    if (n == 0)   // C = 0: the ka x kb entries only (the rows below ka of each column are the caller's)
        return cudaMemset2DAsync(C, sizeof(double) * ldc, 0, sizeof(double) * ka, kb, (cudaStream_t)stream) ==
                       cudaSuccess
                   ? SSTEP_OK
                   : SSTEP_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    Scratch sc{(double*)((char*)work + kAlign), (unsigned*)work};
    CUDA_TRY(cudaMemsetAsync(work, 0, sizeof(unsigned), st));
    Epi e;
    e.mode = EPI_NONE;
    e.out = C;
    e.ldo = ldc;
    launch_gram(n, V, ldv, ka, Y, ldy, kb, 0, sc, e, GATE_NONE, st);
    return check_launch();
}

int sstep_block_update(int64_t n, const double* V, int64_t ldv, int ka, double* Y, int64_t ldy, int kb,
                       const double* T, int ldt, double* Gout, void* work, size_t work_bytes, void* stream) {
    size_t need = 0;
    if (sstep_gram_workspace_size(n, 1, kb, &need)) return SSTEP_ERR_ARG;
    if (ka < 0 || ka > SSTEP_MAX_COLS || !Y || !Gout || !work || work_bytes < need || ldy < n) return SSTEP_ERR_ARG;
    if (ka > 0 && (!V || !T || ldv < n || ldt < ka)) return SSTEP_ERR_ARG;
    if (((uintptr_t)work) % kAlign) return SSTEP_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (n == 0) return cudaMemsetAsync(Gout, 0, sizeof(double) * kb * kb, st) == cudaSuccess ? SSTEP_OK : SSTEP_ERR_CUDA;
    Scratch sc{(double*)((char*)work + kAlign), (unsigned*)work};
    CUDA_TRY(cudaMemsetAsync(work, 0, sizeof(unsigned), st));
    Epi e;
    e.mode = EPI_NONE;
    e.out = Gout;
    e.ldo = kb;
    launch_update(n, V, ldv, ka, Y, ldy, Y, ldy, kb, 0, T, ldt, -1.0, true, sc, e, GATE_NONE, st);
    return check_launch();
}

int sstep_block_update_tc(int64_t n, const double* V, int64_t ldv, int ka, double* Y, int64_t ldy, int kb,
                          const double* T, int ldt, double* Gout, void* work, size_t work_bytes, void* stream) {
    size_t need = 0;
    if (sstep_gram_workspace_size(n, 1, kb, &need)) return SSTEP_ERR_ARG;
    if (ka < 0 || ka > 32 || !Y || !Gout || !work || work_bytes < need || ldy < n) return SSTEP_ERR_ARG;
    if (ka > 0 && (!V || !T || ldv < n || ldt < ka)) return SSTEP_ERR_ARG;
    if (((uintptr_t)work) % kAlign || n > ((int64_t)1 << 27) || ((uintptr_t)Y & 7)) return SSTEP_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (n == 0) return cudaMemsetAsync(Gout, 0, sizeof(double) * kb * kb, st) == cudaSuccess ? SSTEP_OK : SSTEP_ERR_CUDA;
    Scratch sc{(double*)((char*)work + kAlign), (unsigned*)work};
    sc.acc = (unsigned long long*)sc.partials;
    unsigned* bnd = (unsigned*)((char*)work + kAlign + sizeof(double) * (size_t)max_partials_doubles());
    unsigned* vb = bnd;          // ka bounds of V
    unsigned* yb = bnd + 32;     // kb bounds of the updated Y
    CUDA_TRY(cudaMemsetAsync(work, 0, kAlign, st));
    CUDA_TRY(cudaMemsetAsync(sc.acc, 0, sizeof(unsigned long long) * kOzAccWords, st));
    CUDA_TRY(cudaMemsetAsync(bnd, 0, kGramBndBytes, st));
    if (ka > 0) {
        launch_colmax(n, V, ldv, ka, vb, st);
        if (!launch_update_oz(n, V, ldv, ka, vb, Y, ldy, 0, kb, T, ldt, yb, nullptr, 0, nullptr, nullptr, nullptr,
                              GATE_NONE, st, (unsigned*)work + 1))
            return SSTEP_ERR_ARG;
    } else {
        launch_colmax(n, Y, ldy, kb, yb, st);
    }
    Epi e;
    e.mode = EPI_NONE;
    e.out = Gout;
    e.ldo = kb;
    if (!launch_gram_oz(n, Y, ldy, kb, yb, Y, ldy, kb, yb, sc, e, GATE_NONE, st)) return SSTEP_ERR_ARG;
    return check_launch();
}

// ------------------------------------------------------------------ s-step GMRES (Alg. 4.1 / 4.2)
int sstep_gmres_solve(sstep_matrix M, const double* f, double* x, const sstep_params* p, sstep_result* res,
                      void* stream) {
    int rc = common_checks(M, f, x, p, res);
    if (rc) return rc;
    const int s = p->s, m = p->m;
    if (s < 1 || s > SSTEP_MAX_S || m < s || m > SSTEP_MAX_M || m % s != 0 || p->max_cycles < 0) return SSTEP_ERR_ARG;
    if (p->basis != SSTEP_BASIS_MONOMIAL && p->basis != SSTEP_BASIS_NEWTON) return SSTEP_ERR_ARG;
    if (p->precond != SSTEP_PRECOND_NONE &&
        ((p->precond != SSTEP_PRECOND_RBILU0 && p->precond != SSTEP_PRECOND_ILU0) || p->precision != SSTEP_PREC_FP64))
        return SSTEP_ERR_ARG;
    const int pk = p->precond;
    const bool pre = pk != SSTEP_PRECOND_NONE;
    cudaStream_t stream_ = (cudaStream_t)stream;
    if (p->precision == SSTEP_PREC_DF64) return sstep_gmres_mp<PREC_DF64>(M, f, x, p, res, stream_);
    if (p->precision == SSTEP_PREC_FP32) return sstep_gmres_mp<PREC_FP32>(M, f, x, p, res, stream_);
    if (p->precision != SSTEP_PREC_FP64) return SSTEP_ERR_ARG;
    const int64_t n = M->A.n, ld = col_ld(n);
    // tensor-core Gram pass and block update (off with a preconditioner)
    const bool tcg = !pre && tc_gram_enabled();
    // columns: U (m+1), the raw start vector and, preconditioned, M^-1 of a power; with the
    // tensor-core passes also m columns of the basis in fixed-point words
    const int ncols0 = m + 2 + (pre ? 1 : 0);
    Layout l = plan(n, ncols0 + (tcg ? m : 0), m, p->history ? p->history_cap : 0);
    if ((rc = ensure_workspace(M, l.total))) return rc;
    if (pre && (rc = ensure_precond(M, pk, stream_))) return rc;   // the factors, once per matrix
    SolverState h = init_state(l, M->ws, p, s, m, 0);
    // sigma: 1 / ||A||_inf; preconditioned, A M^-1 has its spectrum near 1 and sigma = 1
    h.sigma = p->sigma > 0.0 ? p->sigma : (pre ? 1.0 : 1.0 / M->norm_inf);
    SolverState* st = (SolverState*)(M->ws + l.state);
    double* U = (double*)(M->ws + l.cols);
    double* uraw = U + (int64_t)(m + 1) * ld;
    double* ptmp = U + (int64_t)(m + 2) * ld;   // preconditioned: M^-1 y^j, then V y
    Scratch sc{(double*)(M->ws + l.partials), (unsigned*)(M->ws + l.counter)};
    CUDA_TRY(cudaMemcpyAsync(st, &h, sizeof(h), cudaMemcpyHostToDevice, stream_));
    CUDA_TRY(cudaMemsetAsync(M->ws + l.counter, 0, kAlign, stream_));
    CUDA_TRY(cudaMemsetAsync(M->ws + l.G, 0, sizeof(double) * (m + 1) * m, stream_));
    CUDA_TRY(cudaMemsetAsync(M->ws + l.theta, 0, sizeof(double) * kMaxS, stream_));
    Epi e;
    e.st = st;
    e.mode = EPI_NF;
    TRACED(K_RESIDUAL, stream_, launch_residual(M->A, f, nullptr, nullptr, sc, e, GATE_NONE, stream_));
    if (p->x0_guard && (rc = apply_x0_guard(M, l, st, f, x, stream_))) return rc;
    const double sigma = h.sigma;
    const int nb = m / s;
    // tensor-core Gram pass: the producers of every basis and power column record its bound
    // (bnd[c] for basis column c, pbnd(k)[j] for power j of block k), zeroed per cycle. The
    // pass that forms block k's Gram matrix also keeps the block's columns as fixed-point
    // words (Wp, relative to the same bounds), which the later inner products and updates
    // of the cycle read instead of converting the FP64 columns again.
    uint64_t* Wp = (tcg && tc_words_enabled()) ? (uint64_t*)(U + (int64_t)ncols0 * ld) : nullptr;
    unsigned* bnd = (unsigned*)(M->ws + l.bnd);
    auto pbnd = [&](int k) { return tcg ? bnd + (m + 1) + k * (s + 1) : nullptr; };
    auto ubnd = [&](int k) { return tcg ? bnd + (m + 1) + (nb + k) * (s + 1) : nullptr; };
    if (tcg) {   // the exact accumulators start at zero; every launch leaves them at zero
        sc.acc = (unsigned long long*)(M->ws + l.ozacc);
        CUDA_TRY(cudaMemsetAsync(sc.acc, 0, sizeof(unsigned long long) * kOzAccWords, stream_));
    }
    std::vector<double> theta(s, 0.0);   // Newton shifts (zero: monomial powers)
    bool shifted = false;
    M->shifts.clear();
    for (;;) {
        if (tcg) CUDA_TRY(cudaMemsetAsync(bnd, 0, sizeof(unsigned) * kBndSlots, stream_));
        int wcols = 0;   // basis columns of this cycle whose words are in Wp
        e = Epi();
        e.st = st;
        e.mode = EPI_RESTART;
        TRACED(K_RESIDUAL, stream_, launch_residual(M->A, f, x, uraw, sc, e, GATE_ACTIVE, stream_));
        for (int k = 0; k < nb; ++k) {
            const int o = k * s;
            unsigned* pb = pbnd(k);
            unsigned* ub = ubnd(k);
            // bounds: the copy v_k^1 -> bnd[o] and pb[0]; power j -> pb[j]; in the first block
            // the powers 1..s-1 are final basis columns as they stand -> bnd[o + j] too
            auto fin = [&](int j) { return (tcg && k == 0 && j < s) ? bnd + o + j : nullptr; };
            // Alg. 4.1 step 3: v_k^1 = u / ||u|| and its s scaled powers (in one fused launch with
            // TMA-staged tiles when SSTEP_FUSED_POWERS=1: the same columns, bit for bit)
            bool fusedp = false;
            if (!pre && fused_powers_enabled()) {
                unsigned* b1[kMaxS + 1] = {};
                unsigned* b2[kMaxS + 1] = {};
                if (tcg) {
                    b1[0] = bnd + o;   // the copy v_k^1: basis column o and power 0 of the block
                    b2[0] = pb;
                    for (int j = 1; j <= s; ++j) {
                        b1[j] = pb + j;
                        b2[j] = fin(j);
                    }
                }
                TRACED(K_STENCIL, stream_,
                       fusedp = launch_powers_fused(M->A, uraw, sigma, &st->vscale, U + o * ld, ld, s, theta.data(), b1,
                                                    b2, st, GATE_BUILDING, stream_));
            }
            if (!pre && !fusedp) {
                TRACED(K_STENCIL, stream_, launch_stencil(M->A, uraw, sigma, U + (o + 1) * ld, 1.0, U + o * ld,
                                                          &st->vscale, st, GATE_BUILDING, stream_, theta[0], nullptr,
                                                          tcg ? pb + 1 : nullptr, tcg ? bnd + o : nullptr, fin(1),
                                                          tcg ? pb : nullptr));
                for (int j = 2; j <= s; ++j)
                    TRACED(K_STENCIL, stream_, launch_stencil(M->A, U + (o + j - 1) * ld, sigma, U + (o + j) * ld, 0.0,
                                                              nullptr, nullptr, st, GATE_BUILDING, stream_, theta[j - 1],
                                                              nullptr, tcg ? pb + j : nullptr, nullptr, fin(j)));
            } else if (pre) {   // right preconditioning: y^{j+1} = sigma (A M^-1 y^j - theta_j y^j)
                launch_scale_copy(uraw, U + o * ld, n, &st->vscale, st, GATE_BUILDING, stream_);
                for (int j = 1; j <= s; ++j) {
                    TRACED(K_PRECOND, stream_, precond_apply(M, pk, U + (o + j - 1) * ld, ptmp, st, GATE_BUILDING,
                                                             stream_));
                    TRACED(K_STENCIL, stream_, launch_stencil(M->A, ptmp, sigma, U + (o + j) * ld, 0.0, nullptr,
                                                              nullptr, st, GATE_BUILDING, stream_, theta[j - 1],
                                                              U + (o + j - 1) * ld));
                }
            }
            if (k > 0) {   // steps 4-5 and Scalar2: inner products with the earlier blocks
                e = Epi();
                e.st = st;
                e.mode = EPI_GM_T;
                e.o = o;
                const bool vw = wcols >= o;   // every earlier column's words are kept
                TRACED(K_GRAM, stream_,
                       if (!tcg || !launch_gram_oz(n, vw ? (const double*)Wp : U, ld, o, bnd, U + (o + 1) * ld, ld, s,
                                                   pb + 1, sc, e, GATE_BUILDING, stream_, vw ? 1 : 0))
                           launch_gram(n, U, ld, o, U + (o + 1) * ld, ld, s, 0, sc, e, GATE_BUILDING, stream_));
            }
            // step 7 and Scalar1: project, then Gram of the projected block
            e = Epi();
            e.st = st;
            e.mode = EPI_GM_W;
            e.o = o;
            bool done = false;
            if (tcg) {   // tensor cores: projection (k > 0), then the Gram pass of the s + 1 columns
                bool proj = k == 0;
                if (k > 0) {
                    const bool vw = wcols >= o;
                    TRACED(K_UPDATE, stream_,
                           proj = launch_update_oz(n, vw ? (const double*)Wp : U, ld, o, bnd, U + o * ld, ld, 1, s, h.T,
                                                   m, ub + 1, bnd + o + 1, s - 1, pb, ub, st, GATE_BUILDING, stream_,
                                                   nullptr, vw ? 1 : 0));
                }
                unsigned* yb = k > 0 ? ub : pb;
                if (proj)
                    TRACED(K_UPDATE, stream_,
                           done = launch_gram_oz(n, U + o * ld, ld, s + 1, yb, U + o * ld, ld, s + 1, yb, sc, e,
                                                 GATE_BUILDING, stream_, 0, Wp ? Wp + (int64_t)o * ld : nullptr, ld,
                                                 Wp ? s : 0));
                if (done && Wp && wcols == o) wcols = o + s;   // this block's words are kept
                if (proj && !done)   // projected on the tensor cores; Gram in FP64
                    TRACED(K_UPDATE, stream_, launch_update(n, U, ld, 0, U + o * ld, ld, U + o * ld, ld, s + 1, 1, h.T, m,
                                                            -1.0, true, sc, e, GATE_BUILDING, stream_));
                done = done || proj;
            }
            if (!done)
                TRACED(K_UPDATE, stream_, launch_update(n, U, ld, o, U + o * ld, ld, U + o * ld, ld, s + 1, 1, h.T, m, -1.0,
                                                        true, sc, e, GATE_BUILDING, stream_, tcg ? bnd + o + 1 : nullptr,
                                                        s));
            // step 2: the next start vector u = z - V_k S and its norm; G, Givens
            e = Epi();
            e.st = st;
            e.mode = EPI_GM_NU;
            e.o = o;
            e.lastblock = (k == nb - 1);
            TRACED(K_NEXT, stream_, launch_update(n, U + o * ld, ld, s, U + (o + s) * ld, ld, uraw, ld, 1, 0, h.S, s, -1.0, true, sc, e,
                          GATE_BUILDING, stream_));
        }
        // Alg. 4.2 step 3: x = x0 + V y
        TRACED(K_LSQ, stream_, launch_lsq_solve(st, GATE_ACTIVE, stream_));
        e = Epi();
        e.st = st;
        if (!pre) {
            TRACED(K_AXPY, stream_, launch_update(n, U, ld, -1, x, n, x, n, 1, 0, nullptr, 0, 1.0, false, sc, e,
                                                  GATE_ACTIVE, stream_));
        } else {   // x += M^-1 (V y)
            CUDA_TRY(cudaMemsetAsync(ptmp, 0, sizeof(double) * n, stream_));
            TRACED(K_AXPY, stream_, launch_update(n, U, ld, -1, ptmp, ld, ptmp, ld, 1, 0, nullptr, 0, 1.0, false, sc,
                                                  e, GATE_ACTIVE, stream_));
            TRACED(K_PRECOND, stream_, precond_apply(M, pk, ptmp, uraw, st, GATE_ACTIVE, stream_));
            launch_add(x, uraw, n, st, GATE_ACTIVE, stream_);
        }
        CUDA_TRY(cudaGetLastError());
        if ((rc = read_header(M, st, stream_))) return rc;
        if (!M->hdr->active) break;
        if (p->basis == SSTEP_BASIS_NEWTON && !shifted) {   // shifts from the first cycle's Ritz values
            std::vector<double> th = newton_shifts_from_device(h.G, m, M->hdr->K, s, h.theta, stream_);
            if (!th.empty()) {
                theta = th;
                M->shifts = th;
            }
            shifted = true;
        }
    }
    return finish(M, l, st, f, x, p, res, stream_);
}

// ------------------------------------------------------------------ GMRES(m), Alg. 2.2
int gmres_solve(sstep_matrix M, const double* f, double* x, const sstep_params* p, sstep_result* res, void* stream) {
    int rc = common_checks(M, f, x, p, res);
    if (rc) return rc;
    const int m = p->m;
    if (m < 1 || m > SSTEP_MAX_M || p->max_cycles < 0 || p->precond != SSTEP_PRECOND_NONE) return SSTEP_ERR_ARG;
    cudaStream_t stream_ = (cudaStream_t)stream;
    if (p->precision == SSTEP_PREC_DF64) return gmres_mp<PREC_DF64>(M, f, x, p, res, stream_);
    if (p->precision == SSTEP_PREC_FP32) return gmres_mp<PREC_FP32>(M, f, x, p, res, stream_);
    if (p->precision != SSTEP_PREC_FP64) return SSTEP_ERR_ARG;
    const int64_t n = M->A.n, ld = col_ld(n);
    Layout l = plan(n, m + 3, m, p->history ? p->history_cap : 0);
    if ((rc = ensure_workspace(M, l.total))) return rc;
    SolverState h = init_state(l, M->ws, p, 1, m, 0);
    h.sigma = 1.0;
    SolverState* st = (SolverState*)(M->ws + l.state);
    double* U = (double*)(M->ws + l.cols);
    double* wraw = U + (int64_t)(m + 1) * ld;
    double* ybuf = wraw + ld;
    Scratch sc{(double*)(M->ws + l.partials), (unsigned*)(M->ws + l.counter)};
    CUDA_TRY(cudaMemcpyAsync(st, &h, sizeof(h), cudaMemcpyHostToDevice, stream_));
    CUDA_TRY(cudaMemsetAsync(M->ws + l.counter, 0, kAlign, stream_));
    CUDA_TRY(cudaMemsetAsync(M->ws + l.G, 0, sizeof(double) * (m + 1) * m, stream_));
    Epi e;
    e.st = st;
    e.mode = EPI_NF;
    TRACED(K_RESIDUAL, stream_, launch_residual(M->A, f, nullptr, nullptr, sc, e, GATE_NONE, stream_));
    if (p->x0_guard && (rc = apply_x0_guard(M, l, st, f, x, stream_))) return rc;
    for (;;) {
        e = Epi();
        e.st = st;
        e.mode = EPI_RESTART;
        TRACED(K_RESIDUAL, stream_, launch_residual(M->A, f, x, wraw, sc, e, GATE_ACTIVE, stream_));
        for (int j = 0; j < m; ++j) {
            // step 4 of the previous step (q_j = q^_j / h) fused with A q_j
            TRACED(K_STENCIL, stream_, launch_stencil(M->A, wraw, 1.0, ybuf, 1.0, U + j * ld, &st->vscale, st, GATE_BUILDING, stream_));
            e = Epi();
            e.st = st;
            e.mode = EPI_ST_H;
            e.o = j;
            TRACED(K_GRAM, stream_, launch_gram(n, U, ld, j + 1, ybuf, ld, 1, 0, sc, e, GATE_BUILDING, stream_));   // step 1
            e = Epi();
            e.st = st;
            e.mode = EPI_ST_NORM;
            e.o = j;
            e.lastblock = (j == m - 1);
            TRACED(K_UPDATE, stream_, launch_update(n, U, ld, j + 1, ybuf, ld, wraw, ld, 1, 0, h.G + (int64_t)j * (m + 1), m + 1, -1.0, true,
                          sc, e, GATE_BUILDING, stream_));   // steps 2-3
        }
        TRACED(K_LSQ, stream_, launch_lsq_solve(st, GATE_ACTIVE, stream_));
        e = Epi();
        e.st = st;
        TRACED(K_AXPY, stream_, launch_update(n, U, ld, -1, x, n, x, n, 1, 0, nullptr, 0, 1.0, false, sc, e, GATE_ACTIVE, stream_));
        CUDA_TRY(cudaGetLastError());
        if ((rc = read_header(M, st, stream_))) return rc;
        if (!M->hdr->active) break;
    }
    return finish(M, l, st, f, x, p, res, stream_);
}

// ------------------------------------------------------------------ s-step Orthomin(k), Alg. 3.1
int sstep_omin_solve(sstep_matrix M, const double* f, double* x, const sstep_params* p, sstep_result* res,
                     void* stream) {
    int rc = common_checks(M, f, x, p, res);
    if (rc) return rc;
    const int s = p->s, k = p->k;
    if (s < 1 || s > SSTEP_MAX_S || k < 0 || (int64_t)k * s > SSTEP_MAX_COLS || p->max_iters < 0) return SSTEP_ERR_ARG;
    if (p->precision != SSTEP_PREC_FP64 || (p->precond != SSTEP_PRECOND_NONE && p->precond != SSTEP_PRECOND_RBILU0 &&
                                             p->precond != SSTEP_PRECOND_ILU0))
        return SSTEP_ERR_ARG;
    if (p->basis != SSTEP_BASIS_MONOMIAL && p->basis != SSTEP_BASIS_ORTHO) return SSTEP_ERR_ARG;
    const int pk = p->precond;
    const bool pre = pk != SSTEP_PRECOND_NONE;
    const int ortho = p->basis == SSTEP_BASIS_ORTHO;
    if (ortho && (int64_t)(k + 1) * s > SSTEP_MAX_COLS) return SSTEP_ERR_ARG;
    cudaStream_t stream_ = (cudaStream_t)stream;
    const int64_t n = M->A.n, ld = col_ld(n);
    const int keep = std::max(k, 1);
    const int nslots = keep + 1;
    // columns: P and AP panels (nslots*s each), AR (s), r (1); preconditioned also the
    // accumulated correction du (the method runs on A M^-1: x = x0 + M^-1 du) and a scratch
    Layout l = plan(n, 2 * nslots * s + s + 1 + (pre ? 2 : 0), 1, p->history ? p->history_cap : 0);
    if ((rc = ensure_workspace(M, l.total))) return rc;
    if (pre && (rc = ensure_precond(M, pk, stream_))) return rc;
    SolverState h = init_state(l, M->ws, p, s, 1, k);
    h.sigma = p->sigma > 0.0 ? p->sigma : (pre ? 1.0 : 1.0 / M->norm_inf);
    SolverState* st = (SolverState*)(M->ws + l.state);
    double* Ppanel = (double*)(M->ws + l.cols);
    double* APpanel = Ppanel + (int64_t)nslots * s * ld;
    double* AR = APpanel + (int64_t)nslots * s * ld;
    double* r = AR + (int64_t)s * ld;
    double* du = r + ld;          // preconditioned: sum of the steps P a since the last explicit residual
    double* ptmp = du + ld;       // preconditioned: M^-1 of a power, M^-1 du
    Scratch sc{(double*)(M->ws + l.partials), (unsigned*)(M->ws + l.counter)};
    CUDA_TRY(cudaMemcpyAsync(st, &h, sizeof(h), cudaMemcpyHostToDevice, stream_));
    CUDA_TRY(cudaMemsetAsync(M->ws + l.counter, 0, kAlign, stream_));
    if (pre) CUDA_TRY(cudaMemsetAsync(du, 0, sizeof(double) * n, stream_));
    Epi e;
    e.st = st;
    e.mode = EPI_NF;
    TRACED(K_RESIDUAL, stream_, launch_residual(M->A, f, nullptr, nullptr, sc, e, GATE_NONE, stream_));
    if (p->x0_guard && (rc = apply_x0_guard(M, l, st, f, x, stream_))) return rc;
    const double sigma = h.sigma;
    auto powers = [&]() {   // A R_{i+1}: A r, then A (sigma A R_j); preconditioned: A M^-1 ...
        if (!pre) {
            TRACED(K_STENCIL, stream_, launch_stencil(M->A, r, 1.0, AR, 0.0, nullptr, nullptr, st, GATE_BUILDING, stream_));
            for (int j = 1; j < s; ++j)
                TRACED(K_STENCIL, stream_, launch_stencil(M->A, AR + (j - 1) * ld, sigma, AR + j * ld, 0.0, nullptr,
                                                          nullptr, st, GATE_BUILDING, stream_));
            return;
        }
        for (int j = 0; j < s; ++j) {
            TRACED(K_PRECOND, stream_, precond_apply(M, pk, j == 0 ? r : AR + (j - 1) * ld, ptmp, st, GATE_BUILDING,
                                                     stream_));
            TRACED(K_STENCIL, stream_, launch_stencil(M->A, ptmp, j == 0 ? 1.0 : sigma, AR + j * ld, 0.0, nullptr,
                                                      nullptr, st, GATE_BUILDING, stream_));
        }
    };
    // x += M^-1 du, du = 0 (at a restart the solve is active, so the gated kernels run)
    auto fold = [&](int gate) -> int {
        if (!pre) return SSTEP_OK;
        TRACED(K_PRECOND, stream_, precond_apply(M, pk, du, ptmp, st, gate, stream_));
        launch_add(x, ptmp, n, st, gate, stream_);
        return cudaMemsetAsync(du, 0, sizeof(double) * n, stream_) == cudaSuccess ? SSTEP_OK : SSTEP_ERR_CUDA;
    };
    std::vector<int> ring;
    bool restart = true;
    const int batch = 8;
    for (;;) {
        if (restart) {
            if ((rc = fold(GATE_ACTIVE))) return rc;
            e = Epi();
            e.st = st;
            e.mode = EPI_OM_RESTART;
            TRACED(K_RESIDUAL, stream_, launch_residual(M->A, f, x, r, sc, e, GATE_ACTIVE, stream_));
            powers();   // R_0, A R_0; P_0 = R_0
            e = Epi();
            e.st = st;
            e.nwin = 0;
            if (ortho) {   // A R^T A R: the factor that makes P_0 A^T A-orthonormal
                e.mode = EPI_OM_B;
                e.ortho = 1;
                e.win[0] = nslots;   // A R sits right after the A P slots
                TRACED(K_GRAM, stream_, launch_gram(n, APpanel, ld, s, AR, ld, s, s, sc, e, GATE_BUILDING, stream_));
            }
            e.mode = EPI_OM_W;
            e.slot = 0;
            TRACED(K_OMIN_PUPDATE, stream_, launch_omin_pupdate(n, r, AR, Ppanel, APpanel, ld, s, sigma, sc, e, GATE_BUILDING, stream_));
            ring.assign(1, 0);
            restart = false;
        }
        for (int b = 0; b < batch; ++b) {
            const int cur = ring.back();
            e = Epi();
            e.st = st;
            e.mode = EPI_OM_R;
            TRACED(K_OMIN_XR, stream_, launch_omin_xr(n, Ppanel + (int64_t)cur * s * ld, APpanel + (int64_t)cur * s * ld,
                                                      ld, s, pre ? du : x, r, sc, e, GATE_BUILDING, stream_));   // steps 3-4
            powers();                                 // step 5
            const int nwin = std::min<int>(k, (int)ring.size());
            Epi w;
            w.st = st;
            w.nwin = nwin;
            w.ortho = ortho;
            for (int i = 0; i < nwin; ++i) w.win[i] = ring[ring.size() - nwin + i];
            if (ortho) w.win[nwin] = nslots;   // the A R block, right after the A P slots ((k+1) s <= 64)
            if (nwin + ortho > 0) {   // steps 6-7
                w.mode = EPI_OM_B;
                TRACED(K_GRAM, stream_, launch_gram(n, APpanel, ld, (nwin + ortho) * s, AR, ld, s, s, sc, w,
                                                    GATE_BUILDING, stream_));
            }
            int nslot = 0;
            while (std::find(ring.begin(), ring.end(), nslot) != ring.end()) ++nslot;
            w.mode = EPI_OM_W;   // steps 8-9 and the next step's 1-2
            w.slot = nslot;
            TRACED(K_OMIN_PUPDATE, stream_, launch_omin_pupdate(n, r, AR, Ppanel, APpanel, ld, s, sigma, sc, w, GATE_BUILDING, stream_));
            ring.push_back(nslot);
            if ((int)ring.size() > keep) ring.erase(ring.begin());
        }
        CUDA_TRY(cudaGetLastError());
        if ((rc = read_header(M, st, stream_))) return rc;
        if (!M->hdr->active) break;
        if (M->hdr->confirm) restart = true;
    }
    if ((rc = fold(GATE_NONE))) return rc;   // steps taken since the last explicit residual
    return finish(M, l, st, f, x, p, res, stream_);
}


int sstep_batch_create(sstep_batch* out, int nsys, const sstep_matrix* A, const sstep_params* p) {
    if (!out || nsys < 1 || !A || !p) return SSTEP_ERR_ARG;
    *out = nullptr;
    const int s = p->s, m = p->m;
    if (!(s == 1 || s == 2 || s == 4 || s == 8) || m < s || m > kBatchMaxM || m % s || p->max_cycles < 0 ||
        !(p->tol > 0.0) || p->sigma < 0.0 || (p->precision != SSTEP_PREC_FP64 && p->precision != SSTEP_PREC_FP32) ||
        p->basis != SSTEP_BASIS_MONOMIAL ||
        p->precond != SSTEP_PRECOND_NONE)
        return SSTEP_ERR_ARG;
    for (int i = 0; i < nsys; ++i)
        if (!A[i]) return SSTEP_ERR_ARG;
    sstep_batch B = new (std::nothrow) sstep_batch_s;
    if (!B) return SSTEP_ERR_OOM;
    B->nsys = nsys;
    B->s = s;
    B->m = m;
    B->p = *p;
    B->mats.assign(A, A + nsys);
    // workspace: per system a state block and an (m+2)-column panel
    const size_t sb = batch_state_bytes(m);
    size_t total = 0;
    B->state_off.resize(nsys);
    std::vector<size_t> col_off(nsys);
    for (int i = 0; i < nsys; ++i) {
        B->state_off[i] = total;
        total += sb * kBatchCopies;
    }
    for (int i = 0; i < nsys; ++i) {
        col_off[i] = total;
        const size_t elem = p->precision == SSTEP_PREC_FP32 ? sizeof(float) : sizeof(double);
        total += align_up(elem * (size_t)col_ld(A[i]->A.n) * (m + 2));
    }
    int rc = SSTEP_OK;
    if (cudaMalloc((void**)&B->ws, total) != cudaSuccess || cudaMalloc((void**)&B->d_sys, sizeof(BatchSys) * nsys) !=
            cudaSuccess || cudaMalloc((void**)&B->d_order, sizeof(int) * nsys) != cudaSuccess ||
        cudaMalloc((void**)&B->d_queue, sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc((void**)&B->d_init, sizeof(SolverState) * nsys * kBatchCopies) != cudaSuccess ||
        cudaMallocHost((void**)&B->h_states, sizeof(SolverState) * nsys) != cudaSuccess) {
        cudaGetLastError();
        rc = SSTEP_ERR_OOM;
    }
    if (rc) {
        sstep_batch_destroy(B);
        return rc;
    }
    B->ws_bytes = total;
    B->h_sys.resize(nsys);
    B->h_init.resize((size_t)nsys * kBatchCopies);
    for (int i = 0; i < nsys; ++i) {
        const double sigma = p->sigma > 0.0 ? p->sigma : 1.0 / A[i]->norm_inf;
        for (int g = 0; g < kBatchCopies; ++g)
            B->h_init[(size_t)i * kBatchCopies + g] = batch_state(B->ws + B->state_off[i] + g * sb, m, s, p, sigma);
        BatchSys& b = B->h_sys[i];
        b.A = A[i]->A;
        b.U = (double*)(B->ws + col_off[i]);
        b.st = (SolverState*)(B->ws + B->state_off[i]);
        b.st_stride = (int64_t)sb;
        b.ld = col_ld(A[i]->A.n);
        b.f = nullptr;
        b.x = nullptr;
    }
    B->order_largest.resize(nsys);
    for (int i = 0; i < nsys; ++i) B->order_largest[i] = i;
    std::stable_sort(B->order_largest.begin(), B->order_largest.end(),
                     [&](int a, int b) { return A[a]->A.n > A[b]->A.n; });
    if (cudaMemcpy(B->d_order, B->order_largest.data(), sizeof(int) * nsys, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(B->d_init, B->h_init.data(), sizeof(SolverState) * B->h_init.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemset(B->ws, 0, total) != cudaSuccess) {
        sstep_batch_destroy(B);
        return SSTEP_ERR_CUDA;
    }
    *out = B;
    return SSTEP_OK;
}

int sstep_batch_solve(sstep_batch B, const double* const* f, double* const* x, sstep_result* res, int mode,
                      void* stream) {
    if (!B || !f || !x || !res) return SSTEP_ERR_ARG;
    for (int i = 0; i < B->nsys; ++i)
        if (!f[i] || !x[i]) return SSTEP_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (mode == SSTEP_BATCH_PER_SYSTEM) {
        for (int i = 0; i < B->nsys; ++i) {
            sstep_params q = B->p;
            q.history = nullptr;
            q.history_cap = 0;
            int rc = sstep_gmres_solve(B->mats[i], f[i], x[i], &q, &res[i], stream);
            if (rc < 0) return rc;
        }
        return SSTEP_OK;
    }
    if (mode != SSTEP_BATCH_PERSISTENT) return SSTEP_ERR_ARG;
    int rc = batch_run_persistent(B, f, x, st);
    if (rc) return rc;
    for (int i = 0; i < B->nsys; ++i)
        CUDA_TRY(cudaMemcpyAsync(&B->h_states[i], B->ws + B->state_off[i], sizeof(SolverState), cudaMemcpyDeviceToHost,
                                 st));
    CUDA_TRY(cudaStreamSynchronize(st));
    for (int i = 0; i < B->nsys; ++i) {
        const SolverState& h = B->h_states[i];
        res[i].status = h.status;
        res[i].cycles = h.cycles;
        res[i].iters = h.iters;
        res[i].matvecs = h.matvecs;
        res[i].relres = h.relres;
        res[i].history_len = 0;
    }
    return SSTEP_OK;
}

int sstep_batch_tune(sstep_batch B, const double* const* f, double* const* x, int* threads, int* ctas_per_sm,
                     int* largest_first, int* cluster, int64_t* coop_min_n, void* stream) {
    if (!B || !f || !x) return SSTEP_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    // keep the initial guesses to restore them after every trial
    std::vector<double*> saved(B->nsys, nullptr);
    int rc = SSTEP_OK;
    for (int i = 0; i < B->nsys && !rc; ++i) {
        const size_t bytes = sizeof(double) * B->mats[i]->A.n;
        if (cudaMalloc((void**)&saved[i], bytes) != cudaSuccess) rc = SSTEP_ERR_OOM;
        else if (cudaMemcpyAsync(saved[i], x[i], bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) rc = SSTEP_ERR_CUDA;
    }
    int64_t nmax = 1;
    for (int i = 0; i < B->nsys; ++i) nmax = std::max<int64_t>(nmax, B->mats[i]->A.n);
    // candidates: one CTA per system (block size, CTAs per SM, queue order), and clusters
    // of 2, 4 or 8 CTAs for the systems with at least a quarter or a half of the largest n
    struct Cand {
        int t, c, o, g;
        int64_t nb;
    };
    std::vector<Cand> cands;
    for (int t : {128, 256})
        for (int c : {1, 2, 4})
            for (int o : {1, 0})
                if (!(t == 256 && c == 4)) cands.push_back({t, c, o, 1, 0});
    for (int g : {2, 4, 8})
        for (int c : {1, 2})
            for (int64_t nb : {std::max<int64_t>(1, nmax / 4), std::max<int64_t>(1, nmax / 2)})
                cands.push_back({256, c, 1, g, nb});
    double best = 1e300;
    Cand bestc{B->threads, B->ctas_per_sm, B->largest_first, B->cluster, B->nbig};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (const Cand& cd : cands) {
        if (rc) break;
        B->threads = cd.t;
        B->ctas_per_sm = cd.c;
        B->largest_first = cd.o;
        B->cluster = cd.g;
        B->nbig = cd.nb;
        for (int i = 0; i < B->nsys; ++i)
            cudaMemcpyAsync(x[i], saved[i], sizeof(double) * B->mats[i]->A.n, cudaMemcpyDeviceToDevice, st);
        cudaEventRecord(e0, st);
        const int r = batch_run_persistent(B, f, x, st);
        cudaEventRecord(e1, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) rc = SSTEP_ERR_CUDA;
        if (r == SSTEP_ERR_ARG) continue;      // this configuration cannot be launched here
        if (r) rc = r;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (!rc && ms < best) {
            best = ms;
            bestc = cd;
        }
    }
    for (int i = 0; i < B->nsys; ++i) {
        if (saved[i]) {
            cudaMemcpyAsync(x[i], saved[i], sizeof(double) * B->mats[i]->A.n, cudaMemcpyDeviceToDevice, st);
        }
    }
    cudaStreamSynchronize(st);
    for (double* q : saved)
        if (q) cudaFree(q);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    B->threads = bestc.t;
    B->ctas_per_sm = bestc.c;
    B->largest_first = bestc.o;
    B->cluster = bestc.g;
    B->nbig = bestc.nb;
    if (threads) *threads = bestc.t;
    if (ctas_per_sm) *ctas_per_sm = bestc.c;
    if (largest_first) *largest_first = bestc.o;
    if (cluster) *cluster = bestc.g;
    if (coop_min_n) *coop_min_n = bestc.nb;
    return rc;
}

int sstep_batch_configure(sstep_batch B, int threads, int ctas_per_sm, int largest_first, int cluster,
                          int64_t coop_min_n) {
    if (!B || threads < 32 || threads > 256 || threads % 32 || ctas_per_sm < 1 || ctas_per_sm > 16 || cluster < 1 ||
        cluster > kBatchCopies || coop_min_n < 0)
        return SSTEP_ERR_ARG;
    B->threads = threads;
    B->ctas_per_sm = ctas_per_sm;
    B->largest_first = largest_first ? 1 : 0;
    B->cluster = cluster;
    B->nbig = coop_min_n;
    return SSTEP_OK;
}

int sstep_batch_destroy(sstep_batch B) {
    if (!B) return SSTEP_ERR_ARG;
    if (B->graph) cudaGraphExecDestroy(B->graph);
    if (B->ws) cudaFree(B->ws);
    if (B->d_sys) cudaFree(B->d_sys);
    if (B->d_order) cudaFree(B->d_order);
    if (B->d_queue) cudaFree(B->d_queue);
    if (B->d_init) cudaFree(B->d_init);
    if (B->h_states) cudaFreeHost(B->h_states);
    delete B;
    return SSTEP_OK;
}

}  // extern "C"
