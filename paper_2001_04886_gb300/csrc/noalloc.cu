// The Gram pass without any device allocation.
//
// sstep_gram needs a caller-supplied scratch buffer (per-CTA partial sums and an
// arrival counter). Some callers cannot allocate device memory at the point of
// the call: applications that fix their device-memory budget at start-up and
// forbid later allocations, and plug-in hosts whose own allocator owns all device
// memory (an allocation behind its back breaks its accounting or fails). For them
// this file keeps the scratch in a fixed, file-scope device array that exists on
// every GPU that loads the library, for the life of the process.
#include <mutex>

#include "kernels.cuh"

using namespace sstep;

namespace {

// 256 bytes for the arrival counter, then the per-CTA partials of the largest
// Gram grid on a device of up to 192 multiprocessors (8 CTAs per multiprocessor,
// 8 x 9 doubles each): 884,992 bytes in all. A device with more multiprocessors
// is refused (SSTEP_ERR_ARG).
constexpr size_t kCounterBytes = 256;
constexpr size_t kMaxSms = 192;
constexpr size_t kPartialDoubles = kMaxSms * 8 * 8 * (SSTEP_MAX_S + 1);
constexpr size_t kScratchBytes = kCounterBytes + kPartialDoubles * sizeof(double);

static __device__ __align__(256) unsigned char g_gram_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_lock;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of g_gram_scratch on the current device. In host code the
// array's name is only a host-side stand-in, so the address must come from the
// runtime, with that device current: once per device at the first call, and again
// at every call on a stream that is not being captured (a cudaDeviceReset reloads
// the module, and the array may then live elsewhere).
int scratch_address(cudaStream_t st, void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SSTEP_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return SSTEP_ERR_ARG;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
        cudaGetLastError();
        return SSTEP_ERR_CUDA;
    }
    std::lock_guard<std::mutex> guard(g_setup_lock);
    if (!g_scratch_addr[dev] || cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_gram_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return SSTEP_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return SSTEP_OK;
}

}  // namespace

extern "C" int sstep_gram_noalloc(int64_t n, const double* V, int64_t ldv, int ka, const double* Y, int64_t ldy,
                                  int kb, double* C, int ldc, void* stream) {
    if (ka < 1 || ka > SSTEP_MAX_COLS || kb < 1 || kb > SSTEP_MAX_S + 1) return SSTEP_ERR_ARG;
    if (n < 0 || !V || !Y || !C || ldv < n || ldy < n || ldc < ka) return SSTEP_ERR_ARG;
    if ((size_t)fp64_gram_partials_doubles() > kPartialDoubles) return SSTEP_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (n == 0)   // C = 0: the ka x kb entries only (the rows below ka of each column are the caller's)
        return cudaMemset2DAsync(C, sizeof(double) * ldc, 0, sizeof(double) * ka, kb, st) == cudaSuccess
                   ? SSTEP_OK
                   : SSTEP_ERR_CUDA;
    void* base = nullptr;
    int rc = scratch_address(st, &base);
    if (rc) return rc;
    // the arrival counter must start at zero; the partials are overwritten before use
    if (cudaMemsetAsync(base, 0, sizeof(unsigned), st) != cudaSuccess) return SSTEP_ERR_CUDA;
    Scratch sc{(double*)((char*)base + kCounterBytes), (unsigned*)base};
    Epi e;
    e.mode = EPI_NONE;
    e.out = C;
    e.ldo = ldc;
    launch_gram(n, V, ldv, ka, Y, ldy, kb, 0, sc, e, GATE_NONE, st);
    return cudaGetLastError() == cudaSuccess ? SSTEP_OK : SSTEP_ERR_CUDA;
}
