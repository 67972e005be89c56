// bf_apply_noalloc: the butterfly apply of bf_apply for callers that must not
// allocate device memory.
//
// Some callers cannot let a library call cudaMalloc: a host framework that
// owns every byte of device memory through its own allocator (and accounts
// for it), or a latency-critical loop in which a cudaMalloc -- which may
// synchronize the whole device -- is not acceptable.  bf_apply grows a
// per-handle scratch buffer on demand; this entry point instead keeps its
// coefficient state in one fixed array compiled into the library, so it
// never allocates or frees anything.
//
// The array is `static __device__`: every GPU that loads this library holds
// its kNoAllocScratchElems complex64 elements (32 MiB) until the process exits.
// In host code its name is only a host-side stand-in for the device symbol,
// so the device address is obtained with cudaGetSymbolAddress, once per
// device, by the first call made on that device (with that device current).
// Make that first call before starting any stream capture.
//
// Every call shares the one array and leaves its last contents behind.  The
// kernels write every state element before reading it, so nothing needs to
// be cleared between calls -- but two calls whose GPU work overlaps (on
// different streams, or from different host threads on the same device)
// race on the array: order them on one stream.
#include <mutex>

#include "bf.cuh"

namespace fio {
namespace {

constexpr int64_t kNoAllocScratchElems = int64_t(1) << 22;   // complex64 elements (32 MiB)
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float2 g_noalloc_scratch[kNoAllocScratchElems];

std::mutex g_noalloc_mu;
float2* g_noalloc_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (resolved once).
fio_status noalloc_scratch(float2** out) {
    int dev = 0;
    FIO_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(FIO_EINVAL, "bf_apply_noalloc: device index out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_status(e, "bf_apply_noalloc: cudaGetSymbolAddress of the scratch array");
        if (!p) return fail(FIO_ECUDA, "bf_apply_noalloc: scratch array has no device address");
        g_noalloc_ptr[dev] = static_cast<float2*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return FIO_OK;
}

}  // namespace
}  // namespace fio

using namespace fio;

extern "C" fio_status bf_apply_noalloc(const fio_bf* bf, const void* X, void* Y, int64_t ld, int k, int adjoint,
                                       void* stream) {
    if (!bf) return fail(FIO_EINVAL, "bf_apply_noalloc: null handle");
    if (k < 0 || ld < bf->n) return fail(FIO_EINVAL, "bf_apply_noalloc: need k >= 0 and ld >= N");
    if (k == 0) return FIO_OK;
    if (!X || !Y) return fail(FIO_EINVAL, "bf_apply_noalloc: null vector");
    if (bf->d != 1) return fail(FIO_EINVAL, "bf_apply_noalloc: 1D handles only (use bf_apply)");
    const int64_t stateN = int64_t(bf->n) * bf->r;   // one column of coefficient state
    const bool fused = bf_fused_ok(bf) && (!bf->force_unfused || bf->split);
    const int nstate = fused ? 1 : 2;
    if (nstate * stateN > kNoAllocScratchElems)
        return fail(FIO_EINVAL, "bf_apply_noalloc: one column needs " + std::to_string(nstate * stateN) +
                                    " complex64 elements of state; the fixed scratch holds " +
                                    std::to_string(kNoAllocScratchElems) + " (use bf_apply)");
    float2* scratch = nullptr;
    FIO_TRY(noalloc_scratch(&scratch));
    const int kc = int(std::min<int64_t>(std::min<int64_t>(k, 64), kNoAllocScratchElems / (nstate * stateN)));
    float2* s0 = scratch;
    float2* s1 = scratch + stateN * kc;
    cudaStream_t st = as_stream(stream);
    for (int c0 = 0; c0 < k; c0 += kc) {
        const int cc = std::min(kc, k - c0);
        const float2* Xc = static_cast<const float2*>(X) + c0 * ld;
        float2* Yc = static_cast<float2*>(Y) + c0 * ld;
        if (fused) FIO_TRY(bf_apply_fused(bf, Xc, Yc, ld, cc, adjoint, s0, st));
        else FIO_TRY(bf_apply_cols(bf, Xc, Yc, ld, cc, adjoint, s0, s1, st));
    }
    return FIO_OK;
}
