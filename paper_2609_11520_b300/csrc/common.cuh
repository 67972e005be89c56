// Shared device/host utilities of the FIO library: complex arithmetic,
// status plumbing, allocation helpers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/fio.h"

namespace fio {

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
fio_status fail(fio_status st, const std::string& msg);
fio_status cuda_status(cudaError_t e, const char* what);

#define FIO_CUDA(call)                                                      \
    do {                                                                    \
        cudaError_t e__ = (call);                                           \
        if (e__ != cudaSuccess) return ::fio::cuda_status(e__, #call);      \
    } while (0)

#define FIO_TRY(call)                                                       \
    do {                                                                    \
        fio_status s__ = (call);                                            \
        if (s__ != FIO_OK) return s__;                                      \
    } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// ---------------------------------------------------------------- profiling
// When enabled (fio_profile_enable), every kernel launch of the library is
// bracketed by a pair of CUDA events on its stream; fio_profile_report sums
// the elapsed times per kernel name.
bool profiling_enabled();
void prof_begin(const char* name, cudaStream_t st);
void prof_end(cudaStream_t st);
struct ProfScope {
    cudaStream_t st;
    bool on;
    ProfScope(const char* name, cudaStream_t s) : st(s), on(profiling_enabled()) {
        if (on) prof_begin(name, st);
    }
    ~ProfScope() {
        if (on) prof_end(st);
    }
};
#define FIO_LAUNCH(name, st, ...)            \
    do {                                    \
        ::fio::ProfScope ps__(name, st);    \
        __VA_ARGS__;                        \
    } while (0)

// Device buffer owned by a handle.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    fio_status ensure(size_t need) {
        if (need <= bytes) return FIO_OK;
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        if (cudaMalloc(&p, need) != cudaSuccess) {
            cudaGetLastError();
            return fail(FIO_ENOMEM, "cudaMalloc of " + std::to_string(need) + " bytes failed");
        }
        bytes = need;
        return FIO_OK;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <class T> T* as() const { return reinterpret_cast<T*>(p); }
};

// ---------------------------------------------------------------- complex
struct cf { float x, y; };

__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) {
    return make_float2(a.x + b.x, a.y + b.y);
}
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) {
    return make_float2(a.x - b.x, a.y - b.y);
}
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) {
    return make_float2(a.x * s, a.y * s);
}
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// acc += a * b
__host__ __device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
}
// acc += conj(a) * b
__host__ __device__ __forceinline__ void cfmac(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y));
}

__host__ __device__ __forceinline__ double2 zmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ void zfma(double2& acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}
__host__ __device__ __forceinline__ void zfmac(double2& acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(-a.y, b.x, acc.y));
}

inline int ilog2_exact(int64_t v) {
    int l = 0;
    while ((int64_t(1) << l) < v) ++l;
    return ((int64_t(1) << l) == v) ? l : -1;
}

inline unsigned cdiv(int64_t a, int64_t b) { return unsigned((a + b - 1) / b); }

// One-time set-up per device (kernel attributes are per device).  run(f) calls f()
// with the device current the first time it is asked on that device, under a lock, so
// that no other host thread gets past run() on that device before f() has finished; the
// device counts as done only when f() returned cudaSuccess (a failed set-up is retried
// on the next call and its error is returned).
struct PerDeviceOnce {
    std::mutex mu;
    uint64_t done = 0;
    template <class F> cudaError_t run(F f) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= 64) return f();
        std::lock_guard<std::mutex> lock(mu);
        const uint64_t bit = uint64_t(1) << dev;
        if (done & bit) return cudaSuccess;
        e = f();
        if (e == cudaSuccess) done |= bit;
        return e;
    }
};

}  // namespace fio
