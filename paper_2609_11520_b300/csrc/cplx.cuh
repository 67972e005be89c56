// Precision-generic complex helpers (complex64 = float2, complex128 = double2)
// and block-level reductions used by the per-node dense kernels of the HSS
// construction and the ULV factorization.
#pragma once
#include <cuda_runtime.h>

namespace fio {

template <class C> struct RealOf;
template <> struct RealOf<float2> { using T = float; };
template <> struct RealOf<double2> { using T = double; };

__device__ __forceinline__ float2 cx(float a, float b, float2*) { return make_float2(a, b); }
__device__ __forceinline__ double2 cx(double a, double b, double2*) { return make_double2(a, b); }
template <class C> __device__ __forceinline__ C mkc(typename RealOf<C>::T a, typename RealOf<C>::T b) {
    return cx(a, b, (C*)nullptr);
}
template <class C> __device__ __forceinline__ C czero() { return mkc<C>(0, 0); }

template <class C> __device__ __forceinline__ C cvt(float2 v) { return mkc<C>(v.x, v.y); }
template <class C> __device__ __forceinline__ C cvt(double2 v) {
    return mkc<C>(typename RealOf<C>::T(v.x), typename RealOf<C>::T(v.y));
}
__device__ __forceinline__ float2 to_f2(float2 v) { return v; }
__device__ __forceinline__ float2 to_f2(double2 v) { return make_float2(float(v.x), float(v.y)); }

template <class C> __device__ __forceinline__ C gadd(C a, C b) { return mkc<C>(a.x + b.x, a.y + b.y); }
template <class C> __device__ __forceinline__ C gsub(C a, C b) { return mkc<C>(a.x - b.x, a.y - b.y); }
template <class C> __device__ __forceinline__ C gmul(C a, C b) {
    return mkc<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
template <class C> __device__ __forceinline__ C gmulc(C a, C b) {
    return mkc<C>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
template <class C> __device__ __forceinline__ C gconj(C a) { return mkc<C>(a.x, -a.y); }
template <class C> __device__ __forceinline__ C gscale(C a, typename RealOf<C>::T s) { return mkc<C>(a.x * s, a.y * s); }
template <class C> __device__ __forceinline__ typename RealOf<C>::T gabs2(C a) { return a.x * a.x + a.y * a.y; }
// a / b
template <class C> __device__ __forceinline__ C gdiv(C a, C b) {
    typename RealOf<C>::T d = b.x * b.x + b.y * b.y;
    return mkc<C>((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
// acc += a * b ; acc += conj(a) * b
template <class C> __device__ __forceinline__ void gfma(C& acc, C a, C b) {
    acc.x += a.x * b.x - a.y * b.y;
    acc.y += a.x * b.y + a.y * b.x;
}
template <class C> __device__ __forceinline__ void gfmac(C& acc, C a, C b) {
    acc.x += a.x * b.x + a.y * b.y;
    acc.y += a.x * b.y - a.y * b.x;
}

template <class T> __device__ __forceinline__ T warp_sum(T v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum of one value per thread over the block (blockDim.x multiple of 32, <= 1024).
// `red` needs 32 entries; all threads receive the sum.
template <class T> __device__ T block_sum(T v, T* red) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    T s = (threadIdx.x < nw) ? red[threadIdx.x] : T(0);
    if (w == 0) s = warp_sum(s);
    if (threadIdx.x == 0) red[0] = s;
    __syncthreads();
    s = red[0];
    __syncthreads();
    return s;
}

// Block argmax of (value, index); ties go to the smaller index.
template <class T> __device__ void block_argmax(T& v, int& idx, T* redv, int* redi) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        T ov = __shfl_xor_sync(0xffffffffu, v, o);
        int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
    }
    __syncthreads();
    if (lane == 0) { redv[w] = v; redi[w] = idx; }
    __syncthreads();
    if (w == 0) {
        v = lane < nw ? redv[lane] : T(-1);
        idx = lane < nw ? redi[lane] : 0x7fffffff;
        for (int o = 16; o > 0; o >>= 1) {
            T ov = __shfl_xor_sync(0xffffffffu, v, o);
            int oi = __shfl_xor_sync(0xffffffffu, idx, o);
            if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
        }
        if (lane == 0) { redv[0] = v; redi[0] = idx; }
    }
    __syncthreads();
    v = redv[0];
    idx = redi[0];
    __syncthreads();
}

}  // namespace fio
