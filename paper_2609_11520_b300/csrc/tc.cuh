// Blackwell (sm_100 family) tensor-core and TMA primitives as inline PTX:
// tensor memory (TMEM) allocation, tcgen05.st / tcgen05.ld, tcgen05.mma of
// kind::f16 with the A operand in TMEM and the B operand in shared memory,
// commit to an mbarrier, bounded mbarrier waits, and TMA tile loads
// (cp.async.bulk.tensor) completing on an mbarrier.
//
// Operand layouts (checked on the device against a CPU product):
//  * B in shared memory, K-major, no swizzle: 8 x 16-byte core matrices; the
//    element (n, k) of a 16-bit operand sits at byte
//        (n / 8) * SBO + (k / 8) * LBO + (n % 8) * 16 + (k % 8) * 2,
//    LBO = distance of core matrices adjacent in K, SBO = distance of 8-row
//    groups.  One MMA consumes K = 16 (two core matrices along K).
//  * A in TMEM: row m in lane m, two consecutive 16-bit K elements per 32-bit
//    column (even k in the low half); one MMA consumes 8 columns.
//  * D in TMEM: row m in lane m, column n = FP32 D[m][n].
// A warp reaches the TMEM lanes 32 * (warp % 4) .. + 31.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace fio {
namespace tc {

// 16-bit operand parts: v = hi + lo with hi, lo FP16 (BF = false) or BF16 (BF = true).
template <bool BF> struct Half16;
template <> struct Half16<false> {
    using T2 = __half2;
    static __device__ __forceinline__ T2 pack(float a, float b) { return __floats2half2_rn(a, b); }
    static __device__ __forceinline__ float2 unpack(T2 v) { return __half22float2(v); }
    static __device__ __forceinline__ uint16_t one(float a) { return __half_as_ushort(__float2half_rn(a)); }
    static __device__ __forceinline__ float back(uint16_t v) { return __half2float(__ushort_as_half(v)); }
};
template <> struct Half16<true> {
    using T2 = __nv_bfloat162;
    static __device__ __forceinline__ T2 pack(float a, float b) { return __floats2bfloat162_rn(a, b); }
    static __device__ __forceinline__ float2 unpack(T2 v) { return __bfloat1622float2(v); }
    static __device__ __forceinline__ uint16_t one(float a) { return __bfloat16_as_ushort(__float2bfloat16_rn(a)); }
    static __device__ __forceinline__ float back(uint16_t v) { return __bfloat162float(__ushort_as_bfloat16(v)); }
};

// hi / lo parts of (a, b) as two packed 16-bit pairs
template <bool BF> __device__ __forceinline__ void split_pair(float a, float b, uint32_t& hi, uint32_t& lo) {
    using H = Half16<BF>;
    const typename H::T2 h = H::pack(a, b);
    const float2 f = H::unpack(h);
    const typename H::T2 l = H::pack(a - f.x, b - f.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

// Power-of-two scale sc (and 1 / sc) for the FP16 parts: largest |entry| (bounded by mx) into
// [2^14, 2^15), so that neither part overflows or loses bits to the FP16 exponent range.
__device__ __forceinline__ void row_scale(float mx, float& sc, float& isc) {
    const int ex = int((__float_as_uint(mx) >> 23) & 0xFF);
    const int se = ex == 0 ? 127 : min(max(268 - ex, 1), 253);
    sc = __uint_as_float(uint32_t(se) << 23);
    isc = __uint_as_float(uint32_t(254 - se) << 23);
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Generic-proxy shared-memory writes made visible to the tensor core / TMA (async proxy).
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Whole warp: allocate ncols (power of two, 32..512) TMEM columns; the base address is written to *dst.
// The CTA keeps its permit to allocate (a persistent CTA allocates again for its next work item).
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, int ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst)), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, int ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 32 lanes x 16 consecutive 32-bit columns (one lane per thread).
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor (K-major, no swizzle).
__host__ __device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return uint64_t((addr >> 4) & 0x3FFF) | (uint64_t((lbo >> 4) & 0x3FFF) << 16) | (uint64_t((sbo >> 4) & 0x3FFF) << 32) |
           (uint64_t(1) << 46);
}
// Instruction descriptor of kind::f16: FP32 accumulator, A and B both FP16 (bf16 = false) or
// both BF16 (bf16 = true), both K-major, M x N.
__host__ __device__ __forceinline__ uint32_t idesc_f16(bool bf16, int M, int N) {
    const uint32_t f = bf16 ? 1u : 0u;
    return (1u << 4) | (f << 7) | (f << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}
// D (+)= A B, A in TMEM, B by descriptor; issued by one thread.
__device__ __forceinline__ void mma_f16_ts(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t idesc, int accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
        "r"(a), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// Arrive on the mbarrier once every previously issued MMA of this thread has completed.
__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(mbar))
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* m, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(m)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ uint32_t mbar_try(uint64_t* m, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(m)), "r"(parity)
        : "memory");
    return ok;
}
// Wait for the phase with the given parity to complete, at most `limit` polls
// (each poll may suspend the thread for a short, hardware-chosen time).
// Returns false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* m, uint32_t parity, int limit = 1 << 22) {
    for (int i = 0; i < limit; ++i)
        if (mbar_try(m, parity)) return true;
    return false;
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* m, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(m)), "r"(bytes) : "memory");
}
// TMA tile loads into this CTA's shared memory, completing `bytes` on the mbarrier.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* mbar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(mbar))
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* mbar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(mbar))
        : "memory");
}

}  // namespace tc
}  // namespace fio
