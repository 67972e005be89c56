// Online stage of Algorithm 1: f = G~^{-1} K~^* u (Eq. 4.2), with optional
// iterative refinement on the approximate normal equation (Eq. 4.3):
//   f <- f + G~^{-1} (K~^* u - K~^* K~ f),
// the residual always formed with the FP32 applies of K~ and K~^* (also when
// the handle computes its applies in split BF16), so that the iteration
// converges to the FP32 solution of Eq. 4.3 at a rate set by ||I - G~^{-1} K~^*K~||.
#include "bf.cuh"
#include "hss.cuh"

namespace fio {
namespace {
// r = a - b ; f += d  (column blocks, ld)
__global__ void k_sub(const float2* __restrict__ a, const float2* __restrict__ b, float2* __restrict__ r, int64_t n,
                      int64_t lda, int64_t ldb, int64_t ldr) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    int col = blockIdx.y;
    if (i < n) r[col * ldr + i] = csub(a[col * lda + i], b[col * ldb + i]);
}
__global__ void k_add(float2* __restrict__ f, const float2* __restrict__ d, int64_t n, int64_t ldf, int64_t ldd) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    int col = blockIdx.y;
    if (i < n) f[col * ldf + i] = cadd(f[col * ldf + i], d[col * ldd + i]);
}
}  // namespace
}  // namespace fio

using namespace fio;

extern "C" fio_status fio_solve(const fio_bf* bf, const fio_hss* hc, const void* U, void* F, int64_t ld, int k,
                                int refine_steps, void* stream) {
    if (!bf || !hc) return fail(FIO_EINVAL, "fio_solve: null handle");
    if (bf->N() != hc->N) return fail(FIO_EINVAL, "fio_solve: BF and HSS sizes differ");
    if (k < 0 || ld < hc->N || refine_steps < 0) return fail(FIO_EINVAL, "fio_solve: bad k, ld or refine_steps");
    if (k == 0) return FIO_OK;
    if (!U || !F) return fail(FIO_EINVAL, "fio_solve: null vector");
    fio_hss* h = const_cast<fio_hss*>(hc);
    cudaStream_t st = as_stream(stream);
    const int64_t N = h->N;
    // 2D: the HSS is over the frequency index in quadtree (Morton) order; the
    // solve runs in that order and the result is reordered at the end.
    const bool mort = bf->d == 2;
    // buffers: T (K~^* u in the handle's precision), R1, R2 (refinement), T32 (FP32 K~^* u
    // when the handle computes in split precision)
    const bool split_refine = refine_steps > 0 && bf->split;
    const int nbuf = (refine_steps > 0 ? (split_refine ? 4 : 3) : 1) + (mort ? 1 : 0);
    FIO_TRY(h->fio_ws.ensure(size_t(nbuf) * ld * k * 8));
    float2* T = h->fio_ws.as<float2>();
    float2* Fout = static_cast<float2*>(F);
    if (mort) F = T + size_t(nbuf - 1) * ld * k;               // solution in Morton order
    const float2* Uc = static_cast<const float2*>(U);
    FIO_TRY(bf_apply_ord(bf, Uc, T, ld, k, 1, mort, st));      // T = K~^* u
    const int hp = bf->split ? 1 : 0;                          // node products in the handle's precision
    FIO_TRY(hss_solve_prec(h, T, F, ld, k, hp, st));           // f = G~^{-1} T
    if (refine_steps > 0) {
        float2* R1 = T + ld * k;
        float2* R2 = R1 + ld * k;
        // residuals of Eq. 4.3 against the FP32 applies of K~ and K~^* (precision request 0;
        // the handle's own setting is left as it is)
        float2* T32 = T;
        fio_status s = FIO_OK;
        if (split_refine) {
            T32 = R2 + ld * k;
            s = bf_apply_ord(bf, Uc, T32, ld, k, 1, mort, st, 0);
        }
        dim3 g(cdiv(N, 256), k);
        for (int it = 0; it < refine_steps && s == FIO_OK; ++it) {
            s = bf_apply_ord(bf, static_cast<const float2*>(F), R1, ld, k, 0, mort, st, 0);   // K~ f
            if (s == FIO_OK) s = bf_apply_ord(bf, R1, R2, ld, k, 1, mort, st, 0);             // K~^* K~ f
            if (s != FIO_OK) break;
            FIO_LAUNCH("k_sub", st, k_sub<<<g, 256, 0, st>>>(T32, R2, R1, N, ld, ld, ld));
            s = hss_solve_prec(h, R1, R2, ld, k, hp, st);
            if (s == FIO_OK) FIO_LAUNCH("k_add", st, k_add<<<g, 256, 0, st>>>(static_cast<float2*>(F), R2, N, ld, ld));
        }
        FIO_TRY(s);
    }
    if (mort) FIO_TRY(bf2d_unmorton(bf, static_cast<const float2*>(F), Fout, ld, k, st));
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}
