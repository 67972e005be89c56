// Batched complex GEMM (declared in gemm.cuh).  One CTA computes a 64 x 64
// tile of one batch entry: 256 threads, each a 4 x 4 block of outputs
// (rows ty + 16 a, columns tx + 16 b); the K dimension advances in slabs of
// BK staged in shared memory, op(A) as [k][i] and op(B) as [k][j], with the
// global loads coalesced along the stored leading dimension of each operand.
#include <algorithm>

#include "cplx.cuh"
#include "gemm.cuh"

namespace fio {
namespace {

constexpr int TM = 64, TN = 64, NTH = 256;

template <class C, int BK, bool CA, bool CB>
__global__ void __launch_bounds__(NTH) k_bgemm(int m, int n, int k, typename RealOf<C>::T alpha, const C* __restrict__ A,
                                               int64_t lda, int64_t sA, const C* __restrict__ B, int64_t ldb, int64_t sB,
                                               typename RealOf<C>::T beta, C* __restrict__ Cm, int64_t ldc, int64_t sC) {
    using R = typename RealOf<C>::T;
    __shared__ C As[BK][TM + 1];
    __shared__ C Bs[BK][TN + 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int i0 = blockIdx.x * TM, j0 = blockIdx.y * TN;
    const int64_t bz = blockIdx.z;
    A += bz * sA;
    B += bz * sB;
    Cm += bz * sC;
    C acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = czero<C>();
    for (int k0 = 0; k0 < k; k0 += BK) {
        // op(A)(i, kk): 'N' reads A[i + kk lda] (consecutive i), 'C' reads conj A[kk + i lda] (consecutive kk)
#pragma unroll
        for (int q = 0; q < TM * BK / NTH; ++q) {
            const int e = tid + q * NTH;
            int i, kk;
            if (!CA) {
                i = e % TM;
                kk = e / TM;
            } else {
                kk = e % BK;
                i = e / BK;
            }
            const int gi = i0 + i, gk = k0 + kk;
            C v = czero<C>();
            if (gi < m && gk < k) v = CA ? gconj(A[gk + int64_t(gi) * lda]) : A[gi + int64_t(gk) * lda];
            As[kk][i] = v;
        }
        // op(B)(kk, j): 'N' reads B[kk + j ldb] (consecutive kk), 'C' reads conj B[j + kk ldb] (consecutive j)
#pragma unroll
        for (int q = 0; q < TN * BK / NTH; ++q) {
            const int e = tid + q * NTH;
            int j, kk;
            if (!CB) {
                kk = e % BK;
                j = e / BK;
            } else {
                j = e % TN;
                kk = e / TN;
            }
            const int gj = j0 + j, gk = k0 + kk;
            C v = czero<C>();
            if (gj < n && gk < k) v = CB ? gconj(B[gj + int64_t(gk) * ldb]) : B[gk + int64_t(gj) * ldb];
            Bs[kk][j] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            C av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[kk][ty + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tx + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) gfma(acc[a][b], av[a], bv[b]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int gi = i0 + ty + 16 * a;
        if (gi >= m) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int gj = j0 + tx + 16 * b;
            if (gj >= n) continue;
            C* c = Cm + gi + int64_t(gj) * ldc;
            C v = gscale(acc[a][b], alpha);
            if (beta != R(0)) v = gadd(v, gscale(*c, beta));
            *c = v;
        }
    }
}

// C = beta C where op(A) op(B) is empty (k = 0)
template <class C>
__global__ void k_scale(int m, int n, typename RealOf<C>::T beta, C* Cm, int64_t ldc, int64_t sC) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= int64_t(m) * n) return;
    C* c = Cm + int64_t(blockIdx.y) * sC + (e % m) + (e / m) * ldc;
    *c = beta == 0 ? czero<C>() : gscale(*c, beta);
}

template <class C, int BK, bool CA, bool CB>
fio_status launch(int m, int n, int k, double alpha, const C* A, int64_t lda, int64_t sA, const C* B, int64_t ldb,
                  int64_t sB, double beta, C* Cm, int64_t ldc, int64_t sC, int batch, cudaStream_t st) {
    using R = typename RealOf<C>::T;
    for (int b0 = 0; b0 < batch; b0 += 65535) {
        const int nb = std::min(batch - b0, 65535);
        dim3 g(cdiv(m, TM), cdiv(n, TN), nb);
        FIO_LAUNCH("k_bgemm", st,
                   (k_bgemm<C, BK, CA, CB><<<g, NTH, 0, st>>>(m, n, k, R(alpha), A + b0 * sA, lda, sA, B + b0 * sB, ldb, sB,
                                                              R(beta), Cm + b0 * sC, ldc, sC)));
    }
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}

}  // namespace

template <class C>
fio_status bgemm(char ta, char tb, int m, int n, int k, double alpha, const C* A, int64_t lda, int64_t sA, const C* B,
                 int64_t ldb, int64_t sB, double beta, C* Cm, int64_t ldc, int64_t sC, int batch, cudaStream_t st) {
    if (m <= 0 || n <= 0 || batch <= 0) return FIO_OK;
    if ((ta != 'N' && ta != 'C') || (tb != 'N' && tb != 'C')) return fail(FIO_EINVAL, "bgemm: op must be 'N' or 'C'");
    if (k <= 0) {
        using R = typename RealOf<C>::T;
        for (int b0 = 0; b0 < batch; b0 += 65535) {
            dim3 g(cdiv(int64_t(m) * n, 256), std::min(batch - b0, 65535));
            k_scale<C><<<g, 256, 0, st>>>(m, n, R(beta), Cm + b0 * sC, ldc, sC);
        }
        FIO_CUDA(cudaGetLastError());
        return FIO_OK;
    }
    constexpr int BK = sizeof(C) == 8 ? 16 : 8;
    const bool ca = ta == 'C', cb = tb == 'C';
    if (!ca && !cb) return launch<C, BK, false, false>(m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, Cm, ldc, sC, batch, st);
    if (!ca && cb) return launch<C, BK, false, true>(m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, Cm, ldc, sC, batch, st);
    if (ca && !cb) return launch<C, BK, true, false>(m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, Cm, ldc, sC, batch, st);
    return launch<C, BK, true, true>(m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, Cm, ldc, sC, batch, st);
}

template fio_status bgemm<float2>(char, char, int, int, int, double, const float2*, int64_t, int64_t, const float2*,
                                  int64_t, int64_t, double, float2*, int64_t, int64_t, int, cudaStream_t);
template fio_status bgemm<double2>(char, char, int, int, int, double, const double2*, int64_t, int64_t, const double2*,
                                   int64_t, int64_t, double, double2*, int64_t, int64_t, int, cudaStream_t);

}  // namespace fio
