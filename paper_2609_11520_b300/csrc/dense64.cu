// Large HSS nodes (levels with few nodes of size m in the hundreds to
// thousands, as in 2D where the ranks grow like sqrt(N)): level-3
// formulations of the per-node steps of Section 3.1-3.3 and of the ULV
// factorization (Section 2.4), batched over the nodes of a level.
//
// The one-CTA-per-node kernels apply Householder reflectors one at a time,
// which streams O(m^2 r) data through one SM.  Here every step is a sequence
// of batched GEMMs (the library's own, gemm.cu) and small blocked factorizations
// (one CTA per node and diagonal block):
//   Omega^+ = Omega^* (Omega Omega^*)^{-1}, W = Y Omega^+   (Gram matrix, Cholesky)
//   Gamma = orthonormal basis of null(Omega): (I - Omega^+ Omega) E for a
//       Gaussian E (s x (s-m)), projected twice, CholQR2
//   rank-revealing step: pivoted Cholesky of A^* A, A = Y Gamma, truncated where
//       the pivot |R_kk|^2 <= thr^2 -- the pivots and order of the column-pivoted
//       QR of A; U = orthonormalized pivot columns of A (CholQR2), completed by
//       Gaussian columns where a node's rank is below the level rank
//   ULV: Q2 = U R^{-1} (CholQR2), Q1 = orthonormal complement (projected
//       Gaussian block, CholQR2), Q = [Q1 Q2] with Q^* U = [0; R]; then the
//       same partial Cholesky, D^_21, D^_22 and W as the one-CTA kernels.
//
// Precision.  The bulk products of the node pass run in FP32 (complex64 CGEMM)
// when the HSS tolerance is at least 1e-4 (FP64 below): the Gram matrix
// Omega Omega^* of a Gaussian block with s >= m + p columns is well
// conditioned, and FP32 rounding (~1e-6 relative) stays 100x under the
// truncation threshold.  The postprocessing and ULV products run in FP32.
// FP64 is kept where the arithmetic needs it: the Gram matrix A^* A and its
// pivoted Cholesky (the pivots are compared with thr^2 = tol^2 max |Y_j|^2),
// the root (whose sample block is nearly square), the Cholesky factorization
// of the eliminated diagonal blocks of the ULV, the merge and the root
// Cholesky.
#include <mutex>
#include <string>
#include <type_traits>

#include "cplx.cuh"
#include "gemm.cuh"
#include "hss.cuh"

namespace fio {
namespace dense {

using z = double2;
using c = float2;
constexpr int NB = 32;     // block size of the blocked factorizations
constexpr int TBD = 256;
constexpr double kFp32Tol = 1e-4;

int g_large_min = 384;

template <class C> inline C cval(double re) {
    C v;
    v.x = decltype(v.x)(re);
    v.y = 0;
    return v;
}

// ---------------------------------------------------------------- GEMM
// C = alpha op(A) op(B) + beta C for `batch` nodes (element strides sA, sB, sC); op: 'N' or 'C'.
// The library's own batched complex GEMM (gemm.cu).
template <class T>
fio_status gemm(char ta, char tb, int m, int n, int k, double alpha, const T* A, int64_t lda, int64_t sA, const T* B,
                int64_t ldb, int64_t sB, double beta, T* C, int64_t ldc, int64_t sC, int batch, cudaStream_t st) {
    return bgemm<T>(ta, tb, m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch, st);
}

// ---------------------------------------------------------------- kernels
// Cholesky of the jb x jb diagonal block at (j0, j0), lower, in place; one CTA per node.
template <class C>
__global__ void k_potrf_diag(C* A, int64_t lda, int64_t sA, int j0, int jb, int* status) {
    using R = typename RealOf<C>::T;
    __shared__ C L[NB][NB + 1];
    C* At = A + blockIdx.x * sA + j0 + j0 * lda;
    for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) L[e % jb][e / jb] = At[e % jb + (e / jb) * lda];
    __syncthreads();
    for (int cc = 0; cc < jb; ++cc) {
        if (threadIdx.x == 0) {
            R d = L[cc][cc].x;
            if (!(d > R(0))) {
                atomicExch(status, FIO_ENOTHPD);
                d = R(1);
            }
            L[cc][cc] = mkc<C>(sqrt(d), R(0));
        }
        __syncthreads();
        const R inv = R(1) / L[cc][cc].x;
        for (int i = cc + 1 + threadIdx.x; i < jb; i += blockDim.x) L[i][cc] = gscale(L[i][cc], inv);
        __syncthreads();
        for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) {
            const int i = e % jb, j = e / jb;
            if (j > cc && i >= j) L[i][j] = gsub(L[i][j], gmul(L[i][cc], gconj(L[j][cc])));
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) {
        const int i = e % jb, j = e / jb;
        At[i + j * lda] = i >= j ? L[i][j] : czero<C>();
    }
}

// Rows of X (nrows x jb, ld ldx) solve X L^* = B in place (HERM: L^* upper, forward
// over columns) or X L = B (backward over columns); L: jb x jb lower at Lm.
template <class C, bool HERM>
__global__ void k_trsm_rows(C* X, int64_t ldx, int64_t sX, int nrows, const C* Lm, int64_t ldl, int64_t sL, int jb) {
    using R = typename RealOf<C>::T;
    __shared__ C L[NB][NB + 1];
    const C* Lt = Lm + blockIdx.y * sL;
    for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) L[e % jb][e / jb] = Lt[e % jb + (e / jb) * ldl];
    __syncthreads();
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    C* x = X + blockIdx.y * sX + r;
    if (HERM) {   // sum_{q <= cc} X[q] conj(L[cc][q]) = B[cc]
        for (int cc = 0; cc < jb; ++cc) {
            C a = x[cc * ldx];
            for (int q = 0; q < cc; ++q) a = gsub(a, gmul(x[q * ldx], gconj(L[cc][q])));
            x[cc * ldx] = gscale(a, R(1) / L[cc][cc].x);
        }
    } else {      // sum_{q >= cc} X[q] L[q][cc] = B[cc]
        for (int cc = jb - 1; cc >= 0; --cc) {
            C a = x[cc * ldx];
            for (int q = cc + 1; q < jb; ++q) a = gsub(a, gmul(x[q * ldx], L[q][cc]));
            x[cc * ldx] = gscale(a, R(1) / L[cc][cc].x);
        }
    }
}

// Columns of X (jb x ncols, ld ldx) solve L X = B in place, L jb x jb lower.
template <class C>
__global__ void k_trsm_cols(C* X, int64_t ldx, int64_t sX, int ncols, const C* Lm, int64_t ldl, int64_t sL, int jb) {
    using R = typename RealOf<C>::T;
    __shared__ C L[NB][NB + 1];
    const C* Lt = Lm + blockIdx.y * sL;
    for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) L[e % jb][e / jb] = Lt[e % jb + (e / jb) * ldl];
    __syncthreads();
    const int cc = blockIdx.x * blockDim.x + threadIdx.x;
    if (cc >= ncols) return;
    C* x = X + blockIdx.y * sX + cc * ldx;
    for (int i = 0; i < jb; ++i) {
        C a = x[i];
        for (int q = 0; q < i; ++q) a = gsub(a, gmul(L[i][q], x[q]));
        x[i] = gscale(a, R(1) / L[i][i].x);
    }
}

// Pivoted Cholesky (FP64) of a Hermitian n x n block (full storage), steps [j0, j1) of
// one panel, one CTA per node.  dg: updated diagonal; perm: row order; stops (done = 1,
// rank = k) at the first step k >= maxk or with largest remaining pivot <= thr2.
__global__ void k_pstrf_panel(z* A, int64_t lda, int64_t sA, int n, int j0, int j1, int maxk, const double* thr2,
                              double* dg_all, int* perm_all, int* rank, int* sat, int* done) {
    __shared__ double rv[32];
    __shared__ int ri[32];
    const int t = blockIdx.x;
    if (done[t]) return;
    z* At = A + t * sA;
    double* dg = dg_all + int64_t(t) * n;
    int* perm = perm_all + int64_t(t) * n;
    for (int k = j0; k < j1; ++k) {
        double bv = -1.0;
        int bi = 0x7fffffff;
        for (int i = k + threadIdx.x; i < n; i += blockDim.x)
            if (dg[i] > bv) { bv = dg[i]; bi = i; }
        block_argmax(bv, bi, rv, ri);
        const int p = bi;
        const double dmax = bv;
        if (k >= maxk || !(dmax > thr2[t])) {
            if (threadIdx.x == 0) {
                rank[t] = k;
                sat[t] = (k >= maxk && dmax > thr2[t]) ? 1 : 0;
                done[t] = 1;
            }
            return;
        }
        if (p != k) {   // symmetric swap of rows and columns k, p
            for (int j = threadIdx.x; j < n; j += blockDim.x) {
                z a = At[k + j * lda];
                At[k + j * lda] = At[p + j * lda];
                At[p + j * lda] = a;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                z a = At[i + int64_t(k) * lda];
                At[i + int64_t(k) * lda] = At[i + int64_t(p) * lda];
                At[i + int64_t(p) * lda] = a;
            }
            if (threadIdx.x == 0) {
                double d = dg[k]; dg[k] = dg[p]; dg[p] = d;
                int q = perm[k]; perm[k] = perm[p]; perm[p] = q;
            }
            __syncthreads();
        }
        const double lkk = sqrt(dmax);
        for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) {
            z a = At[i + int64_t(k) * lda];
            for (int q = j0; q < k; ++q) a = gsub(a, gmul(At[i + int64_t(q) * lda], gconj(At[k + int64_t(q) * lda])));
            a = gscale(a, 1.0 / lkk);
            At[i + int64_t(k) * lda] = a;
            dg[i] -= gabs2(a);
        }
        __syncthreads();
        if (threadIdx.x == 0) At[k + int64_t(k) * lda] = make_double2(lkk, 0.0);
        __syncthreads();
    }
}

// After maxk steps without stopping: rank = maxk, sat if a remaining pivot exceeds thr2.
__global__ void k_pstrf_finish(int n, int maxk, const double* thr2, const double* dg_all, int* rank, int* sat,
                               int* done) {
    __shared__ double rv[32];
    __shared__ int ri[32];
    const int t = blockIdx.x;
    if (done[t]) return;
    const double* dg = dg_all + int64_t(t) * n;
    double bv = -1.0;
    int bi = 0x7fffffff;
    for (int i = maxk + threadIdx.x; i < n; i += blockDim.x)
        if (dg[i] > bv) { bv = dg[i]; bi = i; }
    block_argmax(bv, bi, rv, ri);
    if (threadIdx.x == 0) {
        rank[t] = maxk;
        sat[t] = (maxk < n && bv > thr2[t]) ? 1 : 0;
        done[t] = 1;
    }
}

__global__ void k_pstrf_init(const z* A, int64_t lda, int64_t sA, int n, double* dg, int* perm, int* done) {
    const int t = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) done[t] = 0;
    if (i >= n) return;
    dg[int64_t(t) * n + i] = A[t * sA + i + int64_t(i) * lda].x;
    perm[int64_t(t) * n + i] = i;
}

// Standard complex Gaussian from a counter hash (splitmix64 mixing, Box-Muller).
__device__ inline double2 hash_gauss(uint64_t seed, uint64_t a, uint64_t b) {
    auto mix = [](uint64_t x) {
        x += 0x9e3779b97f4a7c15ull;
        x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
        x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
        return x ^ (x >> 31);
    };
    const uint64_t h1 = mix(seed ^ mix(a * 0x100000001b3ull + b * 2));
    const uint64_t h2 = mix(h1 + 0x632be59bd9b4e019ull);
    const double u1 = (double(h1 >> 11) + 1.0) * (1.0 / 9007199254740992.0);
    const double u2 = double(h2 >> 11) * (1.0 / 9007199254740992.0);
    const double rr = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    return make_double2(rr * cs, rr * sn);
}

// M[:, cc] = A[:, perm[cc]] for cc < rank_t (the pivot columns), a Gaussian column beyond.
template <class C>
__global__ void k_gather_cols(const C* A, int m, int64_t sA, int c_all, const int* perm_all, const int* rank, int rl,
                              C* M, int64_t sM, uint64_t seed) {
    const int t = blockIdx.y;
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= int64_t(m) * rl) return;
    const int i = int(e % m), cc = int(e / m);
    if (cc < rank[t]) M[t * sM + i + int64_t(cc) * m] = A[t * sA + i + int64_t(perm_all[int64_t(t) * c_all + cc]) * m];
    else M[t * sM + i + int64_t(cc) * m] = cvt<C>(hash_gauss(seed, uint64_t(t), uint64_t(e)));
}

// b = a (rows x cols per node, any precisions)
template <class A, class B>
__global__ void k_cvt(const A* a, int64_t lda, int64_t sa, B* b, int64_t ldb, int64_t sb, int rows, int cols) {
    const int t = blockIdx.y;
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= int64_t(rows) * cols) return;
    const int i = int(e % rows), j = int(e / rows);
    b[t * sb + i + j * ldb] = cvt<B>(a[t * sa + i + j * lda]);
}
// b += a (FP64 accumulator, FP32 addend)
__global__ void k_acc(const c* a, int64_t lda, int64_t sa, z* b, int64_t ldb, int64_t sb, int rows, int cols) {
    const int t = blockIdx.y;
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= int64_t(rows) * cols) return;
    const int i = int(e % rows), j = int(e / rows);
    const c v = a[t * sa + i + j * lda];
    z& d = b[t * sb + i + j * ldb];
    d.x += v.x;
    d.y += v.y;
}
// B (cols x rows) = A^* (A rows x cols)
template <class C>
__global__ void k_conjT(const C* a, int64_t lda, int64_t sa, C* b, int64_t ldb, int64_t sb, int rows, int cols) {
    const int t = blockIdx.y;
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= int64_t(rows) * cols) return;
    const int i = int(e % rows), j = int(e / rows);
    b[t * sb + j + i * ldb] = gconj(a[t * sa + i + j * lda]);
}
// A <- (A + A^*) / 2, n x n
template <class C>
__global__ void k_herm(C* a, int64_t lda, int64_t sa, int n) {
    using R = typename RealOf<C>::T;
    const int t = blockIdx.y;
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= int64_t(n) * n) return;
    const int i = int(e % n), j = int(e / n);
    if (i < j) return;
    C* A = a + t * sa;
    const C x = A[i + j * lda], y = A[j + i * lda];
    const C hv = mkc<C>(R(0.5) * (x.x + y.x), R(0.5) * (x.y - y.y));
    A[i + j * lda] = hv;
    A[j + i * lda] = gconj(hv);
}
// zero the strict upper triangle of an n x n block
template <class C>
__global__ void k_zero_upper(C* a, int64_t lda, int64_t sa, int n) {
    const int t = blockIdx.y;
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= int64_t(n) * n) return;
    const int i = int(e % n), j = int(e / n);
    if (i < j) a[t * sa + i + j * lda] = czero<C>();
}
// identity n x n
template <class C>
__global__ void k_eye(C* a, int64_t lda, int64_t sa, int n) {
    const int t = blockIdx.y;
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= int64_t(n) * n) return;
    const int i = int(e % n), j = int(e / n);
    a[t * sa + i + j * lda] = mkc<C>(i == j ? 1 : 0, 0);
}
// Gaussian block (rows x cols per node)
template <class C>
__global__ void k_randn(C* a, int64_t sa, int rows, int cols, uint64_t seed) {
    const int t = blockIdx.y;
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= int64_t(rows) * cols) return;
    a[t * sa + e] = cvt<C>(hash_gauss(seed, uint64_t(t), uint64_t(e)));
}
// per node: max over columns of ||Y(:, j)||^2 (Y float2, m x s, column-major, ld), as ordered bits
__global__ void k_colnorm_max(const float2* Y, int64_t ld, int64_t sY, int m, int s, unsigned long long* out) {
    const int t = blockIdx.y;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= s) return;
    const float2* col = Y + t * sY + int64_t(warp) * ld;
    double a = 0.0;
    for (int i = lane; i < m; i += 32) a += double(col[i].x) * col[i].x + double(col[i].y) * col[i].y;
    a = warp_sum(a);
    if (lane == 0) atomicMax(out + t, (unsigned long long)__double_as_longlong(a));
}
__global__ void k_thr(const unsigned long long* mx, double tol, int nn, double* thr, double* thr2) {
    const int t = threadIdx.x;
    if (t >= nn) return;
    const double v = tol * sqrt(__longlong_as_double((long long)mx[t]));
    thr[t] = v;
    thr2[t] = v * v;
}

inline dim3 g2(int64_t elems, int batch) { return dim3(cdiv(std::max<int64_t>(elems, 1), TBD), unsigned(batch)); }

// ---------------------------------------------------------------- blocked drivers
// Cholesky A = L L^* (lower, in place; strict upper triangle zeroed), n x n per node.
template <class C>
fio_status potrf(C* A, int n, int64_t lda, int64_t sA, int batch, int* status, cudaStream_t st) {
    for (int j0 = 0; j0 < n; j0 += NB) {
        const int jb = std::min(NB, n - j0), j1 = j0 + jb;
        k_potrf_diag<C><<<batch, TBD, 0, st>>>(A, lda, sA, j0, jb, status);
        if (j1 < n) {
            k_trsm_rows<C, true><<<dim3(cdiv(n - j1, TBD), batch), TBD, 0, st>>>(A + j1 + j0 * lda, lda, sA, n - j1,
                                                                                 A + j0 + j0 * lda, lda, sA, jb);
            FIO_TRY(gemm<C>('N', 'C', n - j1, n - j1, jb, -1.0, A + j1 + j0 * lda, lda, sA, A + j1 + j0 * lda, lda, sA,
                            1.0, A + j1 + j1 * lda, lda, sA, batch, st));
        }
    }
    k_zero_upper<C><<<g2(int64_t(n) * n, batch), TBD, 0, st>>>(A, lda, sA, n);
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}
// X L^* = B in place (X: nrows x n), L n x n lower.
template <class C>
fio_status trsm_right_lh(C* X, int nrows, int n, int64_t ldx, int64_t sX, const C* L, int64_t ldl, int64_t sL, int batch,
                         cudaStream_t st) {
    for (int j0 = 0; j0 < n; j0 += NB) {
        const int jb = std::min(NB, n - j0);
        if (j0 > 0)
            FIO_TRY(gemm<C>('N', 'C', nrows, jb, j0, -1.0, X, ldx, sX, L + j0, ldl, sL, 1.0, X + j0 * ldx, ldx, sX, batch,
                            st));
        k_trsm_rows<C, true><<<dim3(cdiv(nrows, TBD), batch), TBD, 0, st>>>(X + j0 * ldx, ldx, sX, nrows,
                                                                             L + j0 + j0 * ldl, ldl, sL, jb);
    }
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}
// X L = B in place (X: nrows x n).
template <class C>
fio_status trsm_right_l(C* X, int nrows, int n, int64_t ldx, int64_t sX, const C* L, int64_t ldl, int64_t sL, int batch,
                        cudaStream_t st) {
    const int nblk = (n + NB - 1) / NB;
    for (int b = nblk - 1; b >= 0; --b) {
        const int j0 = b * NB, jb = std::min(NB, n - j0), j1 = j0 + jb;
        if (j1 < n)
            FIO_TRY(gemm<C>('N', 'N', nrows, jb, n - j1, -1.0, X + j1 * ldx, ldx, sX, L + j1 + j0 * ldl, ldl, sL, 1.0,
                            X + j0 * ldx, ldx, sX, batch, st));
        k_trsm_rows<C, false><<<dim3(cdiv(nrows, TBD), batch), TBD, 0, st>>>(X + j0 * ldx, ldx, sX, nrows,
                                                                              L + j0 + j0 * ldl, ldl, sL, jb);
    }
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}
// L X = B in place (X: n x ncols).
template <class C>
fio_status trsm_left_l(C* X, int n, int ncols, int64_t ldx, int64_t sX, const C* L, int64_t ldl, int64_t sL, int batch,
                       cudaStream_t st) {
    for (int j0 = 0; j0 < n; j0 += NB) {
        const int jb = std::min(NB, n - j0);
        if (j0 > 0)
            FIO_TRY(gemm<C>('N', 'N', jb, ncols, j0, -1.0, L + j0, ldl, sL, X, ldx, sX, 1.0, X + j0, ldx, sX, batch, st));
        k_trsm_cols<C><<<dim3(cdiv(ncols, TBD), batch), TBD, 0, st>>>(X + j0, ldx, sX, ncols, L + j0 + j0 * ldl, ldl, sL,
                                                                      jb);
    }
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}
// FP64 scratch of cholqr2's first pass (grown on demand; one per process, used on one
// stream at a time like the rest of a build or factorization).
DevBuf& chol64_scratch() {
    static DevBuf b;
    return b;
}

// M (m x r) <- orthonormal basis of range(M) by CholQR2; R (r x r, upper) with M_in = M_out R
// when R is given.  G, R2: r x r scratch per node (stride r*r).  The first pass forms
// and factors the Gram matrix in FP64 (a projected Gaussian block spans a subspace of
// its own width and can have condition ~r, squared in the Gram matrix); the second,
// on an almost orthonormal M, runs in C.
template <class C>
fio_status cholqr2(C* M, int m, int r, int64_t sM, C* G, C* R, C* R2, int batch, int* status, cudaStream_t st) {
    const int64_t sG = int64_t(r) * r;
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 0 && !std::is_same<C, z>::value) {
            const int64_t mr = int64_t(m) * r;
            DevBuf& b = chol64_scratch();
            FIO_TRY(b.ensure(size_t(batch) * (mr + sG) * 16));
            z* M64 = b.as<z>();
            z* G64 = M64 + batch * mr;
            k_cvt<C, z><<<g2(mr, batch), TBD, 0, st>>>(M, m, sM, M64, m, mr, m, r);
            FIO_TRY(gemm<z>('C', 'N', r, r, m, 1.0, M64, m, mr, M64, m, mr, 0.0, G64, r, sG, batch, st));
            FIO_TRY(potrf<z>(G64, r, r, sG, batch, status, st));
            k_cvt<z, C><<<g2(sG, batch), TBD, 0, st>>>(G64, r, sG, G, r, sG, r, r);
        } else {
            FIO_TRY(gemm<C>('C', 'N', r, r, m, 1.0, M, m, sM, M, m, sM, 0.0, G, r, sG, batch, st));
            FIO_TRY(potrf<C>(G, r, r, sG, batch, status, st));
        }
        FIO_TRY(trsm_right_lh<C>(M, m, r, m, sM, G, r, sG, batch, st));
        if (R) {
            if (pass == 0) {   // R = L1^*
                k_conjT<C><<<g2(sG, batch), TBD, 0, st>>>(G, r, sG, R, r, sG, r, r);
            } else {           // R = L2^* L1^*
                FIO_TRY(gemm<C>('C', 'N', r, r, r, 1.0, G, r, sG, R, r, sG, 0.0, R2, r, sG, batch, st));
                FIO_CUDA(cudaMemcpyAsync(R, R2, size_t(batch) * sG * sizeof(C), cudaMemcpyDeviceToDevice, st));
            }
        }
    }
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}

}  // namespace dense

using namespace dense;

// Device scratch of the large-node routines, owned by the caller (one per build or
// factorization); buffers grow on demand and are freed with the object.
struct BigScratch {
    DevBuf Op, G, W, E, A, A64, GA, R, R2, dg, perm, rank, sat, done, thr, thr2, mx, M, T1, T2, status;
    DevBuf Q, T, Dc, Df, Bz, Pz, Upz, Li, L64;
    int lvl_m = 0, lvl_c = 0;   // node size and null-basis width of the last node pass
    bool lvl_f64 = false;       // precision of the last node pass
    void release() {
        for (DevBuf* b : {&Op, &G, &W, &E, &A, &A64, &GA, &R, &R2, &dg, &perm, &rank, &sat, &done, &thr, &thr2, &mx, &M,
                          &T1, &T2, &status, &Q, &T, &Dc, &Df, &Bz, &Pz, &Upz, &Li, &L64})
            b->release();
    }
};
BigScratch* big_scratch_new() { return new BigScratch(); }
void big_scratch_free(BigScratch* b) {
    if (!b) return;
    b->release();
    delete b;
}

int g_large_max_nodes = 16;
void set_large_node_min(int m) { g_large_min = m; }
bool large_level(int nodes, int m) { return nodes <= g_large_max_nodes && m >= g_large_min; }

// Node pass of a large level: per node t, Omega^+ and W = Y Omega^+, the null basis
// Gamma, A = Y Gamma (in C) and the pivoted Cholesky of A^* A (FP64, at most `rhat`
// steps); the rank is the number of pivots above thr^2.  khat / sat to host.
template <class C>
fio_status level_nodes_t(BigScratch& w, int nn, int m, int s, int rhat, const float2* Om_f, const float2* Y_f, int64_t ldf,
                         double tol, std::vector<int>& hk, std::vector<int>& hs, cudaStream_t st) {
    constexpr bool F64 = std::is_same<C, z>::value;
    const int nc = s - m;
    const int64_t ms = int64_t(m) * s, mm = int64_t(m) * m, sc = int64_t(s) * nc, mc = int64_t(m) * nc,
                  cc = int64_t(nc) * nc;
    const size_t es = sizeof(C);
    FIO_TRY(w.Op.ensure(size_t(nn) * ms * es));     // Omega^+ (s x m)
    FIO_TRY(w.G.ensure(size_t(nn) * std::max(mm, cc) * es));
    FIO_TRY(w.W.ensure(size_t(nn) * mm * es));
    FIO_TRY(w.E.ensure(size_t(nn) * std::max<int64_t>(sc, 1) * es));   // E -> Gamma (s x c)
    FIO_TRY(w.A.ensure(size_t(nn) * std::max<int64_t>(mc, 1) * es));   // Omega E (m x c), then A = Y Gamma
    if (!F64) FIO_TRY(w.A64.ensure(size_t(nn) * std::max<int64_t>(mc, 1) * 16));
    FIO_TRY(w.GA.ensure(size_t(nn) * std::max<int64_t>(cc, 1) * 16));   // A^* A (FP64)
    FIO_TRY(w.dg.ensure(size_t(nn) * std::max(nc, 1) * 8));
    FIO_TRY(w.perm.ensure(size_t(nn) * std::max(nc, 1) * 4));
    FIO_TRY(w.rank.ensure(size_t(nn) * 4));
    FIO_TRY(w.sat.ensure(size_t(nn) * 4));
    FIO_TRY(w.done.ensure(size_t(nn) * 4));
    FIO_TRY(w.thr.ensure(size_t(nn) * 8));
    FIO_TRY(w.thr2.ensure(size_t(nn) * 8));
    FIO_TRY(w.mx.ensure(size_t(nn) * 8));
    FIO_TRY(w.status.ensure(4));
    // the samples as node blocks: the ld-strided FP32 input itself, or FP64 copies
    const C* Om;
    const C* Y;
    int64_t ld, sO;
    if constexpr (F64) {
        FIO_TRY(w.Q.ensure(size_t(2 * nn) * ms * 16));
        z* Oz = w.Q.as<z>();
        k_cvt<c, z><<<g2(ms, nn), TBD, 0, st>>>(Om_f, ldf, m, Oz, m, ms, m, s);
        k_cvt<c, z><<<g2(ms, nn), TBD, 0, st>>>(Y_f, ldf, m, Oz + nn * ms, m, ms, m, s);
        Om = Oz;
        Y = Oz + nn * ms;
        ld = m;
        sO = ms;
    } else {
        Om = Om_f;
        Y = Y_f;
        ld = ldf;
        sO = m;
    }
    C* G = w.G.as<C>();
    C* W = w.W.as<C>();
    C* Op = w.Op.as<C>();
    C* E = w.E.as<C>();
    C* A = w.A.as<C>();
    z* A64 = F64 ? w.A.as<z>() : w.A64.as<z>();
    z* GA = w.GA.as<z>();
    int* status = w.status.as<int>();
    w.lvl_m = m;
    w.lvl_c = nc;
    w.lvl_f64 = F64;
    FIO_CUDA(cudaMemsetAsync(status, 0, 4, st));
    FIO_CUDA(cudaMemsetAsync(w.mx.p, 0, size_t(nn) * 8, st));
    k_colnorm_max<<<dim3(cdiv(int64_t(s) * 32, TBD), nn), TBD, 0, st>>>(Y_f, ldf, m, m, s, w.mx.as<unsigned long long>());
    k_thr<<<1, 32, 0, st>>>(w.mx.as<unsigned long long>(), tol, nn, w.thr.as<double>(), w.thr2.as<double>());
    // G = Omega Omega^* = L L^*;  Omega^+ = Omega^* G^{-1};  W = Y Omega^+
    FIO_TRY(gemm<C>('N', 'C', m, m, s, 1.0, Om, ld, sO, Om, ld, sO, 0.0, G, m, mm, nn, st));
    FIO_TRY(potrf<C>(G, m, m, mm, nn, status, st));
    k_conjT<C><<<g2(ms, nn), TBD, 0, st>>>(Om, ld, sO, Op, s, ms, m, s);
    FIO_TRY(trsm_right_lh<C>(Op, s, m, s, ms, G, m, mm, nn, st));
    FIO_TRY(trsm_right_l<C>(Op, s, m, s, ms, G, m, mm, nn, st));
    FIO_TRY(gemm<C>('N', 'N', m, m, s, 1.0, Y, ld, sO, Op, s, ms, 0.0, W, m, mm, nn, st));
    if (nc > 0) {
        // Gamma: (I - Omega^+ Omega) E, twice, then CholQR2
        k_randn<C><<<g2(sc, nn), TBD, 0, st>>>(E, sc, s, nc, 0x9a77a5eedull + uint64_t(m) * 131 + s);
        for (int pass = 0; pass < 2; ++pass) {
            FIO_TRY(gemm<C>('N', 'N', m, nc, s, 1.0, Om, ld, sO, E, s, sc, 0.0, A, m, mc, nn, st));
            FIO_TRY(gemm<C>('N', 'N', s, nc, m, -1.0, Op, s, ms, A, m, mc, 1.0, E, s, sc, nn, st));
        }
        FIO_TRY(cholqr2<C>(E, s, nc, sc, G, nullptr, nullptr, nn, status, st));
        // A = Y Gamma, GA = A^* A (FP64)
        FIO_TRY(gemm<C>('N', 'N', m, nc, s, 1.0, Y, ld, sO, E, s, sc, 0.0, A, m, mc, nn, st));
        if (!F64) k_cvt<C, z><<<g2(mc, nn), TBD, 0, st>>>(A, m, mc, A64, m, mc, m, nc);
        FIO_TRY(gemm<z>('C', 'N', nc, nc, m, 1.0, A64, m, mc, A64, m, mc, 0.0, GA, nc, cc, nn, st));
        const int maxk = std::min(rhat, nc);
        k_pstrf_init<<<dim3(cdiv(nc, TBD), nn), TBD, 0, st>>>(GA, nc, cc, nc, w.dg.as<double>(), w.perm.as<int>(),
                                                              w.done.as<int>());
        for (int j0 = 0; j0 < maxk; j0 += NB) {
            const int j1 = std::min(maxk, j0 + NB);
            k_pstrf_panel<<<nn, TBD, 0, st>>>(GA, nc, cc, nc, j0, j1, maxk, w.thr2.as<double>(), w.dg.as<double>(),
                                              w.perm.as<int>(), w.rank.as<int>(), w.sat.as<int>(), w.done.as<int>());
            if (j1 < nc)   // trailing update (harmless for nodes that stopped)
                FIO_TRY(gemm<z>('N', 'C', nc - j1, nc - j1, j1 - j0, -1.0, GA + j1 + int64_t(j0) * nc, nc, cc,
                                GA + j1 + int64_t(j0) * nc, nc, cc, 1.0, GA + j1 + int64_t(j1) * nc, nc, cc, nn, st));
        }
        k_pstrf_finish<<<nn, TBD, 0, st>>>(nc, maxk, w.thr2.as<double>(), w.dg.as<double>(), w.rank.as<int>(),
                                           w.sat.as<int>(), w.done.as<int>());
    } else {
        FIO_CUDA(cudaMemsetAsync(w.rank.p, 0, size_t(nn) * 4, st));
        FIO_CUDA(cudaMemsetAsync(w.sat.p, 0, size_t(nn) * 4, st));
    }
    FIO_CUDA(cudaGetLastError());
    hk.resize(nn);
    hs.resize(nn);
    int hst = 0;
    FIO_CUDA(cudaMemcpyAsync(hk.data(), w.rank.p, size_t(nn) * 4, cudaMemcpyDeviceToHost, st));
    FIO_CUDA(cudaMemcpyAsync(hs.data(), w.sat.p, size_t(nn) * 4, cudaMemcpyDeviceToHost, st));
    FIO_CUDA(cudaMemcpyAsync(&hst, status, 4, cudaMemcpyDeviceToHost, st));
    FIO_CUDA(cudaStreamSynchronize(st));
    if (hst) return fail(FIO_ENOTHPD, "hss_build_from_samples: a Gram matrix of the node pass (Omega_tau Omega_tau^* "
                                      "or the null basis) is not positive definite");
    return FIO_OK;
}

fio_status big_level_nodes(BigScratch& w, int nn, int m, int s, int rhat, const float2* Om, const float2* Y, int64_t ld,
                           double tol, std::vector<int>& hk, std::vector<int>& hs, cudaStream_t st) {
    return tol >= kFp32Tol ? level_nodes_t<c>(w, nn, m, s, rhat, Om, Y, ld, tol, hk, hs, st)
                           : level_nodes_t<z>(w, nn, m, s, rhat, Om, Y, ld, tol, hk, hs, st);
}

// Finishing pass (in the node pass's precision): U (nn x m x rl) from the leading rl pivot
// columns (CholQR2), and D-check (nn x m x m): X = (I - U U^*) W, D = X + U U^* X^*.
template <class C>
fio_status level_finish_t(BigScratch& w, int nn, int m, int rl, float2* Uout, float2* Dchk, cudaStream_t st) {
    const int64_t mm = int64_t(m) * m, mr = int64_t(m) * std::max(rl, 1), rr = int64_t(std::max(rl, 1)) * std::max(rl, 1);
    const size_t es = sizeof(C);
    C* W = w.W.as<C>();
    int* status = w.status.as<int>();
    if (rl > 0) {
        FIO_TRY(w.M.ensure(size_t(nn) * mr * es));
        FIO_TRY(w.R.ensure(size_t(nn) * rr * es));
        FIO_TRY(w.T1.ensure(size_t(nn) * mr * es));
        FIO_TRY(w.T2.ensure(size_t(nn) * mr * es));
        C* M = w.M.as<C>();
        k_gather_cols<C><<<g2(int64_t(m) * rl, nn), TBD, 0, st>>>(w.A.as<C>(), m, int64_t(m) * w.lvl_c, w.lvl_c,
                                                                  w.perm.as<int>(), w.rank.as<int>(), rl, M, mr,
                                                                  0xb4515ull + uint64_t(m) * 7 + rl);
        FIO_TRY(cholqr2<C>(M, m, rl, mr, w.R.as<C>(), nullptr, nullptr, nn, status, st));
        k_cvt<C, c><<<g2(mr, nn), TBD, 0, st>>>(M, m, mr, Uout, m, mr, m, rl);
        // T1 = U^* W (rl x m); W <- X = W - U T1; T2 = X U (m x rl); X <- X + U T2^*
        C* T1 = w.T1.as<C>();
        C* T2 = w.T2.as<C>();
        FIO_TRY(gemm<C>('C', 'N', rl, m, m, 1.0, M, m, mr, W, m, mm, 0.0, T1, rl, mr, nn, st));
        FIO_TRY(gemm<C>('N', 'N', m, m, rl, -1.0, M, m, mr, T1, rl, mr, 1.0, W, m, mm, nn, st));
        FIO_TRY(gemm<C>('N', 'N', m, rl, m, 1.0, W, m, mm, M, m, mr, 0.0, T2, m, mr, nn, st));
        FIO_TRY(gemm<C>('N', 'C', m, m, rl, 1.0, M, m, mr, T2, m, mr, 1.0, W, m, mm, nn, st));
    }
    k_cvt<C, c><<<g2(mm, nn), TBD, 0, st>>>(W, m, mm, Dchk, m, mm, m, m);
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}

fio_status big_level_finish(BigScratch& w, int nn, int m, int rl, float2* Uout, float2* Dchk, cudaStream_t st) {
    return w.lvl_f64 ? level_finish_t<z>(w, nn, m, rl, Uout, Dchk, st) : level_finish_t<c>(w, nn, m, rl, Uout, Dchk, st);
}

// Root of the construction (FP64: the sample block is m0 x (m0 + p), nearly square):
// D0 = Herm(Y Omega^+) (double2, m0 x m0), Omega / Y: m0 x s0 float2.
fio_status big_root(BigScratch& w, int m0, int s0, const float2* Om, const float2* Y, double2* D0, cudaStream_t st) {
    const int64_t ms = int64_t(m0) * s0, mm = int64_t(m0) * m0;
    FIO_TRY(w.A64.ensure(size_t(2 * ms) * 16));
    FIO_TRY(w.GA.ensure(size_t(mm) * 16));
    FIO_TRY(w.status.ensure(4));
    int* status = w.status.as<int>();
    FIO_CUDA(cudaMemsetAsync(status, 0, 4, st));
    z* Oz = w.A64.as<z>();
    z* Yz = Oz + ms;
    z* G = w.GA.as<z>();
    k_cvt<c, z><<<g2(ms, 1), TBD, 0, st>>>(Om, m0, 0, Oz, m0, 0, m0, s0);
    k_cvt<c, z><<<g2(ms, 1), TBD, 0, st>>>(Y, m0, 0, Yz, m0, 0, m0, s0);
    FIO_TRY(gemm<z>('N', 'C', m0, m0, s0, 1.0, Oz, m0, 0, Oz, m0, 0, 0.0, G, m0, 0, 1, st));
    FIO_TRY(gemm<z>('N', 'C', m0, m0, s0, 1.0, Yz, m0, 0, Oz, m0, 0, 0.0, D0, m0, 0, 1, st));
    FIO_TRY(potrf<z>(G, m0, m0, 0, 1, status, st));
    FIO_TRY(trsm_right_lh<z>(D0, m0, m0, m0, 0, G, m0, 0, 1, st));
    FIO_TRY(trsm_right_l<z>(D0, m0, m0, m0, 0, G, m0, 0, 1, st));
    k_herm<z><<<g2(mm, 1), TBD, 0, st>>>(D0, m0, 0, m0);
    int hst = 0;
    FIO_CUDA(cudaMemcpyAsync(&hst, status, 4, cudaMemcpyDeviceToHost, st));
    FIO_CUDA(cudaStreamSynchronize(st));
    if (hst) return fail(FIO_ENOTHPD, "hss_build_from_samples: root Omega Omega^* not positive definite");
    return FIO_OK;
}

// Postprocessing of level l (Section 3.3): for each parent t (Dcur: nn blocks 2rc x 2rc,
// FP64), B_t = Herm(D_t)[rc:, :rc]; child a = 2t + ch: Dnext_a = Dchk_a + U_a H_cc U_a^*
// (products in FP32, accumulated into the FP64 blocks).
fio_status big_post(BigScratch& w, int nn, int rc, int mc, double2* Dcur, const float2* Uc, const float2* Dchk,
                    float2* Bout, double2* Dnext, cudaStream_t st) {
    const int mt = 2 * rc;
    const int64_t st_t = int64_t(mt) * mt, mr = int64_t(mc) * rc, mcc = int64_t(mc) * mc, rr = int64_t(rc) * rc;
    k_cvt<c, z><<<g2(mcc, 2 * nn), TBD, 0, st>>>(Dchk, mc, mcc, Dnext, mc, mcc, mc, mc);
    if (rc == 0) {
        FIO_CUDA(cudaGetLastError());
        return FIO_OK;
    }
    FIO_TRY(w.M.ensure(size_t(2 * nn) * rr * 8));   // H_cc (FP32)
    FIO_TRY(w.T1.ensure(size_t(2 * nn) * mr * 8));
    FIO_TRY(w.T2.ensure(size_t(2 * nn) * mcc * 8));
    k_herm<z><<<g2(st_t, nn), TBD, 0, st>>>(Dcur, mt, st_t, mt);
    k_cvt<z, c><<<g2(rr, nn), TBD, 0, st>>>(Dcur + rc, mt, st_t, Bout, rc, rr, rc, rc);
    c* H = w.M.as<c>();
    c* T = w.T1.as<c>();
    c* Dt = w.T2.as<c>();
    for (int ch = 0; ch < 2; ++ch)   // H of child 2t + ch at H + (2t + ch) rr
        k_cvt<z, c><<<g2(rr, nn), TBD, 0, st>>>(Dcur + ch * rc + int64_t(ch * rc) * mt, mt, st_t, H + ch * rr, rc, 2 * rr,
                                                 rc, rc);
    FIO_TRY(gemm<c>('N', 'N', mc, rc, rc, 1.0, Uc, mc, mr, H, rc, rr, 0.0, T, mc, mr, 2 * nn, st));
    FIO_TRY(gemm<c>('N', 'C', mc, mc, rc, 1.0, T, mc, mr, Uc, mc, mr, 0.0, Dt, mc, mcc, 2 * nn, st));
    k_acc<<<g2(mcc, 2 * nn), TBD, 0, st>>>(Dt, mc, mcc, Dnext, mc, mcc, mc, mc);
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}

// ULV node factorization of a large level: D (nn x m x m), U (nn x m x r), FP64 inputs ->
// W (float2 nn x m x m), Dh22 and Uh2 (double2 nn x r x r).  Products in FP32; the
// Cholesky factorization of the eliminated block D-check_11 in FP64.
fio_status big_ulv_nodes(BigScratch& b, int nn, int m, int r, const double2* D, const double2* U, float2* Wout,
                         double2* Dh22, double2* Uh2, int* d_status, cudaStream_t st) {
    const int n1 = m - r;
    const int64_t mm = int64_t(m) * m, rr = int64_t(std::max(r, 1)) * std::max(r, 1);
    const int64_t n1n1 = int64_t(std::max(n1, 1)) * std::max(n1, 1);
    FIO_TRY(b.Q.ensure(size_t(nn) * mm * 8));
    FIO_TRY(b.T.ensure(size_t(nn) * mm * 8));
    FIO_TRY(b.Dc.ensure(size_t(nn) * mm * 8));
    FIO_TRY(b.Df.ensure(size_t(nn) * mm * 8));
    FIO_TRY(b.G.ensure(size_t(nn) * std::max(rr, n1n1) * 8));
    FIO_TRY(b.R.ensure(size_t(nn) * rr * 8));
    FIO_TRY(b.R2.ensure(size_t(nn) * rr * 8));
    FIO_TRY(b.L64.ensure(size_t(nn) * n1n1 * 16));
    c* Q = b.Q.as<c>();     // [Q1 | Q2]
    c* T = b.T.as<c>();
    c* Dc = b.Dc.as<c>();
    c* Df = b.Df.as<c>();
    c* Q2 = Q + int64_t(n1) * m;
    k_cvt<z, c><<<g2(mm, nn), TBD, 0, st>>>(D, m, mm, Df, m, mm, m, m);
    if (r > 0) {
        // Q2 R = U (CholQR2)
        k_cvt<z, c><<<g2(int64_t(m) * r, nn), TBD, 0, st>>>(U, m, int64_t(m) * r, Q2, m, mm, m, r);
        FIO_TRY(cholqr2<c>(Q2, m, r, mm, b.G.as<c>(), b.R.as<c>(), b.R2.as<c>(), nn, d_status, st));
        k_cvt<c, z><<<g2(rr, nn), TBD, 0, st>>>(b.R.as<c>(), r, rr, Uh2, r, rr, r, r);
    }
    if (n1 > 0) {
        // Q1 = orth((I - Q2 Q2^*) E), E Gaussian m x n1
        k_randn<c><<<g2(int64_t(m) * n1, nn), TBD, 0, st>>>(Q, mm, m, n1, 0x5eedull + uint64_t(m) * 977 + r);
        if (r > 0) {
            FIO_TRY(b.E.ensure(size_t(nn) * int64_t(r) * n1 * 8));
            c* P = b.E.as<c>();
            const int64_t rn = int64_t(r) * n1;
            for (int pass = 0; pass < 2; ++pass) {   // project twice against range(Q2)
                FIO_TRY(gemm<c>('C', 'N', r, n1, m, 1.0, Q2, m, mm, Q, m, mm, 0.0, P, r, rn, nn, st));
                FIO_TRY(gemm<c>('N', 'N', m, n1, r, -1.0, Q2, m, mm, P, r, rn, 1.0, Q, m, mm, nn, st));
            }
        }
        FIO_TRY(cholqr2<c>(Q, m, n1, mm, b.G.as<c>(), nullptr, nullptr, nn, d_status, st));
    }
    // D-check = Q^* D Q
    FIO_TRY(gemm<c>('N', 'N', m, m, m, 1.0, Df, m, mm, Q, m, mm, 0.0, T, m, mm, nn, st));
    FIO_TRY(gemm<c>('C', 'N', m, m, m, 1.0, Q, m, mm, T, m, mm, 0.0, Dc, m, mm, nn, st));
    k_herm<c><<<g2(mm, nn), TBD, 0, st>>>(Dc, m, mm, m);
    c* A1 = T;   // reuse: A1 (n1 x m) at T, Q2^* (r x m) below it -> W (m x m) column-major
    if (n1 > 0) {
        // L11 = chol(D-check_11) in FP64, used in FP32 below
        z* L64 = b.L64.as<z>();
        k_cvt<c, z><<<g2(n1n1, nn), TBD, 0, st>>>(Dc, m, mm, L64, n1, n1n1, n1, n1);
        FIO_TRY(potrf<z>(L64, n1, n1, n1n1, nn, d_status, st));
        k_cvt<z, c><<<g2(n1n1, nn), TBD, 0, st>>>(L64, n1, n1n1, Dc, m, mm, n1, n1);
        if (r > 0) FIO_TRY(trsm_right_lh<c>(Dc + n1, r, n1, m, mm, Dc, m, mm, nn, st));   // D^_21 = D-check_21 L11^{-*}
        // A1 = L11^{-1} Q1^*  (n1 x m, rows 0..n1-1 of T)
        k_conjT<c><<<g2(int64_t(m) * n1, nn), TBD, 0, st>>>(Q, m, mm, A1, m, mm, m, n1);
        FIO_TRY(trsm_left_l<c>(A1, n1, m, m, mm, Dc, m, mm, nn, st));
    }
    if (r > 0) {
        // D^_22 = D-check_22 - D^_21 D^_21^*
        if (n1 > 0)
            FIO_TRY(gemm<c>('N', 'C', r, r, n1, -1.0, Dc + n1, m, mm, Dc + n1, m, mm, 1.0, Dc + n1 + int64_t(n1) * m, m, mm,
                            nn, st));
        k_cvt<c, z><<<g2(rr, nn), TBD, 0, st>>>(Dc + n1 + int64_t(n1) * m, m, mm, Dh22, r, rr, r, r);
        // rows n1..m-1 of W: Q2^* - D^_21 A1
        k_conjT<c><<<g2(int64_t(m) * r, nn), TBD, 0, st>>>(Q2, m, mm, T + n1, m, mm, m, r);
        if (n1 > 0)
            FIO_TRY(gemm<c>('N', 'N', r, m, n1, -1.0, Dc + n1, m, mm, A1, m, mm, 1.0, T + n1, m, mm, nn, st));
    }
    FIO_CUDA(cudaMemcpyAsync(Wout, T, size_t(nn) * mm * 8, cudaMemcpyDeviceToDevice, st));
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}

// Merge (Eq. 2.12), FP64 (r x r products): parents t = 0..np-1, children 2t, 2t+1 of rank r;
// D+ (2r x 2r) = [[D1, U1 B^* U2^*], [U2 B U1^*, D2]], U+ = [U1 Up_top; U2 Up_bot].
// Merge into the parents (Eq. 2.12), every level and precision: D+ = [D^_22(1), (U2 B U1^*)^*; U2 B U1^*,
// D^_22(2)] and U+ = [U^_1 0; 0 U^_2] U_p, the off-diagonal block and U+ as batched GEMMs over the
// np parents (T = B U1^*, then U2 T).
template <class C>
fio_status ulv_merge_gemm(BigScratch& b, int np, int r, const C* Dh22, const C* Uh2, const float2* B, const float2* Up,
                          int rp, C* Dplus, C* Uplus, cudaStream_t st) {
    const int m = 2 * r;
    const int64_t rr = int64_t(r) * r, mm = int64_t(m) * m;
    const size_t es = sizeof(C);
    FIO_TRY(b.Bz.ensure(std::max<size_t>(16, size_t(np) * rr * es)));
    FIO_TRY(b.Pz.ensure(std::max<size_t>(16, size_t(np) * rr * es)));
    C* Bz = b.Bz.as<C>();
    C* T = b.Pz.as<C>();
    k_cvt<c, C><<<g2(rr, np), TBD, 0, st>>>(B, r, rr, Bz, r, rr, r, r);
    const C* U1 = Uh2;
    const C* U2 = Uh2 + rr;
    // T = B U1^*; lower-left = U2 T
    FIO_TRY(gemm<C>('N', 'C', r, r, r, 1.0, Bz, r, rr, U1, r, 2 * rr, 0.0, T, r, rr, np, st));
    FIO_TRY(gemm<C>('N', 'N', r, r, r, 1.0, U2, r, 2 * rr, T, r, rr, 0.0, Dplus + r, m, mm, np, st));
    k_conjT<C><<<g2(rr, np), TBD, 0, st>>>(Dplus + r, m, mm, Dplus + int64_t(r) * m, m, mm, r, r);
    k_cvt<C, C><<<g2(rr, np), TBD, 0, st>>>(Dh22, r, 2 * rr, Dplus, m, mm, r, r);
    k_cvt<C, C><<<g2(rr, np), TBD, 0, st>>>(Dh22 + rr, r, 2 * rr, Dplus + r + int64_t(r) * m, m, mm, r, r);
    if (Up && rp > 0) {
        const int64_t mr = int64_t(m) * rp;
        FIO_TRY(b.Upz.ensure(size_t(np) * mr * es));
        C* Upz = b.Upz.as<C>();
        k_cvt<c, C><<<g2(mr, np), TBD, 0, st>>>(Up, m, mr, Upz, m, mr, m, rp);
        FIO_TRY(gemm<C>('N', 'N', r, rp, r, 1.0, U1, r, 2 * rr, Upz, m, mr, 0.0, Uplus, m, mr, np, st));
        FIO_TRY(gemm<C>('N', 'N', r, rp, r, 1.0, U2, r, 2 * rr, Upz + r, m, mr, 0.0, Uplus + r, m, mr, np, st));
    }
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}
template fio_status ulv_merge_gemm<float2>(BigScratch&, int, int, const float2*, const float2*, const float2*,
                                           const float2*, int, float2*, float2*, cudaStream_t);
template fio_status ulv_merge_gemm<double2>(BigScratch&, int, int, const double2*, const double2*, const float2*,
                                            const float2*, int, double2*, double2*, cudaStream_t);

// Root: D+ = L L^* (FP64), Rinv = L^{-*} L^{-1} (triangular inverse and product in FP32).
fio_status big_ulv_root(BigScratch& b, int m0, const double2* Dp, float2* Rinv, int* d_status, cudaStream_t st) {
    const int64_t mm = int64_t(m0) * m0;
    FIO_TRY(b.L64.ensure(size_t(mm) * 16));
    FIO_TRY(b.Li.ensure(size_t(mm) * 8));
    FIO_TRY(b.Q.ensure(size_t(mm) * 8));
    z* L = b.L64.as<z>();
    c* Lf = b.Q.as<c>();
    c* Li = b.Li.as<c>();
    k_cvt<z, z><<<g2(mm, 1), TBD, 0, st>>>(Dp, m0, 0, L, m0, 0, m0, m0);
    FIO_TRY(potrf<z>(L, m0, m0, 0, 1, d_status, st));
    k_cvt<z, c><<<g2(mm, 1), TBD, 0, st>>>(L, m0, 0, Lf, m0, 0, m0, m0);
    k_eye<c><<<g2(mm, 1), TBD, 0, st>>>(Li, m0, 0, m0);
    FIO_TRY(trsm_left_l<c>(Li, m0, m0, m0, 0, Lf, m0, 0, 1, st));
    FIO_TRY(gemm<c>('C', 'N', m0, m0, m0, 1.0, Li, m0, 0, Li, m0, 0, 0.0, Rinv, m0, 0, 1, st));
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}

}  // namespace fio

extern "C" fio_status fio_set_large_node_count(int max_nodes) {
    if (max_nodes < 1) return fio::fail(FIO_EINVAL, "fio_set_large_node_count: max_nodes must be >= 1");
    fio::g_large_max_nodes = max_nodes;
    return FIO_OK;
}

extern "C" fio_status fio_set_large_node(int m_min) {
    if (m_min < 1) return fio::fail(FIO_EINVAL, "fio_set_large_node: m_min must be >= 1");
    fio::set_large_node_min(m_min);
    return FIO_OK;
}
