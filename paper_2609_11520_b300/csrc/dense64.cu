// Large HSS nodes (levels with few nodes of size m in the hundreds to
// thousands, as in 2D where the ranks grow like sqrt(N)): FP64 complex
// level-3 formulations of the per-node steps of Section 3.1-3.3 and of the
// ULV factorization (Section 2.4), batched over the nodes of a level.
//
// The one-CTA-per-node kernels apply Householder reflectors one at a time,
// which streams O(m^2 r) data through one SM.  Here every step is a sequence
// of batched GEMMs (cuBLAS ZGEMM, strided batched) and small blocked
// factorizations (one CTA per node and diagonal block):
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
#include <cublas_v2.h>

#include <mutex>
#include <string>

#include "cplx.cuh"
#include "hss.cuh"

namespace fio {
namespace dense {

using z = double2;
constexpr int NB = 32;     // block size of the blocked factorizations
constexpr int TBD = 256;

int g_large_min = 384;

// ---------------------------------------------------------------- cuBLAS
fio_status blas(cublasHandle_t* out, cudaStream_t st) {
    static std::mutex mu;
    static cublasHandle_t hs[64] = {};
    int dev = 0;
    FIO_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(FIO_EINVAL, "cuBLAS: device index out of range");
    std::lock_guard<std::mutex> lock(mu);
    if (!hs[dev] && cublasCreate(&hs[dev]) != CUBLAS_STATUS_SUCCESS) return fail(FIO_ECUDA, "cublasCreate failed");
    if (cublasSetStream(hs[dev], st) != CUBLAS_STATUS_SUCCESS) return fail(FIO_ECUDA, "cublasSetStream failed");
    *out = hs[dev];
    return FIO_OK;
}

// C = alpha op(A) op(B) + beta C for `batch` nodes (element strides sA, sB, sC); op: 'N' or 'C'.
fio_status zgemm(char ta, char tb, int m, int n, int k, z alpha, const z* A, int64_t lda, int64_t sA, const z* B,
                 int64_t ldb, int64_t sB, z beta, z* C, int64_t ldc, int64_t sC, int batch, cudaStream_t st) {
    if (m <= 0 || n <= 0 || batch <= 0) return FIO_OK;
    cublasHandle_t h;
    FIO_TRY(blas(&h, st));
    const cuDoubleComplex al = make_cuDoubleComplex(alpha.x, alpha.y), be = make_cuDoubleComplex(beta.x, beta.y);
    const cublasOperation_t oa = ta == 'C' ? CUBLAS_OP_C : CUBLAS_OP_N, ob = tb == 'C' ? CUBLAS_OP_C : CUBLAS_OP_N;
    cublasStatus_t s = cublasZgemmStridedBatched(
        h, oa, ob, m, n, std::max(k, 0), &al, reinterpret_cast<const cuDoubleComplex*>(A), int(lda), sA,
        reinterpret_cast<const cuDoubleComplex*>(B), int(ldb), sB, &be, reinterpret_cast<cuDoubleComplex*>(C), int(ldc),
        sC, batch);
    if (s != CUBLAS_STATUS_SUCCESS) return fail(FIO_ECUDA, "cublasZgemmStridedBatched failed (" + std::to_string(int(s)) + ")");
    return FIO_OK;
}
const z ONE = {1.0, 0.0}, MONE = {-1.0, 0.0}, ZERO = {0.0, 0.0};

// ---------------------------------------------------------------- kernels
// Cholesky of the jb x jb diagonal block at (j0, j0), lower, in place; one CTA per node.
__global__ void k_potrf_diag(z* A, int64_t lda, int64_t sA, int j0, int jb, int* status) {
    __shared__ z L[NB][NB + 1];
    z* At = A + blockIdx.x * sA + j0 + j0 * lda;
    for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) L[e % jb][e / jb] = At[e % jb + (e / jb) * lda];
    __syncthreads();
    for (int c = 0; c < jb; ++c) {
        if (threadIdx.x == 0) {
            double d = L[c][c].x;
            if (!(d > 0.0)) {
                atomicExch(status, FIO_ENOTHPD);
                d = 1.0;
            }
            L[c][c] = make_double2(sqrt(d), 0.0);
        }
        __syncthreads();
        const double inv = 1.0 / L[c][c].x;
        for (int i = c + 1 + threadIdx.x; i < jb; i += blockDim.x) L[i][c] = gscale(L[i][c], inv);
        __syncthreads();
        for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) {
            const int i = e % jb, j = e / jb;
            if (j > c && i >= j) L[i][j] = gsub(L[i][j], gmul(L[i][c], gconj(L[j][c])));
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) {
        const int i = e % jb, j = e / jb;
        At[i + j * lda] = i >= j ? L[i][j] : make_double2(0.0, 0.0);
    }
}

// Rows of X (nrows x jb, ld ldx) solve X L^* = B in place (FWD: L^* upper, forward over
// columns) or X L = B (backward over columns); L: jb x jb lower at Lm.
template <bool HERM>
__global__ void k_trsm_rows(z* X, int64_t ldx, int64_t sX, int nrows, const z* Lm, int64_t ldl, int64_t sL, int jb) {
    __shared__ z L[NB][NB + 1];
    const z* Lt = Lm + blockIdx.y * sL;
    for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) L[e % jb][e / jb] = Lt[e % jb + (e / jb) * ldl];
    __syncthreads();
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    z* x = X + blockIdx.y * sX + r;
    if (HERM) {   // sum_{q <= c} X[q] conj(L[c][q]) = B[c]
        for (int c = 0; c < jb; ++c) {
            z a = x[c * ldx];
            for (int q = 0; q < c; ++q) a = gsub(a, gmul(x[q * ldx], gconj(L[c][q])));
            x[c * ldx] = gscale(a, 1.0 / L[c][c].x);
        }
    } else {      // sum_{q >= c} X[q] L[q][c] = B[c]
        for (int c = jb - 1; c >= 0; --c) {
            z a = x[c * ldx];
            for (int q = c + 1; q < jb; ++q) a = gsub(a, gmul(x[q * ldx], L[q][c]));
            x[c * ldx] = gscale(a, 1.0 / L[c][c].x);
        }
    }
}

// Columns of X (jb x ncols, ld ldx) solve L X = B in place, L jb x jb lower.
__global__ void k_trsm_cols(z* X, int64_t ldx, int64_t sX, int ncols, const z* Lm, int64_t ldl, int64_t sL, int jb) {
    __shared__ z L[NB][NB + 1];
    const z* Lt = Lm + blockIdx.y * sL;
    for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) L[e % jb][e / jb] = Lt[e % jb + (e / jb) * ldl];
    __syncthreads();
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncols) return;
    z* x = X + blockIdx.y * sX + c * ldx;
    for (int i = 0; i < jb; ++i) {
        z a = x[i];
        for (int q = 0; q < i; ++q) a = gsub(a, gmul(L[i][q], x[q]));
        x[i] = gscale(a, 1.0 / L[i][i].x);
    }
}

// Pivoted Cholesky of a Hermitian n x n block (full storage), steps [j0, j1) of one
// panel, one CTA per node.  dg: updated diagonal; perm: row order; stops (done = 1,
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
    if (i == 0 && threadIdx.x == 0) done[t] = 0;
    if (i >= n) return;
    dg[int64_t(t) * n + i] = A[t * sA + i + int64_t(i) * lda].x;
    perm[int64_t(t) * n + i] = i;
}

// M[:, c] = A[:, perm[c]] for c < rank_t (the pivot columns), a Gaussian column beyond.
__global__ void k_gather_cols(const z* A, int m, int64_t sA, int c_all, const int* perm_all, const int* rank, int rl,
                              z* M, int64_t sM, uint64_t seed) {
    const int t = blockIdx.y;
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= int64_t(m) * rl) return;
    const int i = int(e % m), c = int(e / m);
    z v;
    if (c < rank[t]) {
        v = A[t * sA + i + int64_t(perm_all[int64_t(t) * c_all + c]) * m];
    } else {
        uint64_t x = seed ^ (uint64_t(t) << 40) ^ uint64_t(e) * 0x9e3779b97f4a7c15ull;
        auto nxt = [&]() {
            x += 0x9e3779b97f4a7c15ull;
            uint64_t y = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
            y = (y ^ (y >> 27)) * 0x94d049bb133111ebull;
            return y ^ (y >> 31);
        };
        const double u1 = (double(nxt() >> 11) + 1.0) * (1.0 / 9007199254740992.0);
        const double u2 = double(nxt() >> 11) * (1.0 / 9007199254740992.0);
        const double rr = sqrt(-2.0 * log(u1));
        double sn, cs;
        sincospi(2.0 * u2, &sn, &cs);
        v = make_double2(rr * cs, rr * sn);
    }
    M[t * sM + i + int64_t(c) * m] = v;
}

__global__ void k_f2_to_z(const float2* a, int64_t lda, int64_t sa, z* b, int64_t ldb, int64_t sb, int rows, int cols) {
    const int t = blockIdx.y;
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= int64_t(rows) * cols) return;
    const int i = int(e % rows), j = int(e / rows);
    const float2 v = a[t * sa + i + j * lda];
    b[t * sb + i + j * ldb] = make_double2(v.x, v.y);
}
__global__ void k_z_to_f2(const z* a, int64_t lda, int64_t sa, float2* b, int64_t ldb, int64_t sb, int rows, int cols) {
    const int t = blockIdx.y;
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= int64_t(rows) * cols) return;
    const int i = int(e % rows), j = int(e / rows);
    const z v = a[t * sa + i + j * lda];
    b[t * sb + i + j * ldb] = make_float2(float(v.x), float(v.y));
}
// B (cols x rows) = A^* (A rows x cols)
__global__ void k_conjT(const z* a, int64_t lda, int64_t sa, z* b, int64_t ldb, int64_t sb, int rows, int cols) {
    const int t = blockIdx.y;
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= int64_t(rows) * cols) return;
    const int i = int(e % rows), j = int(e / rows);
    b[t * sb + j + i * ldb] = gconj(a[t * sa + i + j * lda]);
}
__global__ void k_copy(const z* a, int64_t lda, int64_t sa, z* b, int64_t ldb, int64_t sb, int rows, int cols) {
    const int t = blockIdx.y;
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= int64_t(rows) * cols) return;
    const int i = int(e % rows), j = int(e / rows);
    b[t * sb + i + j * ldb] = a[t * sa + i + j * lda];
}
// A <- (A + A^*) / 2, n x n
__global__ void k_herm(z* a, int64_t lda, int64_t sa, int n) {
    const int t = blockIdx.y;
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= int64_t(n) * n) return;
    const int i = int(e % n), j = int(e / n);
    if (i < j) return;
    z* A = a + t * sa;
    const z x = A[i + j * lda], y = A[j + i * lda];
    const z h = make_double2(0.5 * (x.x + y.x), 0.5 * (x.y - y.y));
    A[i + j * lda] = h;
    A[j + i * lda] = gconj(h);
}
// zero the strict upper triangle of an n x n block
__global__ void k_zero_upper(z* a, int64_t lda, int64_t sa, int n) {
    const int t = blockIdx.y;
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= int64_t(n) * n) return;
    const int i = int(e % n), j = int(e / n);
    if (i < j) a[t * sa + i + j * lda] = make_double2(0.0, 0.0);
}
// identity n x n
__global__ void k_eye(z* a, int64_t lda, int64_t sa, int n) {
    const int t = blockIdx.y;
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= int64_t(n) * n) return;
    const int i = int(e % n), j = int(e / n);
    a[t * sa + i + j * lda] = make_double2(i == j ? 1.0 : 0.0, 0.0);
}
// Gaussian block (rows x cols per node) from a counter hash (splitmix64 + Box-Muller).
__global__ void k_randn(z* a, int64_t sa, int rows, int cols, uint64_t seed) {
    const int t = blockIdx.y;
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= int64_t(rows) * cols) return;
    auto mix = [](uint64_t x) {
        x += 0x9e3779b97f4a7c15ull;
        x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
        x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
        return x ^ (x >> 31);
    };
    const uint64_t h1 = mix(seed ^ mix(uint64_t(t) * 0x100000001b3ull + uint64_t(e) * 2));
    const uint64_t h2 = mix(h1 + 0x632be59bd9b4e019ull);
    const double u1 = (double(h1 >> 11) + 1.0) * (1.0 / 9007199254740992.0);
    const double u2 = double(h2 >> 11) * (1.0 / 9007199254740992.0);
    const double rr = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    a[t * sa + e] = make_double2(rr * cs, rr * sn);
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

inline dim3 g2(int64_t elems, int batch) { return dim3(cdiv(elems, TBD), unsigned(batch)); }

// ---------------------------------------------------------------- blocked drivers
// Cholesky A = L L^* (lower, in place; strict upper triangle zeroed), n x n per node.
fio_status potrf(z* A, int n, int64_t lda, int64_t sA, int batch, int* status, cudaStream_t st) {
    for (int j0 = 0; j0 < n; j0 += NB) {
        const int jb = std::min(NB, n - j0), j1 = j0 + jb;
        k_potrf_diag<<<batch, TBD, 0, st>>>(A, lda, sA, j0, jb, status);
        if (j1 < n) {
            k_trsm_rows<true><<<dim3(cdiv(n - j1, TBD), batch), TBD, 0, st>>>(A + j1 + j0 * lda, lda, sA, n - j1,
                                                                              A + j0 + j0 * lda, lda, sA, jb);
            FIO_TRY(zgemm('N', 'C', n - j1, n - j1, jb, MONE, A + j1 + j0 * lda, lda, sA, A + j1 + j0 * lda, lda, sA, ONE,
                          A + j1 + j1 * lda, lda, sA, batch, st));
        }
    }
    k_zero_upper<<<g2(int64_t(n) * n, batch), TBD, 0, st>>>(A, lda, sA, n);
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}
// X L^* = B in place (X: nrows x n), L n x n lower.
fio_status trsm_right_lh(z* X, int nrows, int n, int64_t ldx, int64_t sX, const z* L, int64_t ldl, int64_t sL, int batch,
                         cudaStream_t st) {
    for (int j0 = 0; j0 < n; j0 += NB) {
        const int jb = std::min(NB, n - j0);
        if (j0 > 0)
            FIO_TRY(zgemm('N', 'C', nrows, jb, j0, MONE, X, ldx, sX, L + j0, ldl, sL, ONE, X + j0 * ldx, ldx, sX, batch, st));
        k_trsm_rows<true><<<dim3(cdiv(nrows, TBD), batch), TBD, 0, st>>>(X + j0 * ldx, ldx, sX, nrows, L + j0 + j0 * ldl,
                                                                          ldl, sL, jb);
    }
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}
// X L = B in place (X: nrows x n).
fio_status trsm_right_l(z* X, int nrows, int n, int64_t ldx, int64_t sX, const z* L, int64_t ldl, int64_t sL, int batch,
                        cudaStream_t st) {
    const int nblk = (n + NB - 1) / NB;
    for (int b = nblk - 1; b >= 0; --b) {
        const int j0 = b * NB, jb = std::min(NB, n - j0), j1 = j0 + jb;
        if (j1 < n)
            FIO_TRY(zgemm('N', 'N', nrows, jb, n - j1, MONE, X + j1 * ldx, ldx, sX, L + j1 + j0 * ldl, ldl, sL, ONE,
                          X + j0 * ldx, ldx, sX, batch, st));
        k_trsm_rows<false><<<dim3(cdiv(nrows, TBD), batch), TBD, 0, st>>>(X + j0 * ldx, ldx, sX, nrows,
                                                                           L + j0 + j0 * ldl, ldl, sL, jb);
    }
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}
// L X = B in place (X: n x ncols).
fio_status trsm_left_l(z* X, int n, int ncols, int64_t ldx, int64_t sX, const z* L, int64_t ldl, int64_t sL, int batch,
                       cudaStream_t st) {
    for (int j0 = 0; j0 < n; j0 += NB) {
        const int jb = std::min(NB, n - j0);
        if (j0 > 0)
            FIO_TRY(zgemm('N', 'N', jb, ncols, j0, MONE, L + j0, ldl, sL, X, ldx, sX, ONE, X + j0, ldx, sX, batch, st));
        k_trsm_cols<<<dim3(cdiv(ncols, TBD), batch), TBD, 0, st>>>(X + j0, ldx, sX, ncols, L + j0 + j0 * ldl, ldl, sL, jb);
    }
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}
// M (m x r) <- orthonormal basis of range(M) by CholQR2; R (r x r, upper) with M_in = M_out R
// when R is given.  G: r x r scratch per node (stride r*r), R2 scratch likewise.
fio_status cholqr2(z* M, int m, int r, int64_t sM, z* G, z* R, z* R2, int batch, int* status, cudaStream_t st) {
    const int64_t sG = int64_t(r) * r;
    for (int pass = 0; pass < 2; ++pass) {
        FIO_TRY(zgemm('C', 'N', r, r, m, ONE, M, m, sM, M, m, sM, ZERO, G, r, sG, batch, st));
        FIO_TRY(potrf(G, r, r, sG, batch, status, st));
        FIO_TRY(trsm_right_lh(M, m, r, m, sM, G, r, sG, batch, st));
        if (R) {
            if (pass == 0) {   // R = L1^*
                k_conjT<<<g2(sG, batch), TBD, 0, st>>>(G, r, sG, R, r, sG, r, r);
            } else {           // R = L2^* L1^*
                FIO_TRY(zgemm('C', 'N', r, r, r, ONE, G, r, sG, R, r, sG, ZERO, R2, r, sG, batch, st));
                k_copy<<<g2(sG, batch), TBD, 0, st>>>(R2, r, sG, R, r, sG, r, r);
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
    DevBuf Oz, Yz, G, W, GZ, dg, perm, rank, sat, done, thr, thr2, mx, M, R, R2, T1, T2, status;
    DevBuf Q, T, Dc, E, Bz, Upz, Li;
    int lvl_m = 0, lvl_c = 0;   // node size and null-basis width of the last node pass
    void release() {
        for (DevBuf* b : {&Oz, &Yz, &G, &W, &GZ, &dg, &perm, &rank, &sat, &done, &thr, &thr2, &mx, &M, &R, &R2, &T1, &T2,
                          &status, &Q, &T, &Dc, &E, &Bz, &Upz, &Li})
            b->release();
    }
};
BigScratch* big_scratch_new() { return new BigScratch(); }
void big_scratch_free(BigScratch* b) {
    if (!b) return;
    b->release();
    delete b;
}

void set_large_node_min(int m) { g_large_min = m; }
bool large_level(int nodes, int m) { return nodes <= 16 && m >= g_large_min; }

// Node pass of a large level: per node t, Omega^+ and W = Y Omega^+, the null basis
// Gamma, A = Y Gamma and the pivoted Cholesky of A^* A (at most `rhat` steps); the
// rank is the number of pivots above thr^2.  khat / sat to host.
fio_status big_level_nodes(BigScratch& w, int nn, int m, int s, int rhat, const float2* Om, const float2* Y, int64_t ld,
                           double tol, std::vector<int>& hk, std::vector<int>& hs, cudaStream_t st) {
    const int c = s - m;
    const int64_t ms = int64_t(m) * s, mm = int64_t(m) * m, sc = int64_t(s) * c, mc = int64_t(m) * c,
                  cc = int64_t(c) * c;
    FIO_TRY(w.Oz.ensure(size_t(nn) * ms * 16));
    FIO_TRY(w.Yz.ensure(size_t(nn) * ms * 16));
    FIO_TRY(w.G.ensure(size_t(nn) * std::max(mm, cc) * 16));
    FIO_TRY(w.W.ensure(size_t(nn) * mm * 16));
    FIO_TRY(w.Q.ensure(size_t(nn) * ms * 16));     // Omega^+ (s x m)
    FIO_TRY(w.E.ensure(size_t(nn) * sc * 16));     // E -> Gamma (s x c)
    FIO_TRY(w.T.ensure(size_t(nn) * mc * 16));     // Omega E (m x c), then A = Y Gamma
    FIO_TRY(w.GZ.ensure(size_t(nn) * cc * 16));    // A^* A
    FIO_TRY(w.R.ensure(size_t(nn) * cc * 16));
    FIO_TRY(w.R2.ensure(size_t(nn) * cc * 16));
    FIO_TRY(w.dg.ensure(size_t(nn) * c * 8));
    FIO_TRY(w.perm.ensure(size_t(nn) * c * 4));
    FIO_TRY(w.rank.ensure(size_t(nn) * 4));
    FIO_TRY(w.sat.ensure(size_t(nn) * 4));
    FIO_TRY(w.done.ensure(size_t(nn) * 4));
    FIO_TRY(w.thr.ensure(size_t(nn) * 8));
    FIO_TRY(w.thr2.ensure(size_t(nn) * 8));
    FIO_TRY(w.mx.ensure(size_t(nn) * 8));
    FIO_TRY(w.status.ensure(4));
    z* Oz = w.Oz.as<z>();
    z* Yz = w.Yz.as<z>();
    z* G = w.G.as<z>();
    z* W = w.W.as<z>();
    z* Op = w.Q.as<z>();
    z* E = w.E.as<z>();
    z* A = w.T.as<z>();
    z* GA = w.GZ.as<z>();
    int* status = w.status.as<int>();
    w.lvl_m = m;
    w.lvl_c = c;
    FIO_CUDA(cudaMemsetAsync(status, 0, 4, st));
    FIO_CUDA(cudaMemsetAsync(w.mx.p, 0, size_t(nn) * 8, st));
    k_f2_to_z<<<g2(ms, nn), TBD, 0, st>>>(Om, ld, m, Oz, m, ms, m, s);
    k_f2_to_z<<<g2(ms, nn), TBD, 0, st>>>(Y, ld, m, Yz, m, ms, m, s);
    k_colnorm_max<<<dim3(cdiv(int64_t(s) * 32, TBD), nn), TBD, 0, st>>>(Y, ld, m, m, s, w.mx.as<unsigned long long>());
    k_thr<<<1, 32, 0, st>>>(w.mx.as<unsigned long long>(), tol, nn, w.thr.as<double>(), w.thr2.as<double>());
    // G = Omega Omega^* = L L^*;  Omega^+ = Omega^* G^{-1};  W = Y Omega^+
    FIO_TRY(zgemm('N', 'C', m, m, s, ONE, Oz, m, ms, Oz, m, ms, ZERO, G, m, mm, nn, st));
    FIO_TRY(potrf(G, m, m, mm, nn, status, st));
    k_conjT<<<g2(ms, nn), TBD, 0, st>>>(Oz, m, ms, Op, s, ms, m, s);
    FIO_TRY(trsm_right_lh(Op, s, m, s, ms, G, m, mm, nn, st));
    FIO_TRY(trsm_right_l(Op, s, m, s, ms, G, m, mm, nn, st));
    FIO_TRY(zgemm('N', 'N', m, m, s, ONE, Yz, m, ms, Op, s, ms, ZERO, W, m, mm, nn, st));
    if (c > 0) {
        // Gamma: (I - Omega^+ Omega) E, twice, then CholQR2
        k_randn<<<g2(sc, nn), TBD, 0, st>>>(E, sc, s, c, 0x9a77a5eedull + uint64_t(m) * 131 + s);
        for (int pass = 0; pass < 2; ++pass) {
            FIO_TRY(zgemm('N', 'N', m, c, s, ONE, Oz, m, ms, E, s, sc, ZERO, A, m, mc, nn, st));
            FIO_TRY(zgemm('N', 'N', s, c, m, MONE, Op, s, ms, A, m, mc, ONE, E, s, sc, nn, st));
        }
        FIO_TRY(cholqr2(E, s, c, sc, w.R.as<z>(), nullptr, nullptr, nn, status, st));
        // A = Y Gamma, GA = A^* A
        FIO_TRY(zgemm('N', 'N', m, c, s, ONE, Yz, m, ms, E, s, sc, ZERO, A, m, mc, nn, st));
        FIO_TRY(zgemm('C', 'N', c, c, m, ONE, A, m, mc, A, m, mc, ZERO, GA, c, cc, nn, st));
        const int maxk = std::min(rhat, c);
        k_pstrf_init<<<dim3(cdiv(c, TBD), nn), TBD, 0, st>>>(GA, c, cc, c, w.dg.as<double>(), w.perm.as<int>(),
                                                             w.done.as<int>());
        for (int j0 = 0; j0 < maxk; j0 += NB) {
            const int j1 = std::min(maxk, j0 + NB);
            k_pstrf_panel<<<nn, TBD, 0, st>>>(GA, c, cc, c, j0, j1, maxk, w.thr2.as<double>(), w.dg.as<double>(),
                                              w.perm.as<int>(), w.rank.as<int>(), w.sat.as<int>(), w.done.as<int>());
            if (j1 < c)   // trailing update (harmless for nodes that stopped)
                FIO_TRY(zgemm('N', 'C', c - j1, c - j1, j1 - j0, MONE, GA + j1 + int64_t(j0) * c, c, cc,
                              GA + j1 + int64_t(j0) * c, c, cc, ONE, GA + j1 + int64_t(j1) * c, c, cc, nn, st));
        }
        k_pstrf_finish<<<nn, TBD, 0, st>>>(c, maxk, w.thr2.as<double>(), w.dg.as<double>(), w.rank.as<int>(),
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
    if (hst) return fail(FIO_ENOTHPD, "hss_build_from_samples: Omega_tau Omega_tau^* not positive definite");
    return FIO_OK;
}

// Finishing pass: U (float2, nn x m x rl) from the leading rl pivots (CholQR2), and
// D-check (float2, nn x m x m): X = (I - U U^*) W, D = X + U U^* X^*.
fio_status big_level_finish(BigScratch& w, int nn, int m, int rl, float2* Uout, float2* Dchk, cudaStream_t st) {
    const int64_t mm = int64_t(m) * m, mr = int64_t(m) * std::max(rl, 1), rr = int64_t(std::max(rl, 1)) * std::max(rl, 1);
    z* W = w.W.as<z>();
    int* status = w.status.as<int>();
    if (rl > 0) {
        FIO_TRY(w.M.ensure(size_t(nn) * mr * 16));
        FIO_TRY(w.R.ensure(size_t(nn) * std::max<int64_t>(rr, int64_t(w.lvl_c) * w.lvl_c) * 16));
        FIO_TRY(w.T1.ensure(size_t(nn) * mr * 16));
        FIO_TRY(w.T2.ensure(size_t(nn) * mr * 16));
        z* M = w.M.as<z>();
        k_gather_cols<<<g2(int64_t(m) * rl, nn), TBD, 0, st>>>(w.T.as<z>(), m, int64_t(m) * w.lvl_c, w.lvl_c,
                                                              w.perm.as<int>(), w.rank.as<int>(), rl, M, mr,
                                                              0xb4515ull + uint64_t(m) * 7 + rl);
        FIO_TRY(cholqr2(M, m, rl, mr, w.R.as<z>(), nullptr, nullptr, nn, status, st));
        k_z_to_f2<<<g2(mr, nn), TBD, 0, st>>>(M, m, mr, Uout, m, mr, m, rl);
        // T1 = U^* W (rl x m); W <- X = W - U T1; T2 = X U (m x rl); X <- X + U T2^*
        z* T1 = w.T1.as<z>();
        z* T2 = w.T2.as<z>();
        FIO_TRY(zgemm('C', 'N', rl, m, m, ONE, M, m, mr, W, m, mm, ZERO, T1, rl, mr, nn, st));
        FIO_TRY(zgemm('N', 'N', m, m, rl, MONE, M, m, mr, T1, rl, mr, ONE, W, m, mm, nn, st));
        FIO_TRY(zgemm('N', 'N', m, rl, m, ONE, W, m, mm, M, m, mr, ZERO, T2, m, mr, nn, st));
        FIO_TRY(zgemm('N', 'C', m, m, rl, ONE, M, m, mr, T2, m, mr, ONE, W, m, mm, nn, st));
    }
    k_z_to_f2<<<g2(mm, nn), TBD, 0, st>>>(W, m, mm, Dchk, m, mm, m, m);
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}

// Root of the construction: D0 = Herm(Y Omega^+) (double2, m0 x m0), Omega / Y: m0 x s0 float2.
fio_status big_root(BigScratch& w, int m0, int s0, const float2* Om, const float2* Y, double2* D0, cudaStream_t st) {
    const int64_t ms = int64_t(m0) * s0, mm = int64_t(m0) * m0;
    FIO_TRY(w.Oz.ensure(size_t(ms) * 16));
    FIO_TRY(w.Yz.ensure(size_t(ms) * 16));
    FIO_TRY(w.G.ensure(size_t(mm) * 16));
    FIO_TRY(w.status.ensure(4));
    int* status = w.status.as<int>();
    FIO_CUDA(cudaMemsetAsync(status, 0, 4, st));
    z* Oz = w.Oz.as<z>();
    z* Yz = w.Yz.as<z>();
    z* G = w.G.as<z>();
    k_f2_to_z<<<g2(ms, 1), TBD, 0, st>>>(Om, m0, 0, Oz, m0, 0, m0, s0);
    k_f2_to_z<<<g2(ms, 1), TBD, 0, st>>>(Y, m0, 0, Yz, m0, 0, m0, s0);
    FIO_TRY(zgemm('N', 'C', m0, m0, s0, ONE, Oz, m0, 0, Oz, m0, 0, ZERO, G, m0, 0, 1, st));
    FIO_TRY(zgemm('N', 'C', m0, m0, s0, ONE, Yz, m0, 0, Oz, m0, 0, ZERO, D0, m0, 0, 1, st));
    FIO_TRY(potrf(G, m0, m0, 0, 1, status, st));
    FIO_TRY(trsm_right_lh(D0, m0, m0, m0, 0, G, m0, 0, 1, st));
    FIO_TRY(trsm_right_l(D0, m0, m0, m0, 0, G, m0, 0, 1, st));
    k_herm<<<g2(mm, 1), TBD, 0, st>>>(D0, m0, 0, m0);
    int hst = 0;
    FIO_CUDA(cudaMemcpyAsync(&hst, status, 4, cudaMemcpyDeviceToHost, st));
    FIO_CUDA(cudaStreamSynchronize(st));
    if (hst) return fail(FIO_ENOTHPD, "hss_build_from_samples: root Omega Omega^* not positive definite");
    return FIO_OK;
}

// Postprocessing of level l (Section 3.3) with GEMMs: for each parent t (Dcur: nn blocks
// 2rc x 2rc), B_t = Herm(D_t)[rc:, :rc]; child a = 2t + ch: Dnext_a = Dchk_a + U_a H_cc U_a^*.
fio_status big_post(BigScratch& w, int nn, int rc, int mc, double2* Dcur, const float2* Uc, const float2* Dchk,
                    float2* Bout, double2* Dnext, cudaStream_t st) {
    const int mt = 2 * rc;
    const int64_t st_t = int64_t(mt) * mt, mr = int64_t(mc) * rc, mcc = int64_t(mc) * mc;
    FIO_TRY(w.M.ensure(size_t(2 * nn) * std::max<int64_t>(mr, 1) * 16));
    FIO_TRY(w.T1.ensure(size_t(2 * nn) * std::max<int64_t>(mr, 1) * 16));
    z* Uz = w.M.as<z>();
    z* T = w.T1.as<z>();
    k_f2_to_z<<<g2(mcc, 2 * nn), TBD, 0, st>>>(Dchk, mc, mcc, Dnext, mc, mcc, mc, mc);
    if (rc == 0) {
        FIO_CUDA(cudaGetLastError());
        return FIO_OK;
    }
    k_herm<<<g2(st_t, nn), TBD, 0, st>>>(Dcur, mt, st_t, mt);
    k_z_to_f2<<<g2(int64_t(rc) * rc, nn), TBD, 0, st>>>(Dcur + rc, mt, st_t, Bout, rc, int64_t(rc) * rc, rc, rc);
    k_f2_to_z<<<g2(mr, 2 * nn), TBD, 0, st>>>(Uc, mc, mr, Uz, mc, mr, mc, rc);
    for (int ch = 0; ch < 2; ++ch) {
        // children 2t + ch over t: stride 2 blocks
        const z* H = Dcur + ch * rc + int64_t(ch * rc) * mt;
        z* Ua = Uz + ch * mr;
        z* Ta = T + ch * mr;
        z* Da = Dnext + ch * mcc;
        FIO_TRY(zgemm('N', 'N', mc, rc, rc, ONE, Ua, mc, 2 * mr, H, mt, st_t, ZERO, Ta, mc, 2 * mr, nn, st));
        FIO_TRY(zgemm('N', 'C', mc, mc, rc, ONE, Ta, mc, 2 * mr, Ua, mc, 2 * mr, ONE, Da, mc, 2 * mcc, nn, st));
    }
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}

// ULV node factorization of a large level (FP64): D (nn x m x m), U (nn x m x r) ->
// W (float2 nn x m x m), Dh22 and Uh2 (double2 nn x r x r).
fio_status big_ulv_nodes(BigScratch& b, int nn, int m, int r, const double2* D, const double2* U, float2* Wout,
                         double2* Dh22, double2* Uh2, int* d_status, cudaStream_t st) {
    const int n1 = m - r;
    const int64_t mm = int64_t(m) * m, rr = int64_t(std::max(r, 1)) * std::max(r, 1);
    const int64_t n1n1 = int64_t(std::max(n1, 1)) * std::max(n1, 1);
    FIO_TRY(b.Q.ensure(size_t(nn) * mm * 16));
    FIO_TRY(b.T.ensure(size_t(nn) * mm * 16));
    FIO_TRY(b.Dc.ensure(size_t(nn) * mm * 16));
    FIO_TRY(b.G.ensure(size_t(nn) * std::max(rr, n1n1) * 16));
    FIO_TRY(b.R2.ensure(size_t(nn) * std::max(rr, n1n1) * 16));
    z* Q = b.Q.as<z>();     // [Q1 | Q2]
    z* T = b.T.as<z>();
    z* Dc = b.Dc.as<z>();
    z* Q2 = Q + int64_t(n1) * m;
    if (r > 0) {
        // Q2 R = U (CholQR2)
        k_copy<<<g2(int64_t(m) * r, nn), TBD, 0, st>>>(U, m, int64_t(m) * r, Q2, m, mm, m, r);
        FIO_TRY(cholqr2(Q2, m, r, mm, b.G.as<z>(), Uh2, b.R2.as<z>(), nn, d_status, st));
    }
    if (n1 > 0) {
        // Q1 = orth((I - Q2 Q2^*) E), E Gaussian m x n1
        k_randn<<<g2(int64_t(m) * n1, nn), TBD, 0, st>>>(Q, mm, m, n1, 0x5eedull + uint64_t(m) * 977 + r);
        if (r > 0) {
            FIO_TRY(b.E.ensure(size_t(nn) * int64_t(r) * n1 * 16));
            z* P = b.E.as<z>();
            const int64_t rn = int64_t(r) * n1;
            for (int pass = 0; pass < 2; ++pass) {   // project twice against range(Q2)
                FIO_TRY(zgemm('C', 'N', r, n1, m, ONE, Q2, m, mm, Q, m, mm, ZERO, P, r, rn, nn, st));
                FIO_TRY(zgemm('N', 'N', m, n1, r, MONE, Q2, m, mm, P, r, rn, ONE, Q, m, mm, nn, st));
            }
        }
        FIO_TRY(cholqr2(Q, m, n1, mm, b.G.as<z>(), nullptr, nullptr, nn, d_status, st));
    }
    // D-check = Q^* D Q
    FIO_TRY(zgemm('N', 'N', m, m, m, ONE, D, m, mm, Q, m, mm, ZERO, T, m, mm, nn, st));
    FIO_TRY(zgemm('C', 'N', m, m, m, ONE, Q, m, mm, T, m, mm, ZERO, Dc, m, mm, nn, st));
    k_herm<<<g2(mm, nn), TBD, 0, st>>>(Dc, m, mm, m);
    z* A1 = T;   // reuse: A1 (n1 x m) at T, Q2^* (r x m) below it -> W (m x m) column-major
    if (n1 > 0) {
        FIO_TRY(potrf(Dc, n1, m, mm, nn, d_status, st));                               // L11
        if (r > 0) FIO_TRY(trsm_right_lh(Dc + n1, r, n1, m, mm, Dc, m, mm, nn, st));   // D^_21 = D-check_21 L11^{-*}
        // A1 = L11^{-1} Q1^*  (n1 x m, rows 0..n1-1 of T)
        k_conjT<<<g2(int64_t(m) * n1, nn), TBD, 0, st>>>(Q, m, mm, A1, m, mm, m, n1);
        FIO_TRY(trsm_left_l(A1, n1, m, m, mm, Dc, m, mm, nn, st));
    }
    if (r > 0) {
        // D^_22 = D-check_22 - D^_21 D^_21^*
        if (n1 > 0)
            FIO_TRY(zgemm('N', 'C', r, r, n1, MONE, Dc + n1, m, mm, Dc + n1, m, mm, ONE, Dc + n1 + int64_t(n1) * m, m, mm,
                          nn, st));
        k_copy<<<g2(rr, nn), TBD, 0, st>>>(Dc + n1 + int64_t(n1) * m, m, mm, Dh22, r, rr, r, r);
        // rows n1..m-1 of W: Q2^* - D^_21 A1
        k_conjT<<<g2(int64_t(m) * r, nn), TBD, 0, st>>>(Q2, m, mm, T + n1, m, mm, m, r);
        if (n1 > 0)
            FIO_TRY(zgemm('N', 'N', r, m, n1, MONE, Dc + n1, m, mm, A1, m, mm, ONE, T + n1, m, mm, nn, st));
    }
    k_z_to_f2<<<g2(mm, nn), TBD, 0, st>>>(T, m, mm, Wout, m, mm, m, m);
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}

// Merge (Eq. 2.12) with GEMMs: parents t = 0..np-1, children 2t, 2t+1 of rank r;
// D+ (2r x 2r) = [[D1, U1 B^* U2^*], [U2 B U1^*, D2]], U+ = [U1 Up_top; U2 Up_bot].
fio_status big_ulv_merge(BigScratch& b, int np, int r, const double2* Dh22, const double2* Uh2, const float2* B,
                         const float2* Up, int rp, double2* Dplus, double2* Uplus, cudaStream_t st) {
    const int m = 2 * r;
    const int64_t rr = int64_t(r) * r, mm = int64_t(m) * m;
    FIO_TRY(b.Bz.ensure(size_t(np) * rr * 16));
    FIO_TRY(b.T1.ensure(size_t(np) * rr * 16));
    z* Bz = b.Bz.as<z>();
    z* T = b.T1.as<z>();
    k_f2_to_z<<<g2(rr, np), TBD, 0, st>>>(B, r, rr, Bz, r, rr, r, r);
    const z* U1 = Uh2;
    const z* U2 = Uh2 + rr;
    // T = B U1^*; lower-left = U2 T
    FIO_TRY(zgemm('N', 'C', r, r, r, ONE, Bz, r, rr, U1, r, 2 * rr, ZERO, T, r, rr, np, st));
    FIO_TRY(zgemm('N', 'N', r, r, r, ONE, U2, r, 2 * rr, T, r, rr, ZERO, Dplus + r, m, mm, np, st));
    k_conjT<<<g2(rr, np), TBD, 0, st>>>(Dplus + r, m, mm, Dplus + int64_t(r) * m, m, mm, r, r);
    k_copy<<<g2(rr, np), TBD, 0, st>>>(Dh22, r, 2 * rr, Dplus, m, mm, r, r);
    k_copy<<<g2(rr, np), TBD, 0, st>>>(Dh22 + rr, r, 2 * rr, Dplus + r + int64_t(r) * m, m, mm, r, r);
    if (Up && rp > 0) {
        const int64_t mr = int64_t(m) * rp;
        FIO_TRY(b.Upz.ensure(size_t(np) * mr * 16));
        z* Upz = b.Upz.as<z>();
        k_f2_to_z<<<g2(mr, np), TBD, 0, st>>>(Up, m, mr, Upz, m, mr, m, rp);
        FIO_TRY(zgemm('N', 'N', r, rp, r, ONE, U1, r, 2 * rr, Upz, m, mr, ZERO, Uplus, m, mr, np, st));
        FIO_TRY(zgemm('N', 'N', r, rp, r, ONE, U2, r, 2 * rr, Upz + r, m, mr, ZERO, Uplus + r, m, mr, np, st));
    }
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}

// Root: D+ = L L^*, Rinv = L^{-*} L^{-1} (float2).
fio_status big_ulv_root(BigScratch& b, int m0, const double2* Dp, float2* Rinv, int* d_status, cudaStream_t st) {
    const int64_t mm = int64_t(m0) * m0;
    FIO_TRY(b.Q.ensure(size_t(mm) * 16));
    FIO_TRY(b.Li.ensure(size_t(mm) * 16));
    FIO_TRY(b.T.ensure(size_t(mm) * 16));
    z* L = b.Q.as<z>();
    z* Li = b.Li.as<z>();
    k_copy<<<g2(mm, 1), TBD, 0, st>>>(Dp, m0, 0, L, m0, 0, m0, m0);
    FIO_TRY(potrf(L, m0, m0, 0, 1, d_status, st));
    k_eye<<<g2(mm, 1), TBD, 0, st>>>(Li, m0, 0, m0);
    FIO_TRY(trsm_left_l(Li, m0, m0, m0, 0, L, m0, 0, 1, st));
    FIO_TRY(zgemm('C', 'N', m0, m0, m0, ONE, Li, m0, 0, Li, m0, 0, ZERO, b.T.as<z>(), m0, 0, 1, st));
    k_z_to_f2<<<g2(mm, 1), TBD, 0, st>>>(b.T.as<z>(), m0, 0, Rinv, m0, 0, m0, m0);
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}

}  // namespace fio

extern "C" fio_status fio_set_large_node(int m_min) {
    if (m_min < 1) return fio::fail(FIO_EINVAL, "fio_set_large_node: m_min must be >= 1");
    fio::set_large_node_min(m_min);
    return FIO_OK;
}
