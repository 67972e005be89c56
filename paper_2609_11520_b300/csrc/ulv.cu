// ULV factorization of the HSS matrix G~ (Section 2.4, Eq. 2.9-2.12) and the
// bottom-up / root / top-down solve.
//
// Per node (D: m x m Hermitian, U: m x r with orthonormal columns):
//   QR of U by r Householder reflectors, U = Q_r [R; 0].  Q = Q_r P with P
//   moving the first r rows to the bottom gives Q^* U = [0; R]: U^_2 = R
//   (basis elimination, Eq. 2.9).
//   D-check = Q^* D Q; Cholesky D-check_11 = L11 L11^*; D^_21 = D-check_21 L11^{-*};
//   D^_22 = D-check_22 - D^_21 D^_21^* (partial factorization, Eq. 2.10-2.11).
//   The node keeps the single matrix
//       W = [[L11^{-1} Q1^*], [Q2^* - D^_21 L11^{-1} Q1^*]]   (Q = [Q1 Q2])
//   so that the up pass is [b^_1; y^_2] = W y and the down pass is
//   c = Q [c^_1; c^_2] = W^* [b^_1; c^_2] with c^_1 = L11^{-*}(b^_1 - D^_21^* c^_2).
//   Merge (Eq. 2.12): D+ = [[D^22_1, U^2_1 B^* U^2_2^*], [U^2_2 B U^2_1^*, D^22_2]],
//   U+ = diag(U^2_1, U^2_2) U_parent.  Root: D+ = L L^*, stored as (L L^*)^{-1}.
#include <algorithm>
#include <type_traits>
#include <cmath>

#include "cplx.cuh"
#include "hss.cuh"
#include "tc.cuh"
#include "ulv_body.cuh"

namespace fio {
namespace {

constexpr int TB = 256;
constexpr int kFp64Nodes = 16;   // FP64 on levels with at most this many nodes

template <class C>
__device__ void zlarfg(C alpha, typename RealOf<C>::T xn, typename RealOf<C>::T& beta, C& tau, C& scal) {
    using R = typename RealOf<C>::T;
    if (xn == R(0) && alpha.y == R(0)) {
        beta = alpha.x;
        tau = czero<C>();
        scal = czero<C>();
    } else {
        R nrm = sqrt(alpha.x * alpha.x + alpha.y * alpha.y + xn);
        beta = alpha.x >= 0 ? -nrm : nrm;
        tau = mkc<C>((beta - alpha.x) / beta, -alpha.y / beta);
        scal = gdiv(mkc<C>(1, 0), mkc<C>(alpha.x - beta, alpha.y));
    }
}

// Node factorization.  Inputs: D (float2 Df or C Dc, column-major m x m),
// U (float2 Uf or C Uc, column-major m x r).  Outputs: W (float2, column-major
// m x m), D^22 and U^2 (C, column-major r x r).  Scratch per node (C):
// Dw m*m | Qr m*m | A1 m*m | Ur m*r | Dh21 r*m | tau r.
template <class C>
__global__ void k_ulv_node(const float2* __restrict__ Df, const C* __restrict__ Dc, const float2* __restrict__ Uf,
                           const C* __restrict__ Uc, int m, int r, float2* __restrict__ Wout, C* __restrict__ Dh22,
                           C* __restrict__ Uh2, C* __restrict__ scr, int* status) {
    using R = typename RealOf<C>::T;
    __shared__ R red[32];
    const int t = blockIdx.x, tid = threadIdx.x, bd = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = bd >> 5;
    const int n1 = m - r;
    const int64_t mm = int64_t(m) * m;
    C* Dw = scr + int64_t(t) * (3 * mm + 2 * int64_t(m) * r + r);
    C* Qr = Dw + mm;
    C* A1 = Qr + mm;
    C* Ur = A1 + mm;
    C* Dh21 = Ur + int64_t(m) * r;
    C* taus = Dh21 + int64_t(m) * r;
    for (int64_t e = tid; e < mm; e += bd) Dw[e] = Df ? cvt<C>(Df[t * mm + e]) : Dc[t * mm + e];
    for (int64_t e = tid; e < int64_t(m) * r; e += bd)
        Ur[e] = Uf ? cvt<C>(Uf[t * int64_t(m) * r + e]) : Uc[t * int64_t(m) * r + e];
    __syncthreads();
    // QR of U
    for (int k = 0; k < r; ++k) {
        C* col = Ur + int64_t(k) * m;
        R xn = 0;
        for (int i = k + 1 + tid; i < m; i += bd) xn += gabs2(col[i]);
        xn = block_sum(xn, red);
        R beta;
        C tau, scal;
        zlarfg(col[k], xn, beta, tau, scal);
        __syncthreads();
        for (int i = k + 1 + tid; i < m; i += bd) col[i] = gmul(col[i], scal);
        if (tid == 0) {
            col[k] = mkc<C>(beta, 0);
            taus[k] = tau;
        }
        __syncthreads();
        for (int j = k + 1 + warp; j < r; j += nw) {
            C* cj = Ur + int64_t(j) * m;
            C w = lane == 0 ? cj[k] : czero<C>();
            for (int i = k + 1 + lane; i < m; i += 32) gfmac(w, col[i], cj[i]);
            w.x = warp_sum(w.x);
            w.y = warp_sum(w.y);
            C tw = gmulc(tau, w);
            if (lane == 0) cj[k] = gsub(cj[k], tw);
            for (int i = k + 1 + lane; i < m; i += 32) cj[i] = gsub(cj[i], gmul(col[i], tw));
        }
        __syncthreads();
    }
    // U^_2 = R
    for (int e = tid; e < r * r; e += bd) {
        int i = e % r, j = e / r;
        Uh2[int64_t(t) * r * r + e] = i <= j ? Ur[i + int64_t(j) * m] : czero<C>();
    }
    // D <- Q_r^* D Q_r  (reflector k = 0 first, both sides)
    for (int k = 0; k < r; ++k) {
        const C* v = Ur + int64_t(k) * m;   // v_k = 1 implied, v_i = v[i] for i > k
        C tau = taus[k];
        for (int c = warp; c < m; c += nw) {   // left: columns
            C* dc = Dw + int64_t(c) * m;
            C w = lane == 0 ? dc[k] : czero<C>();
            for (int i = k + 1 + lane; i < m; i += 32) gfmac(w, v[i], dc[i]);
            w.x = warp_sum(w.x);
            w.y = warp_sum(w.y);
            C tw = gmulc(tau, w);
            if (lane == 0) dc[k] = gsub(dc[k], tw);
            for (int i = k + 1 + lane; i < m; i += 32) dc[i] = gsub(dc[i], gmul(v[i], tw));
        }
        __syncthreads();
        for (int i = tid; i < m; i += bd) {   // right: rows
            C w = Dw[i + int64_t(k) * m];
            for (int j = k + 1; j < m; ++j) gfma(w, Dw[i + int64_t(j) * m], v[j]);
            C tw = gmul(tau, w);
            Dw[i + int64_t(k) * m] = gsub(Dw[i + int64_t(k) * m], tw);
            for (int j = k + 1; j < m; ++j) Dw[i + int64_t(j) * m] = gsub(Dw[i + int64_t(j) * m], gmul(tw, gconj(v[j])));
        }
        __syncthreads();
    }
    // explicit Q_r = H_0 .. H_{r-1}
    for (int64_t e = tid; e < mm; e += bd) Qr[e] = (e % m == e / m) ? mkc<C>(1, 0) : czero<C>();
    __syncthreads();
    for (int k = r - 1; k >= 0; --k) {
        const C* v = Ur + int64_t(k) * m;
        C tau = taus[k];
        for (int c = warp; c < m; c += nw) {
            C* qc = Qr + int64_t(c) * m;
            C w = lane == 0 ? qc[k] : czero<C>();
            for (int i = k + 1 + lane; i < m; i += 32) gfmac(w, v[i], qc[i]);
            w.x = warp_sum(w.x);
            w.y = warp_sum(w.y);
            C tw = gmul(tau, w);
            if (lane == 0) qc[k] = gsub(qc[k], tw);
            for (int i = k + 1 + lane; i < m; i += 32) qc[i] = gsub(qc[i], gmul(v[i], tw));
        }
        __syncthreads();
    }
    // Cholesky of D-check_11 = Dw[r:, r:] (left-looking, lower, in place)
    auto L = [&](int i, int j) -> C& { return Dw[(r + i) + int64_t(r + j) * m]; };
    __shared__ R s_d;
    for (int j = 0; j < n1; ++j) {
        if (tid == 0) {
            R d = L(j, j).x;
            for (int k = 0; k < j; ++k) d -= gabs2(L(j, k));
            if (!(d > R(0))) {
                atomicExch(status, FIO_ENOTHPD);
                d = R(1);
            }
            s_d = sqrt(d);
        }
        __syncthreads();
        R dj = s_d;
        for (int i = j + 1 + tid; i < n1; i += bd) {
            C a = L(i, j);
            for (int k = 0; k < j; ++k) a = gsub(a, gmul(L(i, k), gconj(L(j, k))));
            L(i, j) = gscale(a, R(1) / dj);
        }
        __syncthreads();
        if (tid == 0) L(j, j) = mkc<C>(dj, 0);
        __syncthreads();
    }
    // D^_21 = D-check_21 L^{-*}: row i solves L conj(x) = conj(D-check_21[i, :])
    for (int i = tid; i < r; i += bd) {
        for (int j = 0; j < n1; ++j) {
            C y = gconj(Dw[i + int64_t(r + j) * m]);
            for (int k = 0; k < j; ++k) y = gsub(y, gmul(L(j, k), gconj(Dh21[i + int64_t(k) * r])));
            Dh21[i + int64_t(j) * r] = gconj(gscale(y, R(1) / L(j, j).x));
        }
    }
    __syncthreads();
    // D^_22 = D-check_22 - D^_21 D^_21^*
    for (int e = tid; e < r * r; e += bd) {
        int i = e % r, j = e / r;
        C a = Dw[i + int64_t(j) * m];
        for (int k = 0; k < n1; ++k) a = gsub(a, gmul(Dh21[i + int64_t(k) * r], gconj(Dh21[j + int64_t(k) * r])));
        Dh22[int64_t(t) * r * r + e] = a;
    }
    // A1 = L^{-1} Q1^*,  Q1 = Qr[:, r:]  (column c of A1: forward substitution)
    for (int c = tid; c < m; c += bd) {
        for (int j = 0; j < n1; ++j) {
            C y = gconj(Qr[c + int64_t(r + j) * m]);
            for (int k = 0; k < j; ++k) y = gsub(y, gmul(L(j, k), A1[k + int64_t(c) * m]));
            A1[j + int64_t(c) * m] = gscale(y, R(1) / L(j, j).x);
        }
    }
    __syncthreads();
    // W = [A1; Q2^* - D^_21 A1]
    float2* Wt = Wout + int64_t(t) * mm;
    for (int64_t e = tid; e < mm; e += bd) {
        int i = int(e % m), c = int(e / m);
        C a;
        if (i < n1) {
            a = A1[i + int64_t(c) * m];
        } else {
            int ii = i - n1;
            a = gconj(Qr[c + int64_t(ii) * m]);
            for (int k = 0; k < n1; ++k) a = gsub(a, gmul(Dh21[ii + int64_t(k) * r], A1[k + int64_t(c) * m]));
        }
        Wt[e] = to_f2(a);
    }
}


// Root: D+ = L L^*; Rinv = L^{-*} L^{-1} (complex64 column-major).
__global__ void k_ulv_root(const double2* __restrict__ Dp, int m, float2* __restrict__ Rinv, double2* __restrict__ scr,
                           int* status) {
    const int tid = threadIdx.x, bd = blockDim.x;
    double2* Lm = scr;               // m x m
    double2* Li = scr + int64_t(m) * m;
    for (int e = tid; e < m * m; e += bd) Lm[e] = Dp[e];
    __syncthreads();
    __shared__ double s_d;
    for (int j = 0; j < m; ++j) {
        if (tid == 0) {
            double d = Lm[j + int64_t(j) * m].x;
            for (int k = 0; k < j; ++k) d -= gabs2(Lm[j + int64_t(k) * m]);
            if (!(d > 0)) {
                atomicExch(status, FIO_ENOTHPD);
                d = 1;
            }
            s_d = sqrt(d);
        }
        __syncthreads();
        double dj = s_d;
        for (int i = j + 1 + tid; i < m; i += bd) {
            double2 a = Lm[i + int64_t(j) * m];
            for (int k = 0; k < j; ++k) a = gsub(a, gmul(Lm[i + int64_t(k) * m], gconj(Lm[j + int64_t(k) * m])));
            Lm[i + int64_t(j) * m] = gscale(a, 1.0 / dj);
        }
        __syncthreads();
        if (tid == 0) Lm[j + int64_t(j) * m] = make_double2(dj, 0);
        __syncthreads();
    }
    // Li = L^{-1}, column by column
    for (int c = tid; c < m; c += bd)
        for (int j = 0; j < m; ++j) {
            double2 y = make_double2(j == c ? 1.0 : 0.0, 0);
            for (int k = c; k < j; ++k) y = gsub(y, gmul(Lm[j + int64_t(k) * m], Li[k + int64_t(c) * m]));
            Li[j + int64_t(c) * m] = (j < c) ? make_double2(0, 0) : gscale(y, 1.0 / Lm[j + int64_t(j) * m].x);
        }
    __syncthreads();
    for (int e = tid; e < m * m; e += bd) {
        int i = e % m, j = e / m;
        double2 a = make_double2(0, 0);
        for (int k = max(i, j); k < m; ++k) gfmac(a, Li[k + int64_t(i) * m], Li[k + int64_t(j) * m]);
        Rinv[e] = make_float2(float(a.x), float(a.y));
    }
}

template <class C> __global__ void k_to_f64(const C* __restrict__ a, double2* __restrict__ b, int64_t n) {
    int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e < n) b[e] = make_double2(double(a[e].x), double(a[e].y));
}

// ------------------------------------------------------------- solve
using ulvb::KCOL;
using ulvb::RB;
using ulvb::WT;

template <bool CONJ>
__device__ void node_gemm_body(const float2* __restrict__ W, int m, const float2* __restrict__ inA, int nA, int64_t ldA,
                               const float2* __restrict__ inB, int64_t ldB, float2* __restrict__ outC, int nC,
                               int64_t ldC, float2* __restrict__ outD, int64_t ldD, int k, int t, int c0, int r0) {
    __shared__ float2 sx[WT * KCOL];
    __shared__ float2 sw[WT * RB];
    ulvb::node_gemm_body<CONJ>(W, m, inA, nA, ldA, inB, ldB, outC, nC, ldC, outD, ldD, k, t, c0, r0, sx, sw,
                               [] { __syncthreads(); }, int(threadIdx.x));
}

template <bool CONJ>
__global__ void __launch_bounds__(256) k_ulv_node_gemm(const float2* __restrict__ W, int m, const float2* __restrict__ inA,
                                                       int nA, int64_t ldA, const float2* __restrict__ inB, int64_t ldB,
                                                       float2* __restrict__ outC, int nC, int64_t ldC,
                                                       float2* __restrict__ outD, int64_t ldD, int k) {
    node_gemm_body<CONJ>(W, m, inA, nA, ldA, inB, ldB, outC, nC, ldC, outD, ldD, k, blockIdx.x, blockIdx.y * KCOL,
                         blockIdx.z * RB);
}

// Wide node products (k > 8): one CTA per (node, CB columns, 128 rows, slice of the inner index),
// 256 threads as 16 x 16, each owning 8 rows x CB/16 columns (rows ty + 16 a, columns tx + 16 b);
// W and x staged through shared memory in tiles of 16 inner indices, so each W block is read once
// per CB columns.  With nsplit > 1 the inner index is cut into nsplit slices (levels with few
// nodes and large m) whose partial products go to `part` ([slice][column][node][row]) and are
// summed in slice order by k_ulv_wide_reduce; otherwise the CTA writes the outputs directly.
// Same operands and outputs as k_ulv_node_gemm.
constexpr int kWideRows = 128, kWideJ = 16;
template <bool CONJ, int CB>
__global__ void __launch_bounds__(256) k_ulv_wide(const float2* __restrict__ W, int m, const float2* __restrict__ inA,
                                                  int nA, int64_t ldA, const float2* __restrict__ inB, int64_t ldB,
                                                  float2* __restrict__ outC, int nC, int64_t ldC,
                                                  float2* __restrict__ outD, int64_t ldD, int k, int nsplit, int jslice,
                                                  float2* __restrict__ part) {
    constexpr int NB = CB / 16;
    __shared__ float2 sw[kWideJ][kWideRows + 1];
    __shared__ float2 sx[kWideJ][CB + 1];
    const int t = blockIdx.x, nodes = gridDim.x;
    const int cb = blockIdx.y / nsplit, sp = blockIdx.y % nsplit;
    const int c0 = cb * CB, r0 = blockIdx.z * kWideRows;
    const int jbeg = sp * jslice, jend = min(m, jbeg + jslice);
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int kc = min(CB, k - c0), nr = min(kWideRows, m - r0);
    const float2* Wt = W + int64_t(t) * m * m;
    float2 acc[8][NB];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < NB; ++b) acc[a][b] = make_float2(0.f, 0.f);
    for (int j0 = jbeg; j0 < jend; j0 += kWideJ) {
        const int jw = min(kWideJ, jend - j0);
        for (int e = tid; e < kWideJ * kWideRows; e += 256) {
            int jj, il;
            if (!CONJ) {   // column j of W, rows r0..: consecutive il
                il = e % kWideRows;
                jj = e / kWideRows;
            } else {       // row j of W^*: W[j + i m], consecutive jj
                jj = e % kWideJ;
                il = e / kWideJ;
            }
            float2 v = make_float2(0.f, 0.f);
            if (jj < jw && il < nr)
                v = CONJ ? Wt[(j0 + jj) + int64_t(r0 + il) * m] : Wt[(r0 + il) + int64_t(j0 + jj) * m];
            sw[jj][il] = v;
        }
        for (int e = tid; e < kWideJ * CB; e += 256) {
            const int jj = e % kWideJ, c = e / kWideJ, j = j0 + jj;
            float2 v = make_float2(0.f, 0.f);
            if (jj < jw && c < kc)
                v = (j < nA) ? inA[int64_t(c0 + c) * ldA + int64_t(t) * nA + j]
                             : inB[int64_t(c0 + c) * ldB + int64_t(t) * (m - nA) + (j - nA)];
            sx[jj][c] = v;
        }
        __syncthreads();
#pragma unroll
        for (int jj = 0; jj < kWideJ; ++jj) {
            float2 av[8], bv[NB];
#pragma unroll
            for (int a = 0; a < 8; ++a) av[a] = sw[jj][ty + 16 * a];
#pragma unroll
            for (int b = 0; b < NB; ++b) bv[b] = sx[jj][tx + 16 * b];
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    if (CONJ) cfmac(acc[a][b], av[a], bv[b]);
                    else cfma(acc[a][b], av[a], bv[b]);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const int il = ty + 16 * a;
        if (il >= nr) continue;
        const int i = r0 + il;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int c = tx + 16 * b;
            if (c >= kc) continue;
            if (nsplit > 1)
                part[((int64_t(sp) * k + c0 + c) * nodes + t) * m + i] = acc[a][b];
            else if (i < nC)
                outC[int64_t(c0 + c) * ldC + int64_t(t) * nC + i] = acc[a][b];
            else
                outD[int64_t(c0 + c) * ldD + int64_t(t) * (m - nC) + (i - nC)] = acc[a][b];
        }
    }
}

// Sum of the nsplit partial products in slice order, routed to outC / outD.
__global__ void k_ulv_wide_reduce(const float2* __restrict__ part, int nsplit, int nodes, int m, int k,
                                  float2* __restrict__ outC, int nC, int64_t ldC, float2* __restrict__ outD, int64_t ldD) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t per = int64_t(k) * nodes * m;
    if (e >= per) return;
    const int i = int(e % m);
    const int64_t rest = e / m;
    const int t = int(rest % nodes), c = int(rest / nodes);
    float2 v = part[e];
    for (int sp = 1; sp < nsplit; ++sp) v = cadd(v, part[sp * per + e]);
    if (i < nC) outC[int64_t(c) * ldC + int64_t(t) * nC + i] = v;
    else outD[int64_t(c) * ldD + int64_t(t) * (m - nC) + (i - nC)] = v;
}

// Tensor-core node products (solve path 1; k > 8, 32 <= m <= 512): Y = op(W_t) X_t as the real product
//   [Yr | Yi] = [Ar | Ai] [[Xr, Xi], [-Xi, Xr]]     (A = W, or W^* for the down pass)
// on tcgen05.mma of kind::f16.  Both operands are split into 16-bit parts v = hi + lo and the
// three products hi hi + hi lo + lo hi accumulate in FP32 in TMEM: FP16 parts with power-of-two
// scales per row of A and per column of X (FP32 accuracy), or BF16 parts (split precision).
// CTA: 128 threads, one row of the node's 128-row block per thread (TMEM lane = row), 32 complex
// columns (N = 64 real); the inner index in chunks of 32 complex (K = 64 real): each thread
// writes its A row chunk to TMEM (tcgen05.st), the CTA writes the B chunk to shared memory
// (K-major core matrices), one thread issues 4 x 3 MMAs (M = 128, N = 64, K = 16) and commits
// them to an mbarrier that every thread waits on with a bounded wait (a run-out sets
// g_ulv_tc_timeout, read by fio_device_status).
__device__ int g_ulv_tc_timeout = 0;
constexpr int kTcCols = 32, kTcJ = 32, kTcTmem = 128, kTcMaxM = 512;
constexpr uint32_t kTcSbo = (2 * kTcJ / 8) * 128;               // 8-row groups of B (K = 64)
constexpr int kTcPartBytes = 2 * kTcCols * 2 * kTcJ * 2;        // one 16-bit part of B: 8 KB
constexpr int kTcSmem = 2 * kTcPartBytes;                       // B_hi | B_lo (the registers allow three CTAs per SM,
                                                                // within the 4 x 128 TMEM columns)
__device__ __forceinline__ uint32_t tc_boff(int n, int kk) {    // byte offset of B (n, kk), kk even
    return uint32_t(n >> 3) * kTcSbo + uint32_t(kk >> 3) * 128 + uint32_t(n & 7) * 16 + uint32_t(kk & 7) * 2;
}
template <bool CONJ, bool BF>
__global__ void __launch_bounds__(128) k_ulv_tc(const float2* __restrict__ W, const float* __restrict__ Wmx, int m,
                                                const float2* __restrict__ inA, int nA, int64_t ldA,
                                                const float2* __restrict__ inB, int64_t ldB, float2* __restrict__ outC,
                                                int nC, int64_t ldC, float2* __restrict__ outD, int64_t ldD, int k) {
    extern __shared__ __align__(1024) unsigned char tc_smem[];    // B_hi | B_lo
    __shared__ float scol[kTcCols], iscol[kTcCols];
    __shared__ unsigned smax[kTcCols];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_mbar;
    __shared__ int s_fail;
    const int t = blockIdx.x, c0 = blockIdx.y * kTcCols, r0 = blockIdx.z * 128;
    const int tid = threadIdx.x, i = r0 + tid;
    const int kc = min(kTcCols, k - c0);
    const float2* Wt = W + int64_t(t) * m * m;
    auto wv = [&](int j) -> float2 {   // A(i, j) = op(W_t)(i, j)
        if (CONJ) {
            const float2 v = __ldg(Wt + j + int64_t(i) * m);
            return make_float2(v.x, -v.y);
        }
        return __ldg(Wt + i + int64_t(j) * m);
    };
    auto xv = [&](int j, int c) -> float2 {
        return (j < nA) ? inA[int64_t(c0 + c) * ldA + int64_t(t) * nA + j]
                        : inB[int64_t(c0 + c) * ldB + int64_t(t) * (m - nA) + (j - nA)];
    };
    if (tid < 32) tc::tmem_alloc(&s_tmem, kTcTmem);
    if (tid == 0) {
        tc::mbar_init(&s_mbar, 1);
        s_fail = 0;
    }
    if (tid < kTcCols) smax[tid] = 0u;
    __syncthreads();
    float rsc = 1.f, irsc = 1.f;
    if (!BF) {   // power-of-two scales: per column of X (four threads per column), per row of A
        const int c = tid & 31;
        float mx = 0.f;
        if (c < kc)
#pragma unroll 8
            for (int j = tid >> 5; j < m; j += 4) {
                const float2 v = xv(j, c);
                mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
            }
        atomicMax(&smax[c], __float_as_uint(mx));
        // row maxima of W_t and W_t^* stored at factorization
        const float rm = i < m ? Wmx[(CONJ ? int64_t(gridDim.x) * m : 0) + int64_t(t) * m + i] : 0.f;
        tc::row_scale(rm, rsc, irsc);
    }
    __syncthreads();
    if (tid < kTcCols) {
        float sc = 1.f, isc = 1.f;
        if (!BF) tc::row_scale(__uint_as_float(smax[tid]), sc, isc);
        scol[tid] = sc;
        iscol[tid] = isc;
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t tl = tmem + (uint32_t(tid & 0x60) << 16);    // this warp's TMEM lanes
    const uint32_t sb = tc::smem_addr(tc_smem);
    const uint32_t idesc = tc::idesc_f16(BF, 128, 2 * kTcCols);
    uint32_t phase = 0;
    for (int j0 = 0, ch = 0; j0 < m; j0 += kTcJ, ++ch) {
        {   // A chunk of row i: K = 2 (j - j0) + (re, im), hi in TMEM columns 0..31, lo in 32..63
            uint32_t h0[16], h1[16], l0[16], l1[16];
#pragma unroll
            for (int jj = 0; jj < kTcJ; ++jj) {
                const int j = j0 + jj;
                float2 v = make_float2(0.f, 0.f);
                if (i < m && j < m) v = wv(j);
                uint32_t h, l;
                tc::split_pair<BF>(v.x * rsc, v.y * rsc, h, l);
                if (jj < 16) {
                    h0[jj] = h;
                    l0[jj] = l;
                } else {
                    h1[jj - 16] = h;
                    l1[jj - 16] = l;
                }
            }
            tc::tmem_st16(tl + 0, h0);
            tc::tmem_st16(tl + 16, h1);
            tc::tmem_st16(tl + 32, l0);
            tc::tmem_st16(tl + 48, l1);
        }
        // B chunk: row n < 32 -> Yr of column n: (Xr, -Xi); n >= 32 -> Yi of column n - 32: (Xi, Xr)
#pragma unroll
        for (int e = tid; e < kTcCols * kTcJ; e += 128) {
            const int jj = e % kTcJ, c = e / kTcJ, j = j0 + jj;
            float2 x = make_float2(0.f, 0.f);
            if (c < kc && j < m) x = xv(j, c);
            const float sc = scol[c];
            uint32_t h, l;
            tc::split_pair<BF>(x.x * sc, -x.y * sc, h, l);
            *reinterpret_cast<uint32_t*>(tc_smem + tc_boff(c, 2 * jj)) = h;
            *reinterpret_cast<uint32_t*>(tc_smem + kTcPartBytes + tc_boff(c, 2 * jj)) = l;
            tc::split_pair<BF>(x.y * sc, x.x * sc, h, l);
            *reinterpret_cast<uint32_t*>(tc_smem + tc_boff(c + kTcCols, 2 * jj)) = h;
            *reinterpret_cast<uint32_t*>(tc_smem + kTcPartBytes + tc_boff(c + kTcCols, 2 * jj)) = l;
        }
        tc::tmem_wait_st();
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (tid == 0 && !s_fail) {
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                const uint64_t bh = tc::smem_desc(sb + 256 * ks, 128, kTcSbo);
                const uint64_t bl = tc::smem_desc(sb + kTcPartBytes + 256 * ks, 128, kTcSbo);
                tc::mma_f16_ts(tmem + 64, tmem + 8 * ks, bh, idesc, (ch > 0 || ks > 0) ? 1 : 0);
                tc::mma_f16_ts(tmem + 64, tmem + 8 * ks, bl, idesc, 1);
                tc::mma_f16_ts(tmem + 64, tmem + 32 + 8 * ks, bh, idesc, 1);
            }
            tc::mma_commit(&s_mbar);
        }
        if (!s_fail && !tc::mbar_wait(&s_mbar, phase)) {
            s_fail = 1;
            atomicExch(&g_ulv_tc_timeout, 1);
        }
        phase ^= 1u;
        tc::fence_after();
        __syncthreads();   // every thread past the wait before the next chunk overwrites A and B
    }
    uint32_t d0[16], d1[16], d2[16], d3[16];   // D columns 0..31 (Yr), 32..63 (Yi)
    tc::tmem_ld16(tl + 64, d0);
    tc::tmem_ld16(tl + 80, d1);
    tc::tmem_ld16(tl + 96, d2);
    tc::tmem_ld16(tl + 112, d3);
    tc::tmem_wait_ld();
    if (i < m && !s_fail) {
#pragma unroll
        for (int c = 0; c < kTcCols; ++c) {
            if (c >= kc) break;
            const float re = __uint_as_float(c < 16 ? d0[c] : d1[c - 16]);
            const float im = __uint_as_float(c < 16 ? d2[c] : d3[c - 16]);
            const float sc = irsc * iscol[c];
            const float2 y = make_float2(re * sc, im * sc);
            if (i < nC) outC[int64_t(c0 + c) * ldC + int64_t(t) * nC + i] = y;
            else outD[int64_t(c0 + c) * ldD + int64_t(t) * (m - nC) + (i - nC)] = y;
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (tid < 32) tc::tmem_free(tmem, kTcTmem);
}

// Row maxima of the node matrices for the FP16 scales of k_ulv_tc: out[t m + i] = largest |Re|,
// |Im| of row i of W_t; out[nodes m + t m + i] = the same of row i of W_t^* (column i of W_t).
__global__ void k_ulv_rowmax(const float2* __restrict__ W, int m, int nodes, float* __restrict__ out) {
    const int t = blockIdx.x, i = blockIdx.y * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const float2* Wt = W + int64_t(t) * m * m;
    float up = 0.f, dn = 0.f;
    for (int j = 0; j < m; ++j) {
        const float2 a = Wt[i + int64_t(j) * m], b = Wt[j + int64_t(i) * m];
        up = fmaxf(up, fmaxf(fabsf(a.x), fabsf(a.y)));
        dn = fmaxf(dn, fmaxf(fabsf(b.x), fabsf(b.y)));
    }
    out[int64_t(t) * m + i] = up;
    out[int64_t(nodes) * m + int64_t(t) * m + i] = dn;
}

// Skinny node products (k <= KC <= 8 columns): one CTA of 4 x 128 threads per (node, 128 rows);
// thread (group g, row) sums over the g-th quarter of each tile of inner indices, and the four
// partial sums meet in shared memory at the end.  W is streamed from HBM once (up pass: coalesced
// column segments; down pass: each thread's own contiguous column of W, i.e. a row of W^*); x is
// staged through shared memory in tiles of 512 inner indices.
constexpr int kSkinnyJ = 512, kSkinnyG = 4;
template <bool CONJ, int KC>
__global__ void __launch_bounds__(128 * kSkinnyG) k_ulv_skinny(const float2* __restrict__ W, int m,
                                                               const float2* __restrict__ inA, int nA, int64_t ldA,
                                                               const float2* __restrict__ inB, int64_t ldB,
                                                               float2* __restrict__ outC, int nC, int64_t ldC,
                                                               float2* __restrict__ outD, int64_t ldD, int k) {
    __shared__ float2 sx[kSkinnyJ * KC];   // x tile [jj][c]; at the end the partial sums [g][row][c]
    constexpr int NTH = 128 * kSkinnyG;
    const int t = blockIdx.x, il = threadIdx.x & 127, g = threadIdx.x >> 7, i = blockIdx.y * 128 + il;
    const float2* Wt = W + int64_t(t) * m * m;
    float2 acc[KC];
#pragma unroll
    for (int c = 0; c < KC; ++c) acc[c] = make_float2(0.f, 0.f);
    for (int j0 = 0; j0 < m; j0 += kSkinnyJ) {
        const int jw = min(kSkinnyJ, m - j0);
        __syncthreads();
        for (int e = threadIdx.x; e < kSkinnyJ * KC; e += NTH) {
            const int jj = e % kSkinnyJ, c = e / kSkinnyJ, j = j0 + jj;
            float2 v = make_float2(0.f, 0.f);
            if (jj < jw && c < k)
                v = (j < nA) ? inA[int64_t(c) * ldA + int64_t(t) * nA + j]
                             : inB[int64_t(c) * ldB + int64_t(t) * (m - nA) + (j - nA)];
            sx[jj * KC + c] = v;
        }
        __syncthreads();
        const int q = (jw + kSkinnyG - 1) / kSkinnyG, jb = g * q, je = min(jw, jb + q);
        if (i < m) {
            if (!CONJ) {
                const float2* wp = Wt + i + int64_t(j0) * m;
#pragma unroll 8
                for (int jj = jb; jj < je; ++jj) {
                    const float2 w = __ldg(wp + int64_t(jj) * m);
#pragma unroll
                    for (int c = 0; c < KC; ++c) cfma(acc[c], w, sx[jj * KC + c]);
                }
            } else {
                const float2* wp = Wt + int64_t(i) * m + j0;
#pragma unroll 8
                for (int jj = jb; jj < je; ++jj) {
                    const float2 w = __ldg(wp + jj);
#pragma unroll
                    for (int c = 0; c < KC; ++c) cfmac(acc[c], w, sx[jj * KC + c]);
                }
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < KC; ++c) sx[(g * 128 + il) * KC + c] = acc[c];
    __syncthreads();
    if (g != 0 || i >= m) return;
#pragma unroll
    for (int c = 0; c < KC; ++c) {
        if (c >= k) break;
        float2 v = sx[il * KC + c];
#pragma unroll
        for (int gg = 1; gg < kSkinnyG; ++gg) v = cadd(v, sx[(gg * 128 + il) * KC + c]);
        if (i < nC) outC[int64_t(c) * ldC + int64_t(t) * nC + i] = v;
        else outD[int64_t(c) * ldD + int64_t(t) * (m - nC) + (i - nC)] = v;
    }
}

// The small upper levels of a solve with few columns in one CTA: up pass of levels lu..1, the root
// product c_0 = Rinv y_0 and the down pass of levels 1..lu, one output element per thread and
// step (dot products straight from the W blocks), a barrier between levels.
constexpr int kUpperMaxLevels = 32;
struct UpperArgs {
    const float2* W[kUpperMaxLevels];
    int m[kUpperMaxLevels], r[kUpperMaxLevels];
    int64_t ob[kUpperMaxLevels], oy[kUpperMaxLevels], oc[kUpperMaxLevels], rows[kUpperMaxLevels];
    const float2* Rinv;
    int m0, lu, k;
    float2* w;   // solve workspace; vectors at offsets (ob, oy, oc) x k
};
__global__ void __launch_bounds__(1024) k_ulv_upper(const UpperArgs a) {
    const int tid = threadIdx.x, nt = blockDim.x, k = a.k;
    auto bh = [&](int l) { return a.w + a.ob[l] * k; };
    auto yv = [&](int l) { return a.w + a.oy[l] * k; };
    auto cv = [&](int l) { return a.w + a.oc[l] * k; };
    for (int l = a.lu; l >= 1; --l) {   // z = W_t y_t: rows [0, m - r) to b^_1, [m - r, m) to y_{l-1}
        const int m = a.m[l], r = a.r[l], nn = 1 << l;
        if (m > 0) {
            const float2* in = yv(l);
            const int64_t ldin = a.rows[l], nb = max(int64_t(nn) * (m - r), int64_t(1));
            const int64_t ldy = max(a.rows[l - 1], int64_t(1));
            const float2* Wl = a.W[l];
            for (int e = tid; e < nn * m * k; e += nt) {
                const int i = e % m, rest = e / m, t = rest % nn, c = rest / nn;
                const float2* Wt = Wl + int64_t(t) * m * m;
                const float2* x = in + int64_t(c) * ldin + int64_t(t) * m;
                float2 acc = make_float2(0.f, 0.f);
                for (int j = 0; j < m; ++j) cfma(acc, Wt[i + int64_t(j) * m], x[j]);
                if (i < m - r) bh(l)[int64_t(c) * nb + int64_t(t) * (m - r) + i] = acc;
                else yv(l - 1)[int64_t(c) * ldy + int64_t(t) * r + (i - (m - r))] = acc;
            }
        }
        __syncthreads();
    }
    for (int e = tid; e < a.m0 * k; e += nt) {
        const int i = e % a.m0, c = e / a.m0;
        float2 acc = make_float2(0.f, 0.f);
        for (int j = 0; j < a.m0; ++j) cfma(acc, a.Rinv[i + int64_t(j) * a.m0], yv(0)[int64_t(c) * a.m0 + j]);
        cv(0)[int64_t(c) * a.m0 + i] = acc;
    }
    __syncthreads();
    for (int l = 1; l <= a.lu; ++l) {   // c_t = W_t^* [b^_1; c_2] -> c_l
        const int m = a.m[l], r = a.r[l], nn = 1 << l;
        if (m > 0) {
            const int64_t nb = max(int64_t(nn) * (m - r), int64_t(1)), ldp = max(a.rows[l - 1], int64_t(1));
            const int64_t ldo = a.rows[l];
            const float2* Wl = a.W[l];
            for (int e = tid; e < nn * m * k; e += nt) {
                const int i = e % m, rest = e / m, t = rest % nn, c = rest / nn;
                const float2* Wt = Wl + int64_t(t) * m * m + int64_t(i) * m;
                const float2* x1 = bh(l) + int64_t(c) * nb + int64_t(t) * (m - r);
                const float2* x2 = cv(l - 1) + int64_t(c) * ldp + int64_t(t) * r;
                float2 acc = make_float2(0.f, 0.f);
                for (int j = 0; j < m - r; ++j) cfmac(acc, Wt[j], x1[j]);
                for (int j = m - r; j < m; ++j) cfmac(acc, Wt[j], x2[j - (m - r)]);
                cv(l)[int64_t(c) * ldo + int64_t(t) * m + i] = acc;
            }
        }
        __syncthreads();
    }
}

constexpr int kSkinnyMaxK = 8;

// Inner-index slices of a wide node product: enough CTAs for two waves on nsms SMs, slices of at
// least 128 indices.
int wide_cb(int k) { return k <= 16 ? 16 : (k <= 32 ? 32 : 64); }
int wide_nsplit(int m, int k, int nodes, int nsms) {
    const int64_t ctas = int64_t(nodes) * cdiv(m, kWideRows) * cdiv(k, wide_cb(k));
    if (ctas >= 2 * nsms) return 1;
    const int ns = int(std::min<int64_t>(cdiv(2 * nsms, ctas), std::max(1, m / 128)));
    const int jslice = kWideJ * cdiv(cdiv(m, ns), kWideJ);
    return cdiv(m, jslice);
}

// The node products of one solve level with the kernel that suits k: skinny (k <= 8), tensor
// cores (tc: 1 FP16 parts, 2 BF16 parts; 32 <= m <= 512), wide CUDA-core products (m >= 32),
// else the tiled k_ulv_node_gemm.
// part: scratch of at least wide_nsplit(m, k, nodes, nsms) * k * nodes * m complex.
template <bool CONJ>
fio_status node_products(const char* name, const float2* W, const float* Wmx, int m, const float2* inA, int nA,
                         int64_t ldA, const float2* inB, int64_t ldB, float2* outC, int nC, int64_t ldC, float2* outD,
                         int64_t ldD, int k, int nodes, float2* part, int nsms, int tc, cudaStream_t st) {
    if (k > kSkinnyMaxK && tc && Wmx && m >= 32 && m <= kTcMaxM) {
        const dim3 g(nodes, cdiv(k, kTcCols), cdiv(m, 128));
        if (tc == 2)
            FIO_LAUNCH(name, st, (k_ulv_tc<CONJ, true><<<g, 128, kTcSmem, st>>>(W, Wmx, m, inA, nA, ldA, inB, ldB, outC, nC, ldC, outD, ldD, k)));
        else
            FIO_LAUNCH(name, st, (k_ulv_tc<CONJ, false><<<g, 128, kTcSmem, st>>>(W, Wmx, m, inA, nA, ldA, inB, ldB, outC, nC, ldC, outD, ldD, k)));
    } else if (k <= kSkinnyMaxK) {
        const dim3 g(nodes, cdiv(m, 128));
        if (k == 1)
            FIO_LAUNCH(name, st, (k_ulv_skinny<CONJ, 1><<<g, 128 * kSkinnyG, 0, st>>>(W, m, inA, nA, ldA, inB, ldB, outC, nC, ldC, outD, ldD, k)));
        else if (k == 2)
            FIO_LAUNCH(name, st, (k_ulv_skinny<CONJ, 2><<<g, 128 * kSkinnyG, 0, st>>>(W, m, inA, nA, ldA, inB, ldB, outC, nC, ldC, outD, ldD, k)));
        else if (k <= 4)
            FIO_LAUNCH(name, st, (k_ulv_skinny<CONJ, 4><<<g, 128 * kSkinnyG, 0, st>>>(W, m, inA, nA, ldA, inB, ldB, outC, nC, ldC, outD, ldD, k)));
        else
            FIO_LAUNCH(name, st, (k_ulv_skinny<CONJ, 8><<<g, 128 * kSkinnyG, 0, st>>>(W, m, inA, nA, ldA, inB, ldB, outC, nC, ldC, outD, ldD, k)));
    } else if (m >= 32) {
        // columns per CTA to suit k; inner-index slices until the grid covers two waves of SMs
        const int CB = wide_cb(k);
        const int rb = cdiv(m, kWideRows), cbn = cdiv(k, CB);
        const int nsplit = wide_nsplit(m, k, nodes, nsms);
        const int jslice = kWideJ * cdiv(cdiv(m, nsplit), kWideJ);
        const dim3 g(nodes, cbn * nsplit, rb);
        if (CB == 16)
            FIO_LAUNCH(name, st, (k_ulv_wide<CONJ, 16><<<g, 256, 0, st>>>(W, m, inA, nA, ldA, inB, ldB, outC, nC, ldC, outD, ldD, k, nsplit, jslice, part)));
        else if (CB == 32)
            FIO_LAUNCH(name, st, (k_ulv_wide<CONJ, 32><<<g, 256, 0, st>>>(W, m, inA, nA, ldA, inB, ldB, outC, nC, ldC, outD, ldD, k, nsplit, jslice, part)));
        else
            FIO_LAUNCH(name, st, (k_ulv_wide<CONJ, 64><<<g, 256, 0, st>>>(W, m, inA, nA, ldA, inB, ldB, outC, nC, ldC, outD, ldD, k, nsplit, jslice, part)));
        if (nsplit > 1) {
            const int64_t per = int64_t(k) * nodes * m;
            FIO_LAUNCH("k_ulv_reduce", st, (k_ulv_wide_reduce<<<cdiv(per, 256), 256, 0, st>>>(part, nsplit, nodes, m, k, outC, nC, ldC, outD, ldD)));
        }
    } else {
        const dim3 g(nodes, (k + KCOL - 1) / KCOL, (m + RB - 1) / RB);
        FIO_LAUNCH(name, st, (k_ulv_node_gemm<CONJ><<<g, 256, 0, st>>>(W, m, inA, nA, ldA, inB, ldB, outC, nC, ldC, outD, ldD, k)));
    }
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}

// Grouped node products: CTA b runs item (descriptor, node, first column, first row).
template <bool CONJ>
__global__ void __launch_bounds__(256) k_ulv_node_gemm_group(const UlvGemmDesc* __restrict__ d,
                                                             const int4* __restrict__ items) {
    const int4 it = items[blockIdx.x];
    const UlvGemmDesc& g = d[it.x];
    node_gemm_body<CONJ>(g.W, g.m, g.inA, g.nA, g.ldA, g.inB, g.ldB, g.outC, g.nC, g.ldC, g.outD, g.ldD, g.k, it.y,
                         it.z, it.w);
}

// Grouped root products c = Rinv y, one CTA per descriptor.
__global__ void k_root_group(const UlvRootDesc* __restrict__ d) {
    const UlvRootDesc& g = d[blockIdx.x];
    ulvb::root_body(g.A, g.m, g.x, g.y, g.k, int(threadIdx.x));
}

__global__ void k_gemv_sq(const float2* __restrict__ A, int m, const float2* __restrict__ x, int64_t ldx,
                          float2* __restrict__ y, int64_t ldy) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int col = blockIdx.y;
    if (i >= m) return;
    float2 a = make_float2(0.f, 0.f);
    for (int j = 0; j < m; ++j) cfma(a, A[i + int64_t(j) * m], x[col * ldx + j]);
    y[col * ldy + i] = a;
}

template <class C>
fio_status factor_level(fio_hss* h, int l, const C* Dc, const C* Uc, DevBuf& scr, DevBuf& dh22, DevBuf& uh2,
                        int* d_status, cudaStream_t st, BigScratch* big = nullptr) {
    const int nn = 1 << l, m = h->m(l), r = h->ranks[l];
    if (big && std::is_same<C, double2>::value && large_level(nn, m)) {
        FIO_TRY(dh22.ensure(std::max<size_t>(16, size_t(nn) * r * r * 16)));
        FIO_TRY(uh2.ensure(std::max<size_t>(16, size_t(nn) * r * r * 16)));
        FIO_TRY(h->W[l].ensure(size_t(nn) * m * m * 8));
        const double2* D = reinterpret_cast<const double2*>(Dc);
        const double2* U = reinterpret_cast<const double2*>(Uc);
        if (l == h->Lh) {   // leaf generators are complex64
            const int64_t nD = int64_t(nn) * m * m, nU = int64_t(nn) * m * r;
            FIO_TRY(scr.ensure(size_t(nD + nU) * 16 + 16));
            double2* D64 = scr.as<double2>();
            k_to_f64<float2><<<cdiv(nD, TB), TB, 0, st>>>(h->D.as<float2>(), D64, nD);
            if (nU) k_to_f64<float2><<<cdiv(nU, TB), TB, 0, st>>>(h->U[l].as<float2>(), D64 + nD, nU);
            D = D64;
            U = D64 + nD;
        }
        return big_ulv_nodes(*big, nn, m, r, D, U, h->W[l].as<float2>(), dh22.as<double2>(), uh2.as<double2>(), d_status,
                             st);
    }
    const int64_t per = 3 * int64_t(m) * m + 2 * int64_t(m) * r + r;
    FIO_TRY(scr.ensure(size_t(nn) * per * sizeof(C)));
    FIO_TRY(dh22.ensure(std::max<size_t>(16, size_t(nn) * r * r * sizeof(C))));
    FIO_TRY(uh2.ensure(std::max<size_t>(16, size_t(nn) * r * r * sizeof(C))));
    FIO_TRY(h->W[l].ensure(size_t(nn) * m * m * 8));
    const float2* Df = (l == h->Lh) ? h->D.as<float2>() : nullptr;
    const float2* Uf = (l == h->Lh) ? h->U[l].as<float2>() : nullptr;
    k_ulv_node<C><<<nn, TB, 0, st>>>(Df, Dc, Uf, Uc, m, r, h->W[l].as<float2>(), dh22.as<C>(), uh2.as<C>(), scr.as<C>(),
                                     d_status);
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}

}  // namespace
}  // namespace fio

using namespace fio;

extern "C" fio_status hss_ulv_factor(fio_hss* h, void* stream) {
    if (!h) return fail(FIO_EINVAL, "hss_ulv_factor: null handle");
    cudaStream_t st = as_stream(stream);
    const int Lh = h->Lh;
    DevBuf scr, dh22[2], uh2[2], dplus, uplus, dconv, stat;
    BigScratch* big = big_scratch_new();
    auto release = [&]() {
        for (DevBuf* b : {&scr, &dh22[0], &dh22[1], &uh2[0], &uh2[1], &dplus, &uplus, &dconv, &stat}) b->release();
        big_scratch_free(big);
        big = nullptr;
    };
    fio_status s;
    if ((s = stat.ensure(4)) != FIO_OK) { release(); return s; }
    FIO_CUDA(cudaMemsetAsync(stat.p, 0, 4, st));
    int* d_status = stat.as<int>();
    bool cur_f64 = false;
    for (int l = Lh; l >= 1; --l) {
        const int nn = 1 << l;
        const bool f64 = nn <= kFp64Nodes;
        if (h->m(l) == 0) {   // empty level: all ranks at and above it are 0
            cur_f64 = f64;
            continue;
        }
        const int r = h->ranks[l];
        int cur = l & 1;
        // inputs of this level: leaf generators, or D+/U+ of the merge (in dplus/uplus)
        if (l == Lh) {
            s = f64 ? factor_level<double2>(h, l, nullptr, nullptr, scr, dh22[cur], uh2[cur], d_status, st, big)
                    : factor_level<float2>(h, l, nullptr, nullptr, scr, dh22[cur], uh2[cur], d_status, st);
        } else if (f64 && !cur_f64) {
            // promote the merged blocks to FP64
            int64_t nD = int64_t(nn) * h->m(l) * h->m(l), nU = int64_t(nn) * h->m(l) * r;
            if ((s = dconv.ensure(size_t(nD + nU) * 16 + 16)) != FIO_OK) { release(); return s; }
            double2* D64 = dconv.as<double2>();
            double2* U64 = D64 + nD;
            if (nD) k_to_f64<float2><<<cdiv(nD, TB), TB, 0, st>>>(dplus.as<float2>(), D64, nD);
            if (nU) k_to_f64<float2><<<cdiv(nU, TB), TB, 0, st>>>(uplus.as<float2>(), U64, nU);
            s = factor_level<double2>(h, l, D64, U64, scr, dh22[cur], uh2[cur], d_status, st, big);
        } else if (f64) {
            s = factor_level<double2>(h, l, dplus.as<double2>(), uplus.as<double2>(), scr, dh22[cur], uh2[cur], d_status,
                                      st, big);
        } else {
            s = factor_level<float2>(h, l, dplus.as<float2>(), uplus.as<float2>(), scr, dh22[cur], uh2[cur], d_status, st);
        }
        if (s != FIO_OK) { release(); return s; }
        // merge into level l-1
        const int np = nn / 2, mp = 2 * r, rp = h->ranks[l - 1];
        const float2* Up = (l - 1 >= 1) ? h->U[l - 1].as<float2>() : nullptr;
        size_t es = f64 ? 16 : 8;
        DevBuf tmpD, tmpU;
        if ((s = tmpD.ensure(std::max<size_t>(16, size_t(np) * mp * mp * es))) != FIO_OK) { release(); return s; }
        if ((s = tmpU.ensure(std::max<size_t>(16, size_t(np) * mp * std::max(rp, 1) * es))) != FIO_OK) {
            tmpD.release();
            release();
            return s;
        }
        if (mp > 0) {
            s = f64 ? ulv_merge_gemm<double2>(*big, np, r, dh22[cur].as<double2>(), uh2[cur].as<double2>(),
                                              h->B[l - 1].as<float2>(), Up, rp, tmpD.as<double2>(), tmpU.as<double2>(), st)
                    : ulv_merge_gemm<float2>(*big, np, r, dh22[cur].as<float2>(), uh2[cur].as<float2>(),
                                             h->B[l - 1].as<float2>(), Up, rp, tmpD.as<float2>(), tmpU.as<float2>(), st);
            if (s != FIO_OK) {
                tmpD.release();
                tmpU.release();
                release();
                return s;
            }
        }
        cudaError_t e = cudaStreamSynchronize(st);   // the scratch buffers are reused next level
        dplus.release();
        uplus.release();
        dplus = tmpD;
        uplus = tmpU;
        cur_f64 = f64;
        if (e != cudaSuccess) { release(); return cuda_status(e, "hss_ulv_factor: level"); }
    }
    // root
    const int m0 = 2 * h->ranks[1];
    if ((s = h->Rinv.ensure(std::max<size_t>(8, size_t(m0) * m0 * 8))) != FIO_OK) { release(); return s; }
    if (m0 > 0) {
        if ((s = scr.ensure(size_t(2) * m0 * m0 * 16)) != FIO_OK) { release(); return s; }
        const double2* D64 = dplus.as<double2>();
        if (!cur_f64) {
            if ((s = dconv.ensure(size_t(m0) * m0 * 16)) != FIO_OK) { release(); return s; }
            k_to_f64<float2><<<cdiv(int64_t(m0) * m0, TB), TB, 0, st>>>(dplus.as<float2>(), dconv.as<double2>(),
                                                                        int64_t(m0) * m0);
            D64 = dconv.as<double2>();
        }
        if (large_level(1, m0)) {
            if ((s = big_ulv_root(*big, m0, D64, h->Rinv.as<float2>(), d_status, st)) != FIO_OK) { release(); return s; }
        } else {
            k_ulv_root<<<1, TB, 0, st>>>(D64, m0, h->Rinv.as<float2>(), scr.as<double2>(), d_status);
        }
    }
    int hst = 0;
    cudaMemcpyAsync(&hst, d_status, 4, cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    release();
    if (e != cudaSuccess) return cuda_status(e, "hss_ulv_factor");
    if (hst == FIO_ENOTHPD) return fail(FIO_ENOTHPD, "hss_ulv_factor: Cholesky pivot <= 0 (G~ not HPD)");
    // row maxima of the node matrices of the tensor-core solve levels
    h->Wmx.resize(Lh + 1);
    for (int l = 1; l <= Lh; ++l) {
        const int m = h->m(l), nn = 1 << l;
        if (m < 32 || m > kTcMaxM) continue;
        if ((s = h->Wmx[l].ensure(size_t(2) * nn * m * sizeof(float))) != FIO_OK) return s;
        k_ulv_rowmax<<<dim3(nn, cdiv(m, 128)), 128, 0, st>>>(h->W[l].as<float2>(), m, nn, h->Wmx[l].as<float>());
    }
    FIO_CUDA(cudaGetLastError());
    FIO_CUDA(cudaStreamSynchronize(st));
    h->factored = true;
    return FIO_OK;
}

namespace fio {
// hss_solve with the precision of the tensor-core node products (prec 0: FP16 parts, FP32
// accuracy; 1: BF16 parts), used when the handle's solve path is 1; path 0 (default) runs every
// node product on the CUDA cores in FP32.
fio_status hss_solve_prec(const fio_hss* hc, const void* Bv, void* Xv, int64_t ld, int k, int prec, cudaStream_t st) {
    if (!hc) return fail(FIO_EINVAL, "hss_solve: null handle");
    if (!hc->factored) return fail(FIO_EINVAL, "hss_solve: call hss_ulv_factor first");
    if (k < 0 || ld < hc->N) return fail(FIO_EINVAL, "hss_solve: need k >= 0 and ld >= N");
    if (k == 0) return FIO_OK;
    fio_hss* h = const_cast<fio_hss*>(hc);
    const int tc = hc->solve_path == 1 ? (prec == 1 ? 2 : 1) : 0;
    auto wmx = [&](int l) -> const float* {
        return (l < int(h->Wmx.size()) && h->Wmx[l].p) ? h->Wmx[l].as<float>() : nullptr;
    };
    static PerDeviceOnce attrs;
    FIO_CUDA(attrs.run([] {
        cudaError_t e = cudaSuccess;
        for (auto f : {(const void*)k_ulv_tc<false, false>, (const void*)k_ulv_tc<true, false>,
                       (const void*)k_ulv_tc<false, true>, (const void*)k_ulv_tc<true, true>})
            if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        return e;
    }));
    const int Lh = h->Lh;
    // per level: bh1_l (2^l (m_l - r_l)), y_l (rows(l), l < Lh), c_l (rows(l), l < Lh)
    std::vector<int64_t> ob(Lh + 1), oy(Lh + 1), oc(Lh + 1);
    int64_t tot = 0;
    for (int l = 0; l <= Lh; ++l) {
        ob[l] = tot;
        tot += (l >= 1) ? (int64_t(1) << l) * (h->m(l) - h->ranks[l]) : 0;
        oy[l] = tot;
        tot += (l < Lh) ? h->rows(l) : 0;
        oc[l] = tot;
        tot += (l < Lh) ? h->rows(l) : 0;
    }
    FIO_TRY(h->solve_ws.ensure(std::max<size_t>(16, size_t(tot) * k * 8)));
    float2* w = h->solve_ws.as<float2>();
    auto bh = [&](int l) { return w + ob[l] * k; };
    auto yv = [&](int l) { return w + oy[l] * k; };
    auto cv = [&](int l) { return w + oc[l] * k; };
    const float2* B = static_cast<const float2*>(Bv);
    float2* X = static_cast<float2*>(Xv);
    int dev = 0, nsms = 148;
    FIO_CUDA(cudaGetDevice(&dev));
    FIO_CUDA(cudaDeviceGetAttribute(&nsms, cudaDevAttrMultiProcessorCount, dev));
    int64_t part_need = 1;
    if (k > kSkinnyMaxK)
        for (int l = 1; l <= Lh; ++l) {
            const int m = h->m(l);
            if (m >= 32) part_need = std::max<int64_t>(part_need, int64_t(wide_nsplit(m, k, 1 << l, nsms)) * k * (int64_t(1) << l) * m);
        }
    FIO_TRY(h->solve_part.ensure(size_t(part_need) * 8));
    float2* part = h->solve_part.as<float2>();
    // few columns: the small upper levels (m_l <= 64) and the root run in one single-CTA launch
    const int m0 = 2 * h->ranks[1];
    int lu = 0;
    if (k <= kSkinnyMaxK && m0 <= 128 && Lh - 1 < kUpperMaxLevels) {
        int64_t work = int64_t(m0) * m0 * k;
        for (int l = 1; l < Lh; ++l) {
            const int m = h->m(l);
            work += (int64_t(1) << l) * m * m * k;
            if (m > 64 || work > (int64_t(1) << 21)) break;
            lu = l;
        }
    }
    for (int l = Lh; l > lu; --l) {
        const int m = h->m(l), r = h->ranks[l];
        if (m == 0) continue;   // every rank above this level is 0: nothing to pass up
        const float2* in = (l == Lh) ? B : yv(l);
        int64_t ldin = (l == Lh) ? ld : h->rows(l);
        int64_t nb = (int64_t(1) << l) * (m - r);
        FIO_TRY(node_products<false>("k_ulv_up", h->W[l].as<float2>(), wmx(l), m, in, m, ldin, in, ldin, bh(l), m - r,
                                     std::max<int64_t>(nb, 1), yv(l - 1), std::max<int64_t>(h->rows(l - 1), 1), k,
                                     1 << l, part, nsms, tc, st));
    }
    if (lu > 0) {
        UpperArgs ua{};
        for (int l = 1; l <= lu; ++l) {
            ua.W[l] = h->W[l].as<float2>();
            ua.m[l] = h->m(l);
            ua.r[l] = h->ranks[l];
        }
        for (int l = 0; l <= lu; ++l) {
            ua.ob[l] = ob[l];
            ua.oy[l] = oy[l];
            ua.oc[l] = oc[l];
            ua.rows[l] = h->rows(l);
        }
        ua.Rinv = h->Rinv.as<float2>();
        ua.m0 = m0;
        ua.lu = lu;
        ua.k = k;
        ua.w = w;
        FIO_LAUNCH("k_ulv_upper", st, k_ulv_upper<<<1, 1024, 0, st>>>(ua));
    } else if (m0 > 0) {
        dim3 g(cdiv(m0, TB), k);
        FIO_LAUNCH("k_ulv_root", st, k_gemv_sq<<<g, TB, 0, st>>>(h->Rinv.as<float2>(), m0, yv(0), m0, cv(0), m0));
    }
    for (int l = lu + 1; l <= Lh; ++l) {
        const int m = h->m(l), r = h->ranks[l];
        if (m == 0) continue;
        float2* out = (l == Lh) ? X : cv(l);
        int64_t ldo = (l == Lh) ? ld : h->rows(l);
        int64_t nb = (int64_t(1) << l) * (m - r);
        FIO_TRY(node_products<true>("k_ulv_down", h->W[l].as<float2>(), wmx(l), m, bh(l), m - r, std::max<int64_t>(nb, 1),
                                    cv(l - 1), std::max<int64_t>(h->rows(l - 1), 1), out, m, ldo, out, ldo, k, 1 << l,
                                    part, nsms, tc, st));
    }
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}

int ulv_tc_timeouts() {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_ulv_tc_timeout, sizeof(int)) != cudaSuccess) return -1;
    const int z = 0;
    if (v) cudaMemcpyToSymbol(g_ulv_tc_timeout, &z, sizeof(int));
    return v;
}
}  // namespace fio

extern "C" fio_status hss_solve(const fio_hss* hc, const void* Bv, void* Xv, int64_t ld, int k, void* stream) {
    return hss_solve_prec(hc, Bv, Xv, ld, k, 0, as_stream(stream));
}

extern "C" fio_status hss_set_solve_path(fio_hss* h, int path) {
    if (!h || path < 0 || path > 1) return fail(FIO_EINVAL, "hss_set_solve_path: bad handle or path");
    h->solve_path = path;
    return FIO_OK;
}

namespace fio {

// Per-level vector layout of the solve (rows of the b^_1, y and c vectors).
static int64_t solve_layout(const fio_hss* h, std::vector<int64_t>& ob, std::vector<int64_t>& oy, std::vector<int64_t>& oc) {
    const int Lh = h->Lh;
    ob.assign(Lh + 1, 0);
    oy.assign(Lh + 1, 0);
    oc.assign(Lh + 1, 0);
    int64_t tot = 0;
    for (int l = 0; l <= Lh; ++l) {
        ob[l] = tot;
        tot += (l >= 1) ? (int64_t(1) << l) * (h->m(l) - h->ranks[l]) : 0;
        oy[l] = tot;
        tot += (l < Lh) ? h->rows(l) : 0;
        oc[l] = tot;
        tot += (l < Lh) ? h->rows(l) : 0;
    }
    return tot;
}

int64_t ulv_solve_ws_elems(const fio_hss* h, int k) {
    std::vector<int64_t> ob, oy, oc;
    return std::max<int64_t>(2, solve_layout(h, ob, oy, oc) * k);
}

// The solve of one HSS handle as descriptors, on a caller-provided workspace
// of ulv_solve_ws_elems(h, k) complex64 elements.
fio_status ulv_solve_plan(fio_hss* h, const float2* B, float2* X, int64_t ld, int k, float2* w, UlvSolvePlan& plan) {
    if (!h->factored) return fail(FIO_EINVAL, "ulv_solve_plan: call hss_ulv_factor first");
    const int Lh = h->Lh;
    std::vector<int64_t> ob, oy, oc;
    solve_layout(h, ob, oy, oc);
    auto bh = [&](int l) { return w + ob[l] * k; };
    auto yv = [&](int l) { return w + oy[l] * k; };
    auto cv = [&](int l) { return w + oc[l] * k; };
    plan.up.assign(Lh + 1, UlvGemmDesc{});
    plan.down.assign(Lh + 1, UlvGemmDesc{});
    plan.Lh = Lh;
    for (int l = Lh; l >= 1; --l) {
        const int m = h->m(l), r = h->ranks[l];
        UlvGemmDesc& u = plan.up[l];
        UlvGemmDesc& d = plan.down[l];
        u.nodes = d.nodes = (m == 0) ? 0 : (1 << l);
        if (m == 0) continue;
        const int64_t nb = (int64_t(1) << l) * (m - r);
        const float2* in = (l == Lh) ? B : yv(l);
        const int64_t ldin = (l == Lh) ? ld : h->rows(l);
        u.W = d.W = h->W[l].as<float2>();
        u.m = d.m = m;
        u.k = d.k = k;
        u.inA = in; u.nA = m; u.ldA = ldin; u.inB = in; u.ldB = ldin;
        u.outC = bh(l); u.nC = m - r; u.ldC = std::max<int64_t>(nb, 1);
        u.outD = yv(l - 1); u.ldD = std::max<int64_t>(h->rows(l - 1), 1);
        float2* out = (l == Lh) ? X : cv(l);
        const int64_t ldo = (l == Lh) ? ld : h->rows(l);
        d.inA = bh(l); d.nA = m - r; d.ldA = std::max<int64_t>(nb, 1);
        d.inB = cv(l - 1); d.ldB = std::max<int64_t>(h->rows(l - 1), 1);
        d.outC = out; d.nC = m; d.ldC = ldo; d.outD = out; d.ldD = ldo;
    }
    plan.root = UlvRootDesc{h->Rinv.as<float2>(), yv(0), cv(0), 2 * h->ranks[1], k};
    return FIO_OK;
}

void ulv_gemm_items(const UlvGemmDesc& d, int di, std::vector<int4>& items) {
    for (int t = 0; t < d.nodes; ++t)
        for (int c0 = 0; c0 < d.k; c0 += KCOL)
            for (int r0 = 0; r0 < d.m; r0 += RB) items.push_back(make_int4(di, t, c0, r0));
}

fio_status ulv_group_launch(const UlvGemmDesc* dd, const int4* ditems, int nitems, bool down, cudaStream_t st) {
    if (nitems == 0) return FIO_OK;
    if (down) FIO_LAUNCH("k_ulv_down_group", st, k_ulv_node_gemm_group<true><<<nitems, 256, 0, st>>>(dd, ditems));
    else FIO_LAUNCH("k_ulv_up_group", st, k_ulv_node_gemm_group<false><<<nitems, 256, 0, st>>>(dd, ditems));
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}

fio_status ulv_root_group_launch(const UlvRootDesc* dd, int n, cudaStream_t st) {
    if (n == 0) return FIO_OK;
    FIO_LAUNCH("k_ulv_root_group", st, k_root_group<<<n, 256, 0, st>>>(dd));
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}

}  // namespace fio
