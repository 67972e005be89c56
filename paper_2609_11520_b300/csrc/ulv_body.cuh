// Node products of the ULV solve (Section 2.4), shared by the solve kernels
// and the persistent batched kernel.
#pragma once
#include "common.cuh"

namespace fio {
namespace ulvb {

// Batched node products of the solve, one CTA per (node, chunk of KCOL
// columns, block of 256 output rows):
//   up:   z = W_t y_t                 (CONJ = false)
//   down: c = W_t^* [bh1_t; c2_t]     (CONJ = true)
// The m-vector of a node is split into rows [0, nA) read from inA (node
// offset t*nA) and rows [nA, m) from inB (node offset t*(m-nA)); the result
// into rows [0, nC) of outC (offset t*nC) and [nC, m) of outD (offset
// t*(m-nC)).  W (column-major m x m) and x are staged through shared memory
// in tiles of WT inner indices; each thread owns rows i0 + 32 q of its row
// block and two columns.
constexpr int KCOL = 16;
constexpr int WT = 32;
constexpr int RB = 128;   // rows per CTA: 4 per thread

// Run by kUlvThreads threads numbered tid = 0 .. 255; sx (WT * KCOL) and sw (WT * RB) are the
// caller's shared-memory tiles and sync() a barrier over exactly those threads.
constexpr int kUlvThreads = 256;
template <bool CONJ, class Sync>
__device__ void node_gemm_body(const float2* __restrict__ W, int m, const float2* __restrict__ inA, int nA, int64_t ldA,
                               const float2* __restrict__ inB, int64_t ldB, float2* __restrict__ outC, int nC,
                               int64_t ldC, float2* __restrict__ outD, int64_t ldD, int k, int t, int c0, int r0,
                               float2* __restrict__ sx, float2* __restrict__ sw, Sync sync, int tid) {
    const int kc = min(KCOL, k - c0), nr = min(RB, m - r0);
    const float2* Wt = W + int64_t(t) * m * m;
    const int i0 = tid & 31, cg = tid >> 5;   // 8 column groups of 2
    float2 acc[RB / 32][2];
#pragma unroll
    for (int q = 0; q < RB / 32; ++q) acc[q][0] = acc[q][1] = make_float2(0.f, 0.f);
    for (int j0 = 0; j0 < m; j0 += WT) {
        const int jw = min(WT, m - j0);
        sync();
        for (int e = tid; e < WT * KCOL; e += kUlvThreads) {
            const int jj = e / KCOL, c = e % KCOL, j = j0 + jj;
            float2 v = make_float2(0.f, 0.f);
            if (jj < jw && c < kc)
                v = (j < nA) ? inA[int64_t(c0 + c) * ldA + int64_t(t) * nA + j]
                             : inB[int64_t(c0 + c) * ldB + int64_t(t) * (m - nA) + (j - nA)];
            sx[e] = v;
        }
        for (int e = tid; e < jw * nr; e += kUlvThreads) {
            int jj, il;
            float2 v;
            if (!CONJ) {   // columns j of W, rows r0..: W[i + j m]
                il = e % nr;
                jj = e / nr;
                v = Wt[(r0 + il) + int64_t(j0 + jj) * m];
            } else {       // rows j of W, columns r0..: W[j + i m]
                jj = e % jw;
                il = e / jw;
                v = Wt[(j0 + jj) + int64_t(r0 + il) * m];
            }
            sw[jj * RB + il] = v;
        }
        sync();
        for (int jj = 0; jj < jw; ++jj) {
            const float2 x0 = sx[jj * KCOL + 2 * cg], x1 = sx[jj * KCOL + 2 * cg + 1];
#pragma unroll
            for (int q = 0; q < RB / 32; ++q) {
                const int il = i0 + 32 * q;
                if (il < nr) {
                    const float2 w = sw[jj * RB + il];
                    if (CONJ) {
                        cfmac(acc[q][0], w, x0);
                        cfmac(acc[q][1], w, x1);
                    } else {
                        cfma(acc[q][0], w, x0);
                        cfma(acc[q][1], w, x1);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < RB / 32; ++q) {
        const int il = i0 + 32 * q;
        if (il >= nr) continue;
        const int i = r0 + il;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int c = 2 * cg + u;
            if (c >= kc) continue;
            if (i < nC) outC[int64_t(c0 + c) * ldC + int64_t(t) * nC + i] = acc[q][u];
            else outD[int64_t(c0 + c) * ldD + int64_t(t) * (m - nC) + (i - nC)] = acc[q][u];
        }
    }
}

// Root product y = A x (m x m times m x k), threads tid = 0 .. 255.
__device__ __forceinline__ void root_body(const float2* __restrict__ A, int m, const float2* __restrict__ x,
                                          float2* __restrict__ y, int k, int tid) {
    for (int e = tid; e < m * k; e += kUlvThreads) {
        const int i = e % m, col = e / m;
        float2 a = make_float2(0.f, 0.f);
        for (int j = 0; j < m; ++j) cfma(a, A[i + int64_t(j) * m], x[int64_t(col) * m + j]);
        y[int64_t(col) * m + i] = a;
    }
}

}  // namespace ulvb
}  // namespace fio
