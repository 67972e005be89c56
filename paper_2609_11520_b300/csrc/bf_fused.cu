// Fused two-pass butterfly apply (r = 16), the B300 form of Eq. 2.1.
//
// The butterfly splits at the middle level h into two independent halves:
//   left half  (space side):     U, B^[h+1..T]  -- one CTA per space box tau_h
//                                (2^(L-h) pairs, all frequency boxes sigma)
//   right half (frequency side): C^[h+1..T], V  -- one CTA per frequency box
//                                sigma_h (2^h pairs, all space boxes tau)
// K~^* x: left half (U^*, B^*, M^*) -> middle state -> right half (C^*, V^*).
// K~ x:   right half (V, C, M)      -> middle state -> left half (B, U).
// Inside a CTA the coefficient state of KC columns stays in shared memory;
// only the input vectors, the middle state (N r complex per column) and the
// output vectors cross HBM, and every factor table is read once per CTA.
//
// In-place transfer levels: a quad (two input pairs -> two output pairs)
// keeps the two physical slots of its inputs for its outputs.  A pair's
// physical slot is then a partial bit reversal of its logical index; for a
// half with W = number of free frequency (left) / space (right) bits at level
// s and j transfer levels between s and the half's outer end:
//   phys_s(a, b) = a 2^W + rev_j(b mod 2^j) 2^(W-j) + (b >> j),
// and the quad of level s acts on the slot pair {base, base + 2^(W-1)} with
//   base = a 2^W + rev_(j-1)(s' mod 2^(j-1)) 2^(W-j) + (s' >> (j-1)).
// Threads enumerate quads by physical slot, so that consecutive threads touch
// consecutive slots, and shared memory is XOR-swizzled in 16-byte chunks.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>

#include "bf.cuh"
#include "hss.cuh"
#include "tc.cuh"
#include "ulv_body.cuh"

namespace fio {
namespace {

constexpr int R = 16;
// Pc[c] blocks in shared memory are PCS floats apart: the two blocks that the
// lanes of a warp read together fall into different banks.
constexpr int PCS = R * R + 4;
// Leaf Lagrange tables in shared memory: rows of RS floats (lanes that read
// different rows of one column hit different banks); at most kLeafMax rows
// (8 points per leaf box, Section 5.2's practical top level).
constexpr int RS = R + 1;
constexpr int kLeafMax = 8;

struct Tabs {
    const float2* t[24];
};

__device__ __forceinline__ int rev_bits(int x, int bits) { return bits > 0 ? int(__brev(unsigned(x)) >> (32 - bits)) : 0; }

// float2 offset of coefficient i of physical pair slot p (16-byte chunks XOR-swizzled)
__device__ __forceinline__ int sw(int p, int i) { return p * R + ((((i >> 1) ^ (p & 7)) << 1) | (i & 1)); }

__device__ __forceinline__ void load_pair(const float2* S, int p, float2 (&x)[R]) {
#pragma unroll
    for (int m = 0; m < R / 2; ++m) {
        float4 v = *reinterpret_cast<const float4*>(S + p * R + ((m ^ (p & 7)) << 1));
        x[2 * m] = make_float2(v.x, v.y);
        x[2 * m + 1] = make_float2(v.z, v.w);
    }
}
__device__ __forceinline__ void store_pair(float2* S, int p, const float2 (&y)[R]) {
#pragma unroll
    for (int m = 0; m < R / 2; ++m)
        *reinterpret_cast<float4*>(S + p * R + ((m ^ (p & 7)) << 1)) =
            make_float4(y[2 * m].x, y[2 * m].y, y[2 * m + 1].x, y[2 * m + 1].y);
}
__device__ __forceinline__ void load_row(const float2* __restrict__ g, float2 (&v)[R]) {
#pragma unroll
    for (int m = 0; m < R / 2; ++m) {
        float4 a = __ldg(reinterpret_cast<const float4*>(g) + m);
        v[2 * m] = make_float2(a.x, a.y);
        v[2 * m + 1] = make_float2(a.z, a.w);
    }
}

// One transfer level of a half on KC columns of in-place state.
//   MS ("mix, then scale"):  y[o][i] = sum_e Phi(o,e,i) sum_t Pc[o][i][t] x[e][t]
//   SM ("scale, then mix"):  y[o][j] = sum_e sum_t Pc[e][t][j] Phi(o,e,t) x[e][t]
//   Phi(o,e,.) = T[q][o][e][.] (forward) or conj(T[q][e][o][.]) (adjoint).
// LEFT selects the slot/table geometry of the space-side half.
template <int KC, bool LEFT, bool MS, bool ADJ>
__device__ void level_op(float2* S, int P, const float* sPc, const float2* __restrict__ T, int box, int s, int L,
                         int h, int sU) {
    const int W = LEFT ? L - s : h - s;
    const int j = LEFT ? sU - s : h - s;
    const int half = 1 << (W - 1);
    const int ntask = P * KC;
    for (int b0 = 0; b0 < ntask; b0 += blockDim.x) {
        const int id = b0 + threadIdx.x;
        const bool act = id < ntask;
        int col = 0, o = 0, base = 0;
        int64_t q = 0;
        float2 x0[R], x1[R];
        if (act) {
            col = id / P;
            const int rem = id - col * P;
            const int qi = rem >> 1;
            o = rem & 1;
            const int a = qi >> (W - 1), rr = qi & (half - 1);
            base = (a << W) | rr;
            if (LEFT) {
                const int wj = W - j;   // = L - sU
                const int sg = ((rr & ((1 << wj) - 1)) << (j - 1)) | rev_bits(rr >> wj, j - 1);
                q = ((int64_t(box) << (s - h)) + a) * (int64_t(1) << (L - s - 1)) + sg;
            } else {
                const int sl = rev_bits(rr, W - 1);
                q = (int64_t(box) << (h - 1)) + (int64_t(a) << (h - s - 1)) + sl;
            }
            const float2* Sc = S + col * P * R;
            load_pair(Sc, base, x0);
            load_pair(Sc, base + half, x1);
        }
        __syncwarp();
        if (act) {
            float2* Sc = S + col * P * R;
            float2 y[R];
            const float2* tq = T + q * 4 * R;
            if (MS) {
                float2 ph0[R], ph1[R];
                if (!ADJ) {
                    load_row(tq + (o * 2 + 0) * R, ph0);
                    load_row(tq + (o * 2 + 1) * R, ph1);
                } else {
                    load_row(tq + (0 * 2 + o) * R, ph0);
                    load_row(tq + (1 * 2 + o) * R, ph1);
                }
                const float* Po = sPc + o * PCS;
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    float2 h0 = make_float2(0.f, 0.f), h1 = make_float2(0.f, 0.f);
#pragma unroll
                    for (int t4 = 0; t4 < R / 4; ++t4) {
                        float4 pv = *reinterpret_cast<const float4*>(Po + i * R + 4 * t4);
                        float pp[4] = {pv.x, pv.y, pv.z, pv.w};
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int t = 4 * t4 + u;
                            h0.x = fmaf(pp[u], x0[t].x, h0.x);
                            h0.y = fmaf(pp[u], x0[t].y, h0.y);
                            h1.x = fmaf(pp[u], x1[t].x, h1.x);
                            h1.y = fmaf(pp[u], x1[t].y, h1.y);
                        }
                    }
                    float2 acc = make_float2(0.f, 0.f);
                    if (!ADJ) {
                        cfma(acc, ph0[i], h0);
                        cfma(acc, ph1[i], h1);
                    } else {
                        cfmac(acc, ph0[i], h0);
                        cfmac(acc, ph1[i], h1);
                    }
                    y[i] = acc;
                }
            } else {
#pragma unroll
                for (int jj = 0; jj < R; ++jj) y[jj] = make_float2(0.f, 0.f);
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    float2 ph[R];
                    if (!ADJ) load_row(tq + (o * 2 + e) * R, ph);
                    else load_row(tq + (e * 2 + o) * R, ph);
                    const float* Pe = sPc + e * PCS;
#pragma unroll
                    for (int t = 0; t < R; ++t) {
                        const float2 xv = e ? x1[t] : x0[t];
                        const float2 g = ADJ ? cmulc(ph[t], xv) : cmul(ph[t], xv);
#pragma unroll
                        for (int j4 = 0; j4 < R / 4; ++j4) {
                            float4 pv = *reinterpret_cast<const float4*>(Pe + t * R + 4 * j4);
                            y[4 * j4 + 0].x = fmaf(pv.x, g.x, y[4 * j4 + 0].x);
                            y[4 * j4 + 0].y = fmaf(pv.x, g.y, y[4 * j4 + 0].y);
                            y[4 * j4 + 1].x = fmaf(pv.y, g.x, y[4 * j4 + 1].x);
                            y[4 * j4 + 1].y = fmaf(pv.y, g.y, y[4 * j4 + 1].y);
                            y[4 * j4 + 2].x = fmaf(pv.z, g.x, y[4 * j4 + 2].x);
                            y[4 * j4 + 2].y = fmaf(pv.z, g.y, y[4 * j4 + 2].y);
                            y[4 * j4 + 3].x = fmaf(pv.w, g.x, y[4 * j4 + 3].x);
                            y[4 * j4 + 3].y = fmaf(pv.w, g.y, y[4 * j4 + 3].y);
                        }
                    }
                }
            }
            store_pair(Sc, o ? base + half : base, y);
        }
    }
    __syncthreads();
}

// M (forward) / M^* (adjoint) on every pair of the CTA, in place.  `phys`
// maps the logical pair index (within the CTA) to its slot; `pg` the global pair.
template <int KC, bool ADJ, bool LEFT>
__device__ void middle_op(float2* S, int P, const float2* __restrict__ M, int box, int L, int h, int sU) {
    const int ntask = P * KC;
    const int nB = sU - h;
    for (int id = threadIdx.x; id < ntask; id += blockDim.x) {
        const int col = id / P, lp = id - col * P;
        // threads run over physical slots (consecutive slots: no bank conflicts)
        const int slot = lp;
        int64_t pg;
        if (LEFT) {   // slot -> logical sigma (inverse of the inner-end layout of the left half)
            const int lo = L - sU;
            const int sg = ((slot & ((1 << lo) - 1)) << nB) | rev_bits(slot >> lo, nB);
            pg = int64_t(box) * P + sg;
        } else {      // logical tau = slot
            pg = int64_t(slot) * (int64_t(1) << (L - h)) + box;
        }
        float2* Sc = S + col * P * R;
        float2 x[R], y[R];
        load_pair(Sc, slot, x);
        const float2* Mp = M + pg * R * R;
        if (!ADJ) {
#pragma unroll
            for (int i = 0; i < R; ++i) {
                float2 row[R];
                load_row(Mp + i * R, row);
                float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                for (int jj = 0; jj < R; ++jj) cfma(acc, row[jj], x[jj]);
                y[i] = acc;
            }
        } else {
#pragma unroll
            for (int jj = 0; jj < R; ++jj) y[jj] = make_float2(0.f, 0.f);
#pragma unroll
            for (int i = 0; i < R; ++i) {
                float2 row[R];
                load_row(Mp + i * R, row);
#pragma unroll
                for (int jj = 0; jj < R; ++jj) cfmac(y[jj], row[jj], x[i]);
            }
        }
        store_pair(Sc, slot, y);
    }
    __syncthreads();
}

struct HalfArgs {
    const float2* X;     // outer input vectors (N x k, ld) or middle state
    int64_t ldx;
    float2* Y;           // outer output vectors or middle state
    int64_t ldy;
    float2* mid;         // middle state [col][N][R]
    const float2* VP;
    const float2* UP;
    const float2* M;
    const float* P;      // PV | PU | Pc
    int pu_off, pc_off;
    Tabs tab;            // left: E tables by s - h ; right: F tables by s - sV
    Tabs tabs;           // the same tables pre-arranged in the staged shared-memory layout of this
                         // direction (box-major slices of P * 256 B), or null: copied by TMA
    const float2* Ms;    // right half, forward: M pre-arranged in the staged layout, or null
    int n, L, h, sU, sV, k;
    int mode;            // transfer levels of the staged kernels: kSimt, kTcF16 or kTcBF16
};

// Left half, one CTA per space box tau_h (blockIdx.x) and KC columns (blockIdx.y).
// ADJ: g -> U^* -> B^* levels -> M^* -> middle.   !ADJ: middle -> B levels -> U -> y.
template <int KC, bool ADJ>
__global__ void __launch_bounds__(256, 2) k_bf_left(HalfArgs a) {
    extern __shared__ float4 smem4[];
    float2* S = reinterpret_cast<float2*>(smem4);
    const int L = a.L, h = a.h, sU = a.sU;
    const int P = 1 << (L - h);
    float* sPc = reinterpret_cast<float*>(S + KC * P * R);
    float* sPU = sPc + 2 * PCS;
    const int lsU = 1 << (L - sU), nbU = lsU;
    for (int e = threadIdx.x; e < 2 * R * R; e += blockDim.x) sPc[(e / (R * R)) * PCS + e % (R * R)] = a.P[a.pc_off + e];
    for (int e = threadIdx.x; e < lsU * R; e += blockDim.x) sPU[e] = a.P[a.pu_off + e];
    const int box = blockIdx.y, col0 = blockIdx.x * KC;
    const int kc = min(KC, a.k - col0);
    __syncthreads();
    if (ADJ) {
        // U^*: d(leaf, b, i) = sum_q PU[q][i] conj(UP[x_q][b]) g(x_q)
        for (int id = threadIdx.x; id < P * KC; id += blockDim.x) {
            const int col = id / P, lp = id - col * P;
            if (col >= kc) continue;
            const int leaf = lp / nbU, b = lp - leaf * nbU;
            const int64_t x0 = int64_t(box) * P + int64_t(leaf) * lsU;
            const float2* g = a.X + int64_t(col0 + col) * a.ldx + x0;
            float2 y[R];
#pragma unroll
            for (int i = 0; i < R; ++i) y[i] = make_float2(0.f, 0.f);
            for (int qq = 0; qq < lsU; ++qq) {
                const float2 m = cmulc(__ldg(a.UP + (x0 + qq) * nbU + b), g[qq]);
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    const float pu = sPU[qq * R + i];
                    y[i].x = fmaf(pu, m.x, y[i].x);
                    y[i].y = fmaf(pu, m.y, y[i].y);
                }
            }
            store_pair(S + col * P * R, lp, y);
        }
        __syncthreads();
        for (int s = sU - 1; s >= h; --s)
            level_op<KC, true, false, true>(S, P, sPc, a.tab.t[s - h], box, s, L, h, sU);
        middle_op<KC, true, true>(S, P, a.M, box, L, h, sU);
        // middle state out (logical sigma order)
        const int nB = sU - h;
        for (int id = threadIdx.x; id < P * R * KC; id += blockDim.x) {
            const int col = id / (P * R), rem = id - col * P * R, lp = rem / R, i = rem % R;
            if (col >= kc) continue;
            const int slot = (rev_bits(lp & ((1 << nB) - 1), nB) << (L - sU)) | (lp >> nB);
            a.mid[(int64_t(col0 + col) * a.n + int64_t(box) * P + lp) * R + i] = S[col * P * R + sw(slot, i)];
        }
    } else {
        const int nB = sU - h;
        for (int id = threadIdx.x; id < P * R * KC; id += blockDim.x) {
            const int col = id / (P * R), rem = id - col * P * R, lp = rem / R, i = rem % R;
            if (col >= kc) continue;
            const int slot = (rev_bits(lp & ((1 << nB) - 1), nB) << (L - sU)) | (lp >> nB);
            S[col * P * R + sw(slot, i)] = a.mid[(int64_t(col0 + col) * a.n + int64_t(box) * P + lp) * R + i];
        }
        __syncthreads();
        for (int s = h; s < sU; ++s)
            level_op<KC, true, true, false>(S, P, sPc, a.tab.t[s - h], box, s, L, h, sU);
        // U: y(x) = sum_b UP[x][b] sum_i PU[q][i] d(leaf, b, i)
        for (int id = threadIdx.x; id < P * KC; id += blockDim.x) {
            const int col = id / P, xl = id - col * P;
            if (col >= kc) continue;
            const int leaf = xl / lsU, qq = xl - leaf * lsU;
            const int64_t xg = int64_t(box) * P + xl;
            const float2* Sc = S + col * P * R;
            float2 up[kLeafMax];
#pragma unroll
            for (int b = 0; b < kLeafMax; ++b)
                if (b < nbU) up[b] = __ldg(a.UP + xg * nbU + b);
            float2 out = make_float2(0.f, 0.f);
#pragma unroll
            for (int b = 0; b < kLeafMax; ++b) {
                if (b >= nbU) break;
                float2 d[R];
                load_pair(Sc, leaf * nbU + b, d);
                float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    const float pu = sPU[qq * R + i];
                    acc.x = fmaf(pu, d[i].x, acc.x);
                    acc.y = fmaf(pu, d[i].y, acc.y);
                }
                cfma(out, up[b], acc);
            }
            a.Y[int64_t(col0 + col) * a.ldy + xg] = out;
        }
    }
}

// Right half, one CTA per frequency box sigma_h (blockIdx.x) and KC columns.
// ADJ: middle -> C^* levels -> V^* -> f.   !ADJ: f -> V -> C levels -> M -> middle.
template <int KC, bool ADJ>
__global__ void __launch_bounds__(256, 2) k_bf_right(HalfArgs a) {
    extern __shared__ float4 smem4[];
    float2* S = reinterpret_cast<float2*>(smem4);
    const int L = a.L, h = a.h, sV = a.sV;
    const int P = 1 << h;
    float* sPc = reinterpret_cast<float*>(S + KC * P * R);
    float* sPV = sPc + 2 * PCS;
    const int lsV = 1 << sV, na = 1 << sV, nl = 1 << (h - sV);
    for (int e = threadIdx.x; e < 2 * R * R; e += blockDim.x) sPc[(e / (R * R)) * PCS + e % (R * R)] = a.P[a.pc_off + e];
    for (int e = threadIdx.x; e < lsV * R; e += blockDim.x) sPV[e] = a.P[e];
    const int box = blockIdx.y, col0 = blockIdx.x * KC;
    const int kc = min(KC, a.k - col0);
    const int64_t nmid = int64_t(1) << (L - h);
    __syncthreads();
    if (ADJ) {
        for (int id = threadIdx.x; id < P * R * KC; id += blockDim.x) {
            const int col = id / (P * R), rem = id - col * P * R, lp = rem / R, i = rem % R;
            if (col >= kc) continue;
            S[col * P * R + sw(lp, i)] = a.mid[(int64_t(col0 + col) * a.n + int64_t(lp) * nmid + box) * R + i];
        }
        __syncthreads();
        for (int s = h - 1; s >= sV; --s)
            level_op<KC, false, true, true>(S, P, sPc, a.tab.t[s - sV], box, s, L, h, a.sU);
        // V^*: f(xi) = sum_a conj(VP[a][xi]) sum_t PV[q][t] c(a, leaf, t)
        for (int id = threadIdx.x; id < P * KC; id += blockDim.x) {
            const int col = id / P, xl = id - col * P;
            if (col >= kc) continue;
            const int leaf = xl >> sV, qq = xl & (lsV - 1);
            const int64_t xg = int64_t(box) * P + xl;
            const float2* Sc = S + col * P * R;
            const int slotl = rev_bits(leaf, h - sV);
            float2 out = make_float2(0.f, 0.f);
            for (int aa = 0; aa < na; ++aa) {
                float2 c[R];
                load_pair(Sc, aa * nl + slotl, c);
                float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                for (int t = 0; t < R; ++t) {
                    const float pv = sPV[qq * R + t];
                    acc.x = fmaf(pv, c[t].x, acc.x);
                    acc.y = fmaf(pv, c[t].y, acc.y);
                }
                cfmac(out, __ldg(a.VP + int64_t(aa) * a.n + xg), acc);
            }
            a.Y[int64_t(col0 + col) * a.ldy + xg] = out;
        }
    } else {
        // V: c(a, leaf, j) = sum_q PV[q][j] VP[a][xi_q] f(xi_q)
        for (int id = threadIdx.x; id < P * KC; id += blockDim.x) {
            const int col = id / P, lp = id - col * P;
            if (col >= kc) continue;
            const int aa = lp / nl, leaf = lp - aa * nl;
            const int64_t x0 = int64_t(box) * P + int64_t(leaf) * lsV;
            const float2* f = a.X + int64_t(col0 + col) * a.ldx + x0;
            float2 y[R];
#pragma unroll
            for (int jj = 0; jj < R; ++jj) y[jj] = make_float2(0.f, 0.f);
            for (int qq = 0; qq < lsV; ++qq) {
                const float2 m = cmul(__ldg(a.VP + int64_t(aa) * a.n + x0 + qq), f[qq]);
#pragma unroll
                for (int jj = 0; jj < R; ++jj) {
                    const float pv = sPV[qq * R + jj];
                    y[jj].x = fmaf(pv, m.x, y[jj].x);
                    y[jj].y = fmaf(pv, m.y, y[jj].y);
                }
            }
            store_pair(S + col * P * R, aa * nl + rev_bits(leaf, h - sV), y);
        }
        __syncthreads();
        for (int s = sV; s < h; ++s)
            level_op<KC, false, false, false>(S, P, sPc, a.tab.t[s - sV], box, s, L, h, a.sU);
        middle_op<KC, false, false>(S, P, a.M, box, L, h, a.sU);
        for (int id = threadIdx.x; id < P * R * KC; id += blockDim.x) {
            const int col = id / (P * R), rem = id - col * P * R, lp = rem / R, i = rem % R;
            if (col >= kc) continue;
            a.mid[(int64_t(col0 + col) * a.n + int64_t(lp) * nmid + box) * R + i] = S[col * P * R + sw(lp, i)];
        }
    }
}

template <int KC>
size_t half_smem(int P) {
    return size_t(KC) * P * R * sizeof(float2) + (2 * PCS + 8 * R) * sizeof(float);
}

// first/second: the two halves in execution order (adjoint: left then right;
// forward: right then left), each with its own table set.
template <int KC>
fio_status launch_fused_pass(const fio_bf* bf, const HalfArgs& first, const HalfArgs& second, bool adjoint, int kcols,
                             cudaStream_t st) {
    const int Pl = 1 << (bf->L - bf->h), Pr = 1 << bf->h;
    const int nchunk = (kcols + KC - 1) / KC;
    // column chunks of one box are consecutive in launch order: they run together and share the
    // box's factor tables through L2
    dim3 gl(nchunk, 1 << bf->h), gr(nchunk, 1 << (bf->L - bf->h));
    const size_t shl = half_smem<KC>(Pl), shr = half_smem<KC>(Pr);
    static PerDeviceOnce attrs;
    FIO_CUDA(attrs.run([] {
        const int mx = 110 * 1024;
        cudaError_t e = cudaFuncSetAttribute(k_bf_left<KC, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_bf_left<KC, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_bf_right<KC, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_bf_right<KC, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        return e;
    }));
    if (adjoint) {
        FIO_LAUNCH("k_bf_left_adj", st, k_bf_left<KC, true><<<gl, 256, shl, st>>>(first));
        FIO_LAUNCH("k_bf_right_adj", st, k_bf_right<KC, true><<<gr, 256, shr, st>>>(second));
    } else {
        FIO_LAUNCH("k_bf_right_fwd", st, k_bf_right<KC, false><<<gr, 256, shr, st>>>(first));
        FIO_LAUNCH("k_bf_left_fwd", st, k_bf_left<KC, false><<<gl, 256, shl, st>>>(second));
    }
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}


// ===================================================================== v3
// Same halves with 512 threads per CTA and the factor tables staged through
// shared memory: each transfer level's phase slice (P/2 quads x 4 rows of 16
// complex) and the middle-level blocks M (P/8 pairs per chunk) are copied with
// cp.async into one of two buffers while the previous item is computed.  Phase
// rows are stored by physical quad (row = qi*4 + o*2 + e, o the lane-varying
// output half, e the summed input half) with 16-byte chunk m at m ^ ((row>>1)&7),
// so the 8 lanes of a quarter warp (4 quads x 2 o) hit distinct banks.
// Used where P <= 256 (then KC * P = 512: one quad task per thread and level).
namespace v3 {

constexpr int NT = 512;

__device__ __forceinline__ void cp16(void* sdst, const void* gsrc) {
    const unsigned d = unsigned(__cvta_generic_to_shared(sdst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

struct Geo {
    int L, h, sU, sV, n, P, lgP, KC;   // KC * P = NT
};

// Position in the staged buffer of 16-byte chunk e of a box's phase slice of level s: rows by
// physical quad (row = qi*4 + o*2 + e, o the lane-varying output half, e the summed input half),
// chunk m of a row at m ^ ((row >> 1) & 7).
template <bool LEFT, bool ADJ>
__device__ __forceinline__ int stage_pos(int e, int s, const Geo& g) {
    const int W = LEFT ? g.L - s : g.h - s;
    const int j = LEFT ? g.sU - s : g.h - s;
    const int half = 1 << (W - 1);
    const int m = e & 7, row = e >> 3;
    const int ql = row >> 2, c = (row >> 1) & 1, be = row & 1;
    const int a = ql >> (W - 1), lo = ql & (half - 1);
    int rr;
    if (LEFT) {
        const int wj = W - j;
        rr = (rev_bits(lo & ((1 << (j - 1)) - 1), j - 1) << wj) | (lo >> (j - 1));
    } else {
        rr = rev_bits(lo, W - 1);
    }
    const int qi = (a << (W - 1)) | rr;
    const int o = ADJ ? be : c, ee = ADJ ? c : be;
    const int drow = qi * 4 + o * 2 + ee;
    return drow * 8 + (m ^ ((drow >> 1) & 7));
}

// The staged layout of every box of one level, in global memory (one CTA per box): the
// tensor-core passes then stage a level with one TMA bulk copy.
template <bool LEFT, bool ADJ>
__global__ void k_prestage(float4* __restrict__ dst, const float2* __restrict__ T, Geo g, int s) {
    const int box = blockIdx.x;
    const int64_t q0 = LEFT ? (int64_t(box) << (g.L - g.h - 1)) : (int64_t(box) << (g.h - 1));
    const float4* src = reinterpret_cast<const float4*>(T + q0 * 4 * R);
    float4* d = dst + int64_t(box) * g.P * 16;
    const int nch = (g.P / 2) * 4 * 8;
    for (int e = threadIdx.x; e < nch; e += blockDim.x) d[stage_pos<LEFT, ADJ>(e, s, g)] = src[e];
}

// Stage the phase slice of level s (contiguous in global memory) into `buf`.
template <bool LEFT, bool ADJ>
__device__ void stage_level(float4* buf, const float2* __restrict__ T, int box, int s, const Geo& g) {
    const int64_t q0 = LEFT ? (int64_t(box) << (g.L - g.h - 1)) : (int64_t(box) << (g.h - 1));
    const float4* src = reinterpret_cast<const float4*>(T + q0 * 4 * R);
    const int W = LEFT ? g.L - s : g.h - s;
    const int j = LEFT ? g.sU - s : g.h - s;
    const int half = 1 << (W - 1);
    const int nch = (g.P / 2) * 4 * 8;
    for (int e = threadIdx.x; e < nch; e += NT) {
        const int m = e & 7, row = e >> 3;
        const int ql = row >> 2, c = (row >> 1) & 1, be = row & 1;
        const int a = ql >> (W - 1), lo = ql & (half - 1);
        int rr;
        if (LEFT) {
            const int wj = W - j;
            rr = (rev_bits(lo & ((1 << (j - 1)) - 1), j - 1) << wj) | (lo >> (j - 1));
        } else {
            rr = rev_bits(lo, W - 1);
        }
        const int qi = (a << (W - 1)) | rr;
        const int o = ADJ ? be : c, ee = ADJ ? c : be;
        const int drow = qi * 4 + o * 2 + ee;
        cp16(buf + drow * 8 + (m ^ ((drow >> 1) & 7)), src + e);
    }
}

// Stage chunk `ck` of the middle-level blocks: P/8 pairs, 256 complex each.
// LEFT (adjoint M^*, lanes read columns): natural layout; RIGHT (forward M,
// lanes read rows): chunk m of row (pair, i) at m ^ (i & 7).
template <bool LEFT>
__device__ void stage_m(float4* buf, const float2* __restrict__ M, int box, int ck, const Geo& g) {
    const int CH = g.P / 8;
    const int nch = CH * R * 8;
    for (int e = threadIdx.x; e < nch; e += NT) {
        const int m = e & 7, i = (e >> 3) & (R - 1), pl = e >> 7;
        const int lp = ck * CH + pl;
        const int64_t pg = LEFT ? int64_t(box) * g.P + lp : int64_t(lp) * (int64_t(1) << (g.L - g.h)) + box;
        const float4* src = reinterpret_cast<const float4*>(M + pg * R * R) + i * 8 + m;
        const int pos = LEFT ? m : (m ^ (i & 7));
        cp16(buf + (pl * R + i) * 8 + pos, src);
    }
}

// The forward middle-factor chunks of every right-half box in their staged layout (box-major,
// 8 chunks of P/8 pairs each), for one TMA bulk copy per chunk.
__global__ void k_prestage_m(float4* __restrict__ dst, const float2* __restrict__ M, Geo g) {
    const int box = blockIdx.x, ck = blockIdx.y;
    const int CH = g.P / 8, nch = CH * R * 8;
    float4* d = dst + (int64_t(box) * 8 + ck) * nch;
    for (int e = threadIdx.x; e < nch; e += blockDim.x) {
        const int m = e & 7, i = (e >> 3) & (R - 1), pl = e >> 7;
        const int64_t pg = int64_t(ck * CH + pl) * (int64_t(1) << (g.L - g.h)) + box;
        d[(pl * R + i) * 8 + (m ^ (i & 7))] = reinterpret_cast<const float4*>(M + pg * R * R)[i * 8 + m];
    }
}

template <bool LEFT, bool MS, bool ADJ>
__device__ void level3(float2* S, const float* sPc, const float4* ph, int s, const Geo& g) {
    const int P = g.P;
    const int W = LEFT ? g.L - s : g.h - s;
    const int half = 1 << (W - 1);
    const int id = threadIdx.x;   // KC * P == NT: one quad half per thread
    const int col = id >> g.lgP, rem = id & (P - 1), qi = rem >> 1, o = rem & 1;
    const int base = ((qi >> (W - 1)) << W) | (qi & (half - 1));
    float2* Sc = S + col * P * R;
    float2 x0[R], x1[R];
    load_pair(Sc, base, x0);
    load_pair(Sc, base + half, x1);
    __syncwarp();
    const int sw8 = (qi * 2 + o) & 7;
    const float4* r0 = ph + (qi * 4 + o * 2 + 0) * 8;
    const float4* r1 = ph + (qi * 4 + o * 2 + 1) * 8;
    float2 y[R];
    if (MS) {
        const float* Po = sPc + o * PCS;
#pragma unroll
        for (int m = 0; m < R / 2; ++m) {
            const float4 p0 = r0[m ^ sw8], p1 = r1[m ^ sw8];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int i = 2 * m + u;
                float2 h0 = make_float2(0.f, 0.f), h1 = make_float2(0.f, 0.f);
#pragma unroll
                for (int t4 = 0; t4 < R / 4; ++t4) {
                    const float4 pv = *reinterpret_cast<const float4*>(Po + i * R + 4 * t4);
                    const float pp[4] = {pv.x, pv.y, pv.z, pv.w};
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const int t = 4 * t4 + v;
                        h0.x = fmaf(pp[v], x0[t].x, h0.x);
                        h0.y = fmaf(pp[v], x0[t].y, h0.y);
                        h1.x = fmaf(pp[v], x1[t].x, h1.x);
                        h1.y = fmaf(pp[v], x1[t].y, h1.y);
                    }
                }
                const float2 f0 = u ? make_float2(p0.z, p0.w) : make_float2(p0.x, p0.y);
                const float2 f1 = u ? make_float2(p1.z, p1.w) : make_float2(p1.x, p1.y);
                float2 acc = make_float2(0.f, 0.f);
                if (!ADJ) {
                    cfma(acc, f0, h0);
                    cfma(acc, f1, h1);
                } else {
                    cfmac(acc, f0, h0);
                    cfmac(acc, f1, h1);
                }
                y[i] = acc;
            }
        }
    } else {
#pragma unroll
        for (int jj = 0; jj < R; ++jj) y[jj] = make_float2(0.f, 0.f);
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const float4* re = e ? r1 : r0;
            const float* Pe = sPc + e * PCS;
#pragma unroll
            for (int m = 0; m < R / 2; ++m) {
                const float4 pq = re[m ^ sw8];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int t = 2 * m + u;
                    const float2 f = u ? make_float2(pq.z, pq.w) : make_float2(pq.x, pq.y);
                    const float2 xv = e ? x1[t] : x0[t];
                    const float2 gg = ADJ ? cmulc(f, xv) : cmul(f, xv);
#pragma unroll
                    for (int j4 = 0; j4 < R / 4; ++j4) {
                        const float4 pv = *reinterpret_cast<const float4*>(Pe + t * R + 4 * j4);
                        y[4 * j4 + 0].x = fmaf(pv.x, gg.x, y[4 * j4 + 0].x);
                        y[4 * j4 + 0].y = fmaf(pv.x, gg.y, y[4 * j4 + 0].y);
                        y[4 * j4 + 1].x = fmaf(pv.y, gg.x, y[4 * j4 + 1].x);
                        y[4 * j4 + 1].y = fmaf(pv.y, gg.y, y[4 * j4 + 1].y);
                        y[4 * j4 + 2].x = fmaf(pv.z, gg.x, y[4 * j4 + 2].x);
                        y[4 * j4 + 2].y = fmaf(pv.z, gg.y, y[4 * j4 + 2].y);
                        y[4 * j4 + 3].x = fmaf(pv.w, gg.x, y[4 * j4 + 3].x);
                        y[4 * j4 + 3].y = fmaf(pv.w, gg.y, y[4 * j4 + 3].y);
                    }
                }
            }
        }
    }
    store_pair(Sc, o ? base + half : base, y);
}

// ---------------------------------------------------------------- tensor cores
// Transfer level on the 5th-generation tensor cores (tcgen05).  The real
// Lagrange products of a level are GEMMs with one matrix shared by every quad
// of the CTA; one GEMM row per thread (task (column, quad, o)), 4 tiles of
// M = 128 rows per CTA:
//   SM: A row = [g_0 | g_1],  g_e[t] = Phi(o,e,t) x_e[t]  (K = 2 e x 16 t x re/im = 64)
//       B[(j, re/im)][(e, t, re/im)] = Pc[e][t][j]       ->  D row = y_o (N = 32)
//   MS: A row = [J_o x_0 | J_o x_1] (J_o reverses t when o = 0), two products
//       with B[(i, re/im)][(t, re/im)] = Pc[1][i][t]  ->  D_e row = J_o P_o x_e
//       (N = 32 each), since P_0 = J P_1 J (Chebyshev nodes are symmetric);
//       the epilogue reverses back and forms y_o = sum_e Phi(o,e,i) D_e.
// Real and imaginary parts ride as separate K / N indices (B is zero between
// them).  FP32 accuracy comes from a three-term split v = hi + lo of both
// operands, D = A_hi B_hi + A_hi B_lo + A_lo B_hi with FP32 accumulation in
// TMEM: FP16 parts (11 + 11 bits) with every row scaled by a power of two that
// puts its largest entry in [2^14, 2^15) (exact; undone in the epilogue), or
// BF16 parts (8 + 8 bits, no scaling) for the split-precision setting.
// A rows are written to TMEM with tcgen05.st, B sits in shared memory, and one
// thread issues the MMAs and commits them to an mbarrier.
// TMEM columns of tile t: A_hi [128t, +32), A_lo [128t + 32, +32), D [128t + 64, +64).
constexpr int kSimt = 0, kTcF16 = 1, kTcBF16 = 2;
constexpr int kTmemCols = 512;
constexpr uint32_t kBBytesSM = 32 * 64 * 2, kBBytesMS = 32 * 32 * 2;   // one of hi / lo

struct Tc {
    uint32_t tmem;     // TMEM base address
    uint64_t* mbar;    // MMA completion: one barrier per thread group (or one for the CTA)
    int* fail;         // shared flag: a bounded wait ran out
    uint32_t phase;    // parity of the next completion of this thread's MMA barrier
    uint32_t bsm;      // shared address of B_hi; B_lo follows at + bbytes
    uint32_t bbytes;
    bool grp;          // two independent thread groups (one per half of the columns)
};

// The CTA's threads split into two groups of NT / 2 that own disjoint columns (KC >= 2):
// each group synchronizes on its own named barrier and issues its own MMAs.
__device__ __forceinline__ int tgroup() { return threadIdx.x >> 8; }
__device__ __forceinline__ void group_sync() {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + tgroup()), "r"(NT / 2) : "memory");
}

using tc::Half16;
using tc::row_scale;
using tc::split_pair;

// Build B_hi / B_lo of the level form in shared memory (canonical K-major layout,
// LBO = 128 B between core matrices along K, SBO = K / 8 * 128 B between 8-row groups).
template <bool MS, bool BF> __device__ void build_b(unsigned char* bs, const float* sPc) {
    using H = Half16<BF>;
    constexpr int K = MS ? 32 : 64, N = 32;
    uint16_t* hi = reinterpret_cast<uint16_t*>(bs);
    uint16_t* lo = reinterpret_cast<uint16_t*>(bs + N * K * 2);
    for (int e = threadIdx.x; e < N * K; e += blockDim.x) {
        const int n = e / K, k = e % K;
        const int jn = n >> 1, pn = n & 1;
        float v = 0.f;
        if (MS) {   // k = (t, re/im)
            const int t = k >> 1, pk = k & 1;
            if (pk == pn) v = sPc[PCS + jn * R + t];
        } else {    // k = (e, t, re/im)
            const int ee = k >> 5, t = (k >> 1) & (R - 1), pk = k & 1;
            if (pk == pn) v = sPc[ee * PCS + t * R + jn];
        }
        const uint16_t h = H::one(v);
        const uint16_t l = H::one(v - H::back(h));
        const int off = (n >> 3) * (K / 8) * 64 + (k >> 3) * 64 + (n & 7) * 8 + (k & 7);   // in 16-bit elements
        hi[off] = h;
        lo[off] = l;
    }
}

__device__ int g_tc_wait_timeout = 0;

// B operands of the tensor-core levels: the first 128-byte boundary after `after`.
__device__ __forceinline__ unsigned char* tc_bsm(const float* after) {
    const uintptr_t p = reinterpret_cast<uintptr_t>(after);
    return reinterpret_cast<unsigned char*>((p + 127) & ~uintptr_t(127));
}

template <bool LEFT, bool MS, bool ADJ, bool BF>
__device__ void level3_tc(float2* S, const float4* ph, int s, const Geo& g, Tc& tc) {
    const int P = g.P;
    const int W = LEFT ? g.L - s : g.h - s;
    const int half = 1 << (W - 1);
    const int id = threadIdx.x;   // KC * P == NT: one GEMM row per thread
    const int col = id >> g.lgP, rem = id & (P - 1), qi = rem >> 1, o = rem & 1;
    const int base = ((qi >> (W - 1)) << W) | (qi & (half - 1));
    float2* Sc = S + col * P * R;
    const int sw8 = (qi * 2 + o) & 7;
    const float4* r0 = ph + (qi * 4 + o * 2 + 0) * 8;   // Phi(o, e = 0, .)
    const float4* r1 = ph + (qi * 4 + o * 2 + 1) * 8;   // Phi(o, e = 1, .)
    const uint32_t tcol = tc.tmem + (uint32_t(id & 0x60) << 16) + uint32_t(id >> 7) * 128;
    float sc = 1.f, isc = 1.f;
    {
        float2 x0[R], x1[R];
        load_pair(Sc, base, x0);
        load_pair(Sc, base + half, x1);
        if (!BF) {   // |Phi| = 1: |Re g|, |Im g| <= |Re x| + |Im x|
            float mx = 0.f;
#pragma unroll
            for (int t = 0; t < R; ++t) {
                mx = fmaxf(mx, fabsf(x0[t].x) + fabsf(x0[t].y));
                mx = fmaxf(mx, fabsf(x1[t].x) + fabsf(x1[t].y));
            }
            row_scale(mx, sc, isc);
        }
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            uint32_t hi[R], lo[R];
#pragma unroll
            for (int m = 0; m < R / 2; ++m) {
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int t = 2 * m + u;
                    float2 v;
                    if (MS) {
                        const float2 a0 = e ? x1[t] : x0[t], a1 = e ? x1[R - 1 - t] : x0[R - 1 - t];
                        v = o ? a0 : a1;
                    } else {
                        const float4 pq = (e ? r1 : r0)[m ^ sw8];
                        const float2 f = u ? make_float2(pq.z, pq.w) : make_float2(pq.x, pq.y);
                        const float2 xv = e ? x1[t] : x0[t];
                        v = ADJ ? cmulc(f, xv) : cmul(f, xv);
                    }
                    split_pair<BF>(v.x * sc, v.y * sc, hi[t], lo[t]);
                }
            }
            tc::tmem_st16(tcol + 16 * e, hi);
            tc::tmem_st16(tcol + 32 + 16 * e, lo);
        }
        tc::tmem_wait_st();
    }
    tc::fence_before();
    if (tc.grp) group_sync();
    else __syncthreads();
    const int issuer = tc.grp ? tgroup() * (NT / 2) : 0;
    if (id == issuer && !*tc.fail) {
        tc::fence_after();
        const uint32_t idesc = tc::idesc_f16(BF, 128, 32);
        constexpr uint32_t sbo = MS ? 512 : 1024;
        const int t_lo = tc.grp ? 2 * tgroup() : 0, t_hi = tc.grp ? t_lo + 2 : 4;
#pragma unroll 1
        for (int t4 = t_lo; t4 < t_hi; ++t4) {
            const uint32_t A = tc.tmem + 128 * t4, D = A + 64;
            if (MS) {
#pragma unroll
                for (int e = 0; e < 2; ++e)
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks) {
                        const uint64_t bh = tc::smem_desc(tc.bsm + 256 * ks, 128, sbo);
                        const uint64_t bl = tc::smem_desc(tc.bsm + tc.bbytes + 256 * ks, 128, sbo);
                        const uint32_t ah = A + 16 * e + 8 * ks, al = ah + 32;
                        tc::mma_f16_ts(D + 32 * e, ah, bh, idesc, ks);
                        tc::mma_f16_ts(D + 32 * e, ah, bl, idesc, 1);
                        tc::mma_f16_ts(D + 32 * e, al, bh, idesc, 1);
                    }
            } else {
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                    const uint64_t bh = tc::smem_desc(tc.bsm + 256 * ks, 128, sbo);
                    const uint64_t bl = tc::smem_desc(tc.bsm + tc.bbytes + 256 * ks, 128, sbo);
                    const uint32_t ah = A + 8 * ks, al = ah + 32;
                    tc::mma_f16_ts(D, ah, bh, idesc, ks);
                    tc::mma_f16_ts(D, ah, bl, idesc, 1);
                    tc::mma_f16_ts(D, al, bh, idesc, 1);
                }
            }
        }
        tc::mma_commit(tc.mbar);
    }
    if (!*tc.fail && !tc::mbar_wait(tc.mbar, tc.phase)) {
        *tc.fail = 1;
        atomicExch(&g_tc_wait_timeout, 1);
    }
    tc.phase ^= 1u;
    tc::fence_after();
    float2 y[R];
    if (MS) {
#pragma unroll
        for (int i = 0; i < R; ++i) y[i] = make_float2(0.f, 0.f);
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            // D_e columns (2 i' + re/im): i' < 8 in d0, i' >= 8 in d1;  h[o][e][i] = D_e[o ? i : R - 1 - i]
            uint32_t d0[16], d1[16];
            tc::tmem_ld16(tcol + 64 + 32 * e, d0);
            tc::tmem_ld16(tcol + 80 + 32 * e, d1);
            tc::tmem_wait_ld();
            const float4* re = e ? r1 : r0;
#pragma unroll
            for (int m = 0; m < R / 2; ++m) {
                const float4 pq = re[m ^ sw8];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int i = 2 * m + u, ii = R - 1 - i;
                    const float2 hf = i < 8 ? make_float2(__uint_as_float(d0[2 * i]), __uint_as_float(d0[2 * i + 1]))
                                            : make_float2(__uint_as_float(d1[2 * i - 16]), __uint_as_float(d1[2 * i - 15]));
                    const float2 hr = ii < 8 ? make_float2(__uint_as_float(d0[2 * ii]), __uint_as_float(d0[2 * ii + 1]))
                                             : make_float2(__uint_as_float(d1[2 * ii - 16]), __uint_as_float(d1[2 * ii - 15]));
                    const float2 h = cscale(o ? hf : hr, isc);
                    const float2 f = u ? make_float2(pq.z, pq.w) : make_float2(pq.x, pq.y);
                    if (!ADJ) cfma(y[i], f, h);
                    else cfmac(y[i], f, h);
                }
            }
        }
    } else {
        uint32_t d0[16], d1[16];
        tc::tmem_ld16(tcol + 64, d0);
        tc::tmem_ld16(tcol + 80, d1);
        tc::tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < R / 2; ++j) {
            y[j] = make_float2(__uint_as_float(d0[2 * j]) * isc, __uint_as_float(d0[2 * j + 1]) * isc);
            y[j + R / 2] = make_float2(__uint_as_float(d1[2 * j]) * isc, __uint_as_float(d1[2 * j + 1]) * isc);
        }
    }
    store_pair(Sc, o ? base + half : base, y);
    tc::fence_before();
}

// CTA set-up of the tensor-core levels: TMEM (warp 0), mbarriers, B operands.
// s_mbar: [0, 1] MMA completion of group 0 / 1 (or [0] for the CTA), [2, 3] staging buffers
// full, [4, 5] staging buffers consumed by both groups (grouped pipeline only).
template <bool MS, bool BF>
__device__ void tc_setup(Tc& tc, unsigned char* bsmem, const float* sPc, uint32_t* s_tmem, uint64_t* s_mbar, int* s_fail,
                         bool grp) {
    if (threadIdx.x < 32) tc::tmem_alloc(s_tmem, kTmemCols);
    if (threadIdx.x == 0) {
        tc::mbar_init(s_mbar + 0, 1);
        tc::mbar_init(s_mbar + 1, 1);
        tc::mbar_init(s_mbar + 2, NT);
        tc::mbar_init(s_mbar + 3, NT);
        tc::mbar_init(s_mbar + 4, 2);
        tc::mbar_init(s_mbar + 5, 2);
        *s_fail = 0;
    }
    build_b<MS, BF>(bsmem, sPc);
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    tc.tmem = *s_tmem;
    tc.grp = grp;
    tc.mbar = s_mbar + (grp ? tgroup() : 0);
    tc.fail = s_fail;
    tc.phase = 0;
    tc.bsm = tc::smem_addr(bsmem);
    tc.bbytes = MS ? kBBytesMS : kBBytesSM;
}
__device__ __forceinline__ void tc_teardown(const Tc& tc) {
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (threadIdx.x < 32) tc::tmem_free(tc.tmem, kTmemCols);
}

// One chunk of M (forward, RIGHT) or M^* (adjoint, LEFT), in place: task =
// (pair of the chunk, column, output index), 16 lanes per (pair, column).
template <bool LEFT>
__device__ void mchunk3(float2* S, const float4* mb, int ck, const Geo& g) {
    // 8 lanes per (pair, column), two outputs per lane: a quarter warp covers one
    // pair, so its 16-byte M loads are consecutive and its state loads broadcast.
    const int P = g.P, CH = P / 8;
    const int nB = g.sU - g.h, lo = g.L - g.sU;
    const int ntask = CH * g.KC * (R / 2);
    for (int b0 = 0; b0 < ntask; b0 += NT) {
        const int id = b0 + threadIdx.x;
        const bool act = id < ntask;
        const int jq = id & 7, rest = id >> 3;
        const int pl = rest % CH, col = rest / CH;
        const int lp = ck * CH + pl;
        const int slot = LEFT ? ((rev_bits(lp & ((1 << nB) - 1), nB) << lo) | (lp >> nB)) : lp;
        float2* Sc = S + col * P * R;
        float2 x[R];
        if (act) load_pair(Sc, slot, x);
        __syncwarp();
        if (act) {
            float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
            if (LEFT) {   // y_j = sum_i conj(M[i][j]) x_i, natural layout; j = 2 jq, 2 jq + 1
                const float4* mp = mb + pl * R * 8 + jq;
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    const float4 v = mp[i * 8];
                    cfmac(a0, make_float2(v.x, v.y), x[i]);
                    cfmac(a1, make_float2(v.z, v.w), x[i]);
                }
            } else {      // y_i = sum_j M[i][j] x_j, row i swizzled by (i & 7); i = 2 jq, 2 jq + 1
                const float4* r0 = mb + (pl * R + 2 * jq) * 8;
                const float4* r1 = r0 + 8;
                const int s0 = (2 * jq) & 7, s1 = (2 * jq + 1) & 7;
#pragma unroll
                for (int m = 0; m < R / 2; ++m) {
                    const float4 v0 = r0[m ^ s0], v1 = r1[m ^ s1];
                    cfma(a0, make_float2(v0.x, v0.y), x[2 * m]);
                    cfma(a0, make_float2(v0.z, v0.w), x[2 * m + 1]);
                    cfma(a1, make_float2(v1.x, v1.y), x[2 * m]);
                    cfma(a1, make_float2(v1.z, v1.w), x[2 * m + 1]);
                }
            }
            Sc[sw(slot, 2 * jq)] = a0;
            Sc[sw(slot, 2 * jq + 1)] = a1;
        }
    }
}

// Shared-memory layout of one CTA: state (64 KiB), one or two table buffers
// of P * 256 B (two when P <= 256: the next item is staged while the current
// one is computed), the Lagrange matrices.
__device__ __forceinline__ int nbuf3(int P) { return P <= 256 ? 2 : 1; }

// Runs the staged item sequence: items [0, nlev) are transfer levels, the
// rest middle-level chunks; `stage(it, buf)` issues the copies of item it,
// `compute(it, buf)` consumes them.
template <class StageF, class ComputeF>
__device__ void pipeline3(int nitem, int P, float4* buf0, float4* buf1, StageF stage, ComputeF compute) {
    if (nitem == 0) return;
    if (nbuf3(P) == 2) {
        for (int it = 0; it < nitem; ++it) {
            float4* cur = (it & 1) ? buf1 : buf0;
            if (it + 1 < nitem) {
                stage(it + 1, (it & 1) ? buf0 : buf1);
                cp_commit();
                cp_wait1();
            } else {
                cp_wait0();
            }
            __syncthreads();
            compute(it, cur);
            __syncthreads();
        }
    } else {
        for (int it = 0; it < nitem; ++it) {
            if (it > 0) {
                stage(it, buf0);
                cp_commit();
            }
            cp_wait0();
            __syncthreads();
            compute(it, buf0);
            __syncthreads();
        }
    }
}

// The staged item sequence with two independent thread groups (tensor-core levels, KC >= 2, two
// table buffers).  Every thread stages its share of each item with cp.async and arrives on the
// buffer's `full` barrier once its copies complete; a group waits there, computes the item with
// its own barriers, and one thread per group arrives on the buffer's `empty` barrier; the next
// item for that buffer is staged only after both groups consumed it.  The groups drift apart by
// up to one item, so one group's MMA waits overlap the other group's CUDA-core work.
__device__ __forceinline__ void cp_arrive(uint64_t* m) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(tc::smem_addr(m)) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* m) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_addr(m)) : "memory");
}
__device__ __forceinline__ void bounded_wait(uint64_t* m, uint32_t parity, int* fail) {
    if (!*fail && !tc::mbar_wait(m, parity)) {
        *fail = 1;
        atomicExch(&g_tc_wait_timeout, 1);
    }
}
// TMA bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) into this CTA's
// shared memory, completing on the mbarrier: thread 0 arms the barrier with the byte count and
// issues the copy, every other thread arrives.
__device__ __forceinline__ void bulk_stage(float4* dst, const float4* src, uint32_t bytes, uint64_t* full) {
    if (threadIdx.x == 0) {
        tc::mbar_expect_tx(full, bytes);
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         tc::smem_addr(dst)),
                     "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(tc::smem_addr(full))
                     : "memory");
    } else {
        mbar_arrive(full);
    }
}

// stage(it, buf, full) issues item it's copies into buf and arrives on `full` (one arrival per
// thread, by cp_arrive after cp.async copies or through bulk_stage).
template <class StageF, class ComputeF>
__device__ void pipeline_grp(int nitem, float4* buf0, float4* buf1, StageF stage, ComputeF compute, uint64_t* bars,
                             int* fail) {
    uint64_t* full = bars + 2;
    uint64_t* empty = bars + 4;
    if (nitem == 0) return;
    stage(0, buf0, &full[0]);
    for (int it = 0; it < nitem; ++it) {
        const int b = it & 1;
        if (it + 1 < nitem) {
            const int b1 = (it + 1) & 1, use1 = (it + 1) >> 1;
            if (use1 >= 1) bounded_wait(&empty[b1], uint32_t(use1 - 1) & 1u, fail);
            stage(it + 1, b1 ? buf1 : buf0, &full[b1]);
        }
        bounded_wait(&full[b], uint32_t(it >> 1) & 1u, fail);
        compute(it, b ? buf1 : buf0);
        group_sync();
        if ((threadIdx.x & (NT / 2 - 1)) == 0) mbar_arrive(&empty[b]);
    }
}

// Middle state between HBM and the shared state, in 16-byte chunks (two coefficients), eight
// chunks per thread in flight: goff(col, lp) is the float2 offset of pair lp's coefficients in
// `mid` (column col of the CTA), slot(lp) its physical slot.
template <bool IN, class GOff, class Slot>
__device__ __forceinline__ void mid_copy(float2* S, float2* mid, int P, int KC, int kc, GOff goff, Slot slot) {
    constexpr int kBatch = 8;
    const int per_col = P * (R / 2), nch = per_col * KC;
    for (int base = threadIdx.x; base < nch; base += NT * kBatch) {
        float4 v[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int id = base + u * NT, col = id / per_col, rem = id - col * per_col, lp = rem >> 3, i2 = rem & 7;
            if (id < nch && col < kc) {
                const int p = slot(lp);
                if (IN) v[u] = reinterpret_cast<const float4*>(mid + goff(col, lp))[i2];
                else v[u] = reinterpret_cast<const float4*>(S + col * P * R + p * R)[i2 ^ (p & 7)];
            }
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int id = base + u * NT, col = id / per_col, rem = id - col * per_col, lp = rem >> 3, i2 = rem & 7;
            if (id < nch && col < kc) {
                const int p = slot(lp);
                if (IN) reinterpret_cast<float4*>(S + col * P * R + p * R)[i2 ^ (p & 7)] = v[u];
                else reinterpret_cast<float4*>(mid + goff(col, lp))[i2] = v[u];
            }
        }
    }
}

template <bool ADJ, int MODE>
__device__ void left3_body(const HalfArgs& a, int box, int col0) {
    extern __shared__ float4 smem4[];
    Geo g;
    g.L = a.L; g.h = a.h; g.sU = a.sU; g.sV = a.sV; g.n = a.n;
    g.lgP = a.L - a.h; g.P = 1 << g.lgP; g.KC = NT >> g.lgP;
    const int P = g.P, KC = g.KC;
    float2* S = reinterpret_cast<float2*>(smem4);
    float4* buf0 = smem4 + NT * R / 2;
    float4* buf1 = buf0 + P * 16;
    float* sPc = reinterpret_cast<float*>(buf0 + nbuf3(P) * P * 16);
    float* sPU = sPc + 2 * PCS;
    unsigned char* bsm = tc_bsm(sPU + kLeafMax * RS);
    const int lsU = 1 << (g.L - g.sU), nbU = lsU;
    const int kc = min(KC, a.k - col0);
    const int nlev = g.sU - g.h;
    const int nitem = nlev + (ADJ ? 8 : 0);
    constexpr bool TC = MODE != kSimt;
    __shared__ uint32_t s_tmem;
    __shared__ uint64_t s_mbar[6];
    __shared__ int s_fail;
    Tc tc;
    const bool grp = TC && nlev > 0 && KC >= 2 && nbuf3(P) == 2;
    auto stage = [&](int it, float4* b) {
        if (it < nlev) {
            const int s = ADJ ? g.sU - 1 - it : g.h + it;
            stage_level<true, ADJ>(b, a.tab.t[s - g.h], box, s, g);
        } else {
            stage_m<true>(b, a.M, box, it - nlev, g);
        }
    };
    // grouped pipeline: pre-staged level slices and the contiguous M^* chunks by TMA bulk copies
    auto stage_grp = [&](int it, float4* b, uint64_t* full) {
        if (it < nlev) {
            const int s = ADJ ? g.sU - 1 - it : g.h + it;
            if (a.tabs.t[s - g.h]) {
                bulk_stage(b, reinterpret_cast<const float4*>(a.tabs.t[s - g.h]) + int64_t(box) * P * 16,
                           uint32_t(P) * 256, full);
                return;
            }
            stage_level<true, ADJ>(b, a.tab.t[s - g.h], box, s, g);
        } else {
            const int CH = P / 8;
            bulk_stage(b, reinterpret_cast<const float4*>(a.M + (int64_t(box) * P + (it - nlev) * CH) * R * R),
                       uint32_t(CH) * R * R * 8, full);
            return;
        }
        cp_arrive(full);
    };
    auto compute = [&](int it, const float4* cur) {
        if (it < nlev) {
            const int s = ADJ ? g.sU - 1 - it : g.h + it;
            if (TC) {   // adjoint B^* levels scale then mix, forward B levels mix then scale
                if (ADJ) level3_tc<true, false, true, MODE == kTcBF16>(S, cur, s, g, tc);
                else level3_tc<true, true, false, MODE == kTcBF16>(S, cur, s, g, tc);
            } else {
                if (ADJ) level3<true, false, true>(S, sPc, cur, s, g);
                else level3<true, true, false>(S, sPc, cur, s, g);
            }
        } else {
            mchunk3<true>(S, cur, it - nlev, g);
        }
    };
    if (nitem > 0 && !grp) {
        stage(0, buf0);
        cp_commit();
    }
    for (int e = threadIdx.x; e < 2 * R * R; e += NT) sPc[(e / (R * R)) * PCS + e % (R * R)] = a.P[a.pc_off + e];
    for (int e = threadIdx.x; e < lsU * R; e += NT) sPU[(e / R) * RS + e % R] = a.P[a.pu_off + e];
    __syncthreads();
    if (TC && nlev > 0) tc_setup<!ADJ, MODE == kTcBF16>(tc, bsm, sPc, &s_tmem, s_mbar, &s_fail, grp);
    const int nB = nlev, lo = g.L - g.sU;
    if (ADJ) {
        for (int id = threadIdx.x; id < P * KC; id += NT) {   // U^*
            const int col = id >> g.lgP, lp = id & (P - 1);
            if (col >= kc) continue;
            const int leaf = lp / nbU, b = lp - leaf * nbU;
            const int64_t x0 = int64_t(box) * P + int64_t(leaf) * lsU;
            const float2* gv = a.X + int64_t(col0 + col) * a.ldx + x0;
            float2 mm[kLeafMax];   // all global loads of the leaf issued before the products
#pragma unroll
            for (int qq = 0; qq < kLeafMax; ++qq)
                if (qq < lsU) mm[qq] = cmulc(__ldg(a.UP + (x0 + qq) * nbU + b), __ldg(gv + qq));
            float2 y[R];
#pragma unroll
            for (int i = 0; i < R; ++i) y[i] = make_float2(0.f, 0.f);
#pragma unroll
            for (int qq = 0; qq < kLeafMax; ++qq) {
                if (qq >= lsU) break;
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    const float pu = sPU[qq * RS + i];
                    y[i].x = fmaf(pu, mm[qq].x, y[i].x);
                    y[i].y = fmaf(pu, mm[qq].y, y[i].y);
                }
            }
            store_pair(S + col * P * R, lp, y);
        }
    } else {
        mid_copy<true>(S, a.mid, P, KC, kc,   // middle state in
                       [&](int col, int lp) { return (int64_t(col0 + col) * a.n + int64_t(box) * P + lp) * R; },
                       [&](int lp) { return (rev_bits(lp & ((1 << nB) - 1), nB) << lo) | (lp >> nB); });
    }
    if (grp) {
        __syncthreads();
        pipeline_grp(nitem, buf0, buf1, stage_grp, compute, s_mbar, &s_fail);
        __syncthreads();
    } else {
        pipeline3(nitem, P, buf0, buf1, stage, compute);
    }
    if (ADJ) {
        mid_copy<false>(S, a.mid, P, KC, kc,   // middle state out
                        [&](int col, int lp) { return (int64_t(col0 + col) * a.n + int64_t(box) * P + lp) * R; },
                        [&](int lp) { return (rev_bits(lp & ((1 << nB) - 1), nB) << lo) | (lp >> nB); });
    } else {
        for (int id = threadIdx.x; id < P * KC; id += NT) {   // U
            const int col = id >> g.lgP, xl = id & (P - 1);
            if (col >= kc) continue;
            const int leaf = xl / lsU, qq = xl - leaf * lsU;
            const int64_t xg = int64_t(box) * P + xl;
            const float2* Sc = S + col * P * R;
            float2 up[kLeafMax];
#pragma unroll
            for (int b = 0; b < kLeafMax; ++b)
                if (b < nbU) up[b] = __ldg(a.UP + xg * nbU + b);
            float2 out = make_float2(0.f, 0.f);
#pragma unroll
            for (int b = 0; b < kLeafMax; ++b) {
                if (b >= nbU) break;
                float2 d[R];
                load_pair(Sc, leaf * nbU + b, d);
                float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    const float pu = sPU[qq * RS + i];
                    acc.x = fmaf(pu, d[i].x, acc.x);
                    acc.y = fmaf(pu, d[i].y, acc.y);
                }
                cfma(out, up[b], acc);
            }
            a.Y[int64_t(col0 + col) * a.ldy + xg] = out;
        }
    }
    if (TC && nlev > 0) tc_teardown(tc);
}

template <bool ADJ, int MODE>
__device__ void right3_body(const HalfArgs& a, int box, int col0) {
    extern __shared__ float4 smem4[];
    Geo g;
    g.L = a.L; g.h = a.h; g.sU = a.sU; g.sV = a.sV; g.n = a.n;
    g.lgP = a.h; g.P = 1 << g.lgP; g.KC = NT >> g.lgP;
    const int P = g.P, KC = g.KC;
    float2* S = reinterpret_cast<float2*>(smem4);
    float4* buf0 = smem4 + NT * R / 2;
    float4* buf1 = buf0 + P * 16;
    float* sPc = reinterpret_cast<float*>(buf0 + nbuf3(P) * P * 16);
    float* sPV = sPc + 2 * PCS;
    unsigned char* bsm = tc_bsm(sPV + kLeafMax * RS);
    const int lsV = 1 << g.sV, na = 1 << g.sV, nl = 1 << (g.h - g.sV);
    const int kc = min(KC, a.k - col0);
    const int64_t nmid = int64_t(1) << (g.L - g.h);
    const int nlev = g.h - g.sV;
    const int nitem = nlev + (ADJ ? 0 : 8);
    constexpr bool TC = MODE != kSimt;
    __shared__ uint32_t s_tmem;
    __shared__ uint64_t s_mbar[6];
    __shared__ int s_fail;
    Tc tc;
    const bool grp = TC && nlev > 0 && KC >= 2 && nbuf3(P) == 2;
    auto stage = [&](int it, float4* b) {
        if (it < nlev) {
            const int s = ADJ ? g.h - 1 - it : g.sV + it;
            stage_level<false, ADJ>(b, a.tab.t[s - g.sV], box, s, g);
        } else {
            stage_m<false>(b, a.M, box, it - nlev, g);
        }
    };
    // grouped pipeline: pre-staged level slices by TMA bulk copies (the strided M chunks of the
    // forward pass stay on cp.async)
    auto stage_grp = [&](int it, float4* b, uint64_t* full) {
        if (it < nlev) {
            const int s = ADJ ? g.h - 1 - it : g.sV + it;
            if (a.tabs.t[s - g.sV]) {
                bulk_stage(b, reinterpret_cast<const float4*>(a.tabs.t[s - g.sV]) + int64_t(box) * P * 16,
                           uint32_t(P) * 256, full);
                return;
            }
            stage_level<false, ADJ>(b, a.tab.t[s - g.sV], box, s, g);
        } else {
            if (a.Ms) {
                const int nch = (P / 8) * R * 8;
                bulk_stage(b, reinterpret_cast<const float4*>(a.Ms) + (int64_t(box) * 8 + (it - nlev)) * nch,
                           uint32_t(nch) * 16, full);
                return;
            }
            stage_m<false>(b, a.M, box, it - nlev, g);
        }
        cp_arrive(full);
    };
    auto compute = [&](int it, const float4* cur) {
        if (it < nlev) {
            const int s = ADJ ? g.h - 1 - it : g.sV + it;
            if (TC) {   // adjoint C^* levels mix then scale, forward C levels scale then mix
                if (ADJ) level3_tc<false, true, true, MODE == kTcBF16>(S, cur, s, g, tc);
                else level3_tc<false, false, false, MODE == kTcBF16>(S, cur, s, g, tc);
            } else {
                if (ADJ) level3<false, true, true>(S, sPc, cur, s, g);
                else level3<false, false, false>(S, sPc, cur, s, g);
            }
        } else {
            mchunk3<false>(S, cur, it - nlev, g);
        }
    };
    if (nitem > 0 && !grp) {
        stage(0, buf0);
        cp_commit();
    }
    for (int e = threadIdx.x; e < 2 * R * R; e += NT) sPc[(e / (R * R)) * PCS + e % (R * R)] = a.P[a.pc_off + e];
    for (int e = threadIdx.x; e < lsV * R; e += NT) sPV[(e / R) * RS + e % R] = a.P[e];
    __syncthreads();
    if (TC && nlev > 0) tc_setup<ADJ, MODE == kTcBF16>(tc, bsm, sPc, &s_tmem, s_mbar, &s_fail, grp);
    if (ADJ) {
        mid_copy<true>(S, a.mid, P, KC, kc,   // middle state in
                       [&](int col, int lp) { return (int64_t(col0 + col) * a.n + int64_t(lp) * nmid + box) * R; },
                       [](int lp) { return lp; });
    } else {
        for (int id = threadIdx.x; id < P * KC; id += NT) {   // V
            const int col = id >> g.lgP, lp = id & (P - 1);
            if (col >= kc) continue;
            const int aa = lp / nl, leaf = lp - aa * nl;
            const int64_t x0 = int64_t(box) * P + int64_t(leaf) * lsV;
            const float2* f = a.X + int64_t(col0 + col) * a.ldx + x0;
            float2 mm[kLeafMax];
#pragma unroll
            for (int qq = 0; qq < kLeafMax; ++qq)
                if (qq < lsV) mm[qq] = cmul(__ldg(a.VP + int64_t(aa) * a.n + x0 + qq), __ldg(f + qq));
            float2 y[R];
#pragma unroll
            for (int jj = 0; jj < R; ++jj) y[jj] = make_float2(0.f, 0.f);
#pragma unroll
            for (int qq = 0; qq < kLeafMax; ++qq) {
                if (qq >= lsV) break;
#pragma unroll
                for (int jj = 0; jj < R; ++jj) {
                    const float pv = sPV[qq * RS + jj];
                    y[jj].x = fmaf(pv, mm[qq].x, y[jj].x);
                    y[jj].y = fmaf(pv, mm[qq].y, y[jj].y);
                }
            }
            store_pair(S + col * P * R, aa * nl + rev_bits(leaf, g.h - g.sV), y);
        }
    }
    if (grp) {
        __syncthreads();
        pipeline_grp(nitem, buf0, buf1, stage_grp, compute, s_mbar, &s_fail);
        __syncthreads();
    } else {
        pipeline3(nitem, P, buf0, buf1, stage, compute);
    }
    if (ADJ) {
        for (int id = threadIdx.x; id < P * KC; id += NT) {   // V^*
            const int col = id >> g.lgP, xl = id & (P - 1);
            if (col >= kc) continue;
            const int leaf = xl >> g.sV, qq = xl & (lsV - 1);
            const int64_t xg = int64_t(box) * P + xl;
            const float2* Sc = S + col * P * R;
            const int slotl = rev_bits(leaf, g.h - g.sV);
            float2 vp[kLeafMax];
#pragma unroll
            for (int aa = 0; aa < kLeafMax; ++aa)
                if (aa < na) vp[aa] = __ldg(a.VP + int64_t(aa) * a.n + xg);
            float2 out = make_float2(0.f, 0.f);
#pragma unroll
            for (int aa = 0; aa < kLeafMax; ++aa) {
                if (aa >= na) break;
                float2 c[R];
                load_pair(Sc, aa * nl + slotl, c);
                float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                for (int t = 0; t < R; ++t) {
                    const float pv = sPV[qq * RS + t];
                    acc.x = fmaf(pv, c[t].x, acc.x);
                    acc.y = fmaf(pv, c[t].y, acc.y);
                }
                cfmac(out, vp[aa], acc);
            }
            a.Y[int64_t(col0 + col) * a.ldy + xg] = out;
        }
    } else {
        mid_copy<false>(S, a.mid, P, KC, kc,   // middle state out
                        [&](int col, int lp) { return (int64_t(col0 + col) * a.n + int64_t(lp) * nmid + box) * R; },
                        [](int lp) { return lp; });
    }
    if (TC && nlev > 0) tc_teardown(tc);
}

template <bool ADJ, int MODE>
__global__ void __launch_bounds__(NT, 1) k_left3(HalfArgs a) {
    left3_body<ADJ, MODE>(a, blockIdx.y, blockIdx.x * (NT >> (a.L - a.h)));
}
template <bool ADJ, int MODE>
__global__ void __launch_bounds__(NT, 1) k_right3(HalfArgs a) {
    right3_body<ADJ, MODE>(a, blockIdx.y, blockIdx.x * (NT >> a.h));
}

// Grouped launch over several operators: CTA b runs item items[b] =
// (operator, box, first column) of the operators' half passes.
template <bool ADJ, int MODE>
__global__ void __launch_bounds__(NT, 1) k_left3_group(const HalfArgs* __restrict__ args, const int4* __restrict__ items) {
    const int4 it = items[blockIdx.x];
    left3_body<ADJ, MODE>(args[it.x], it.y, it.z);
}
template <bool ADJ, int MODE>
__global__ void __launch_bounds__(NT, 1) k_right3_group(const HalfArgs* __restrict__ args, const int4* __restrict__ items) {
    const int4 it = items[blockIdx.x];
    right3_body<ADJ, MODE>(args[it.x], it.y, it.z);
}

// Dynamic shared memory: state (64 KiB), one or two table buffers of P * 256 B, Lagrange
// tables, and (aligned to 128 B) the B operands of the tensor-core levels.  Tensor-core
// launches ask for at least kSmemTcMin so that one CTA -- which holds all 512 TMEM
// columns -- is resident per SM.
constexpr size_t kSmemB = 2 * kBBytesSM + 128;
inline size_t smem3(int P) {
    return size_t(NT) * R * 8 + size_t(P <= 256 ? 2 : 1) * P * 256 + (2 * PCS + kLeafMax * RS) * sizeof(float) + kSmemB;
}
constexpr size_t kSmem3Max =
    size_t(NT) * R * 8 + size_t(2) * 256 * 256 + (2 * PCS + kLeafMax * RS) * sizeof(float) + kSmemB;
constexpr size_t kSmemTcMin = 120 * 1024;
inline size_t smem3_launch(int P, int mode) { return mode == kSimt ? smem3(P) : std::max(smem3(P), kSmemTcMin); }

template <int MODE> cudaError_t set_attrs3_t() {
    const int mx = int(kSmem3Max);
    const void* fns[] = {(const void*)k_left3<true, MODE>,        (const void*)k_left3<false, MODE>,
                         (const void*)k_right3<true, MODE>,       (const void*)k_right3<false, MODE>,
                         (const void*)k_left3_group<true, MODE>,  (const void*)k_left3_group<false, MODE>,
                         (const void*)k_right3_group<true, MODE>, (const void*)k_right3_group<false, MODE>};
    for (const void* f : fns) {
        const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}
inline fio_status set_attrs3() {
    static PerDeviceOnce attrs;
    FIO_CUDA(attrs.run([] {
        cudaError_t e = set_attrs3_t<kSimt>();
        if (e == cudaSuccess) e = set_attrs3_t<kTcF16>();
        return e == cudaSuccess ? set_attrs3_t<kTcBF16>() : e;
    }));
    return FIO_OK;
}

template <bool ADJ>
fio_status left3(const fio_bf* bf, const HalfArgs& a, int kcols, cudaStream_t st) {
    FIO_TRY(set_attrs3());
    const int P = 1 << (bf->L - bf->h), KC = NT / P;
    dim3 g((kcols + KC - 1) / KC, 1 << bf->h);
    const char* nm = ADJ ? "k_bf_left_adj" : "k_bf_left_fwd";
    const size_t sm = smem3_launch(P, a.mode);
    if (a.mode == kTcF16) FIO_LAUNCH(nm, st, k_left3<ADJ, kTcF16><<<g, NT, sm, st>>>(a));
    else if (a.mode == kTcBF16) FIO_LAUNCH(nm, st, k_left3<ADJ, kTcBF16><<<g, NT, sm, st>>>(a));
    else FIO_LAUNCH(nm, st, k_left3<ADJ, kSimt><<<g, NT, sm, st>>>(a));
    return FIO_OK;
}
template <bool ADJ>
fio_status right3(const fio_bf* bf, const HalfArgs& a, int kcols, cudaStream_t st) {
    FIO_TRY(set_attrs3());
    const int P = 1 << bf->h, KC = NT / P;
    dim3 g((kcols + KC - 1) / KC, 1 << (bf->L - bf->h));
    const char* nm = ADJ ? "k_bf_right_adj" : "k_bf_right_fwd";
    const size_t sm = smem3_launch(P, a.mode);
    if (a.mode == kTcF16) FIO_LAUNCH(nm, st, k_right3<ADJ, kTcF16><<<g, NT, sm, st>>>(a));
    else if (a.mode == kTcBF16) FIO_LAUNCH(nm, st, k_right3<ADJ, kTcBF16><<<g, NT, sm, st>>>(a));
    else FIO_LAUNCH(nm, st, k_right3<ADJ, kSimt><<<g, NT, sm, st>>>(a));
    return FIO_OK;
}

// ---------------------------------------------------------------- persistent batched solve
// One launch for the whole batched online stage (f = G~^{-1} K~^* u of many operators): a
// grid of one CTA per SM walks a device work list of (stage, operator, block) items in
// dependency order -- BF left half passes, right half passes, ULV up levels, roots, ULV down
// levels.  A CTA takes the next item with an atomic, waits (thread 0, bounded spin) until the
// item's prerequisite counter reaches its target -- the number of items of the previous stage
// of the same operator -- runs it, and counts it done.  Items wait only on items taken before
// them by running CTAs, so the walk cannot deadlock; a wait that runs out sets a device flag
// (reported as FIO_ETIMEOUT by fio_device_status) and the item proceeds.
__device__ int g_persist_timeout = 0;

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <int MODE>
__global__ void __launch_bounds__(NT, 1) k_batch_persistent(const HalfArgs* __restrict__ largs,
                                                            const HalfArgs* __restrict__ rargs,
                                                            const UlvGemmDesc* __restrict__ udesc,
                                                            const UlvRootDesc* __restrict__ rdesc,
                                                            const PItem* __restrict__ items, int nitems,
                                                            int* __restrict__ head, int* __restrict__ counters,
                                                            int spin_limit) {
    extern __shared__ float4 smem4[];
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) {
            const int i = atomicAdd(head, 1);
            s_item = i;
            if (i < nitems && items[i].dep >= 0) {
                const PItem it = items[i];
                int n = 0;
                while (ld_acquire(counters + it.dep) < it.target) {
                    if (++n > spin_limit) {
                        atomicExch(&g_persist_timeout, 1);
                        break;
                    }
                    __nanosleep(128);
                }
                __threadfence();
            }
        }
        __syncthreads();
        const int i = s_item;
        if (i >= nitems) break;
        const PItem it = items[i];
        if (it.type == kPLeft) {
            left3_body<true, MODE>(largs[it.a], it.b, it.c);
        } else if (it.type == kPRight) {
            right3_body<true, MODE>(rargs[it.a], it.b, it.c);
        } else if (it.type == kPRoot) {
            if (threadIdx.x < ulvb::kUlvThreads) {
                const UlvRootDesc& g = rdesc[it.a];
                ulvb::root_body(g.A, g.m, g.x, g.y, g.k, threadIdx.x);
            }
        } else {
            // two node-product blocks of one stage, one per half of the CTA (own tiles and barrier)
            const int half = threadIdx.x / ulvb::kUlvThreads, tid = threadIdx.x % ulvb::kUlvThreads;
            const int t = half ? it.b2 : it.b, c0 = half ? it.c2 : it.c, r0 = half ? it.d2 : it.d;
            if (t >= 0) {
                float2* sx = reinterpret_cast<float2*>(smem4) + half * ulvb::WT * (ulvb::KCOL + ulvb::RB);
                float2* sw = sx + ulvb::WT * ulvb::KCOL;
                auto sync = [half] {
                    if (half) asm volatile("bar.sync 4, 256;" ::: "memory");
                    else asm volatile("bar.sync 3, 256;" ::: "memory");
                };
                const UlvGemmDesc& g = udesc[it.a];
                if (it.type == kPUp)
                    ulvb::node_gemm_body<false>(g.W, g.m, g.inA, g.nA, g.ldA, g.inB, g.ldB, g.outC, g.nC, g.ldC, g.outD,
                                                g.ldD, g.k, t, c0, r0, sx, sw, sync, tid);
                else
                    ulvb::node_gemm_body<true>(g.W, g.m, g.inA, g.nA, g.ldA, g.inB, g.ldB, g.outC, g.nC, g.ldC, g.outD,
                                               g.ldD, g.k, t, c0, r0, sx, sw, sync, tid);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(counters + it.done, 1);
        }
    }
}

}  // namespace v3

}  // namespace

fio_status batch_persistent_launch(const void* dleft_args, const void* dright_args, const UlvGemmDesc* udesc,
                                   const UlvRootDesc* rdesc, const PItem* items, int nitems, int* head_and_counters,
                                   int ncounters, int mode, int spin_limit, cudaStream_t st) {
    if (nitems == 0) return FIO_OK;
    FIO_TRY(v3::set_attrs3());
    static PerDeviceOnce attrs;
    FIO_CUDA(attrs.run([] {
        const void* fns[] = {(const void*)v3::k_batch_persistent<v3::kSimt>, (const void*)v3::k_batch_persistent<v3::kTcF16>,
                             (const void*)v3::k_batch_persistent<v3::kTcBF16>};
        for (const void* f : fns) {
            const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, int(v3::kSmem3Max));
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }));
    int dev = 0, sms = 0;
    FIO_CUDA(cudaGetDevice(&dev));
    FIO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    FIO_CUDA(cudaMemsetAsync(head_and_counters, 0, sizeof(int) * (1 + ncounters), st));
    const int grid = std::min(sms, nitems);
    const HalfArgs* la = static_cast<const HalfArgs*>(dleft_args);
    const HalfArgs* ra = static_cast<const HalfArgs*>(dright_args);
    int* head = head_and_counters;
    int* ctr = head_and_counters + 1;
    const size_t sm = v3::kSmem3Max;
    if (mode == v3::kTcF16)
        FIO_LAUNCH("k_batch_persistent", st, (v3::k_batch_persistent<v3::kTcF16><<<grid, v3::NT, sm, st>>>(
                                                 la, ra, udesc, rdesc, items, nitems, head, ctr, spin_limit)));
    else if (mode == v3::kTcBF16)
        FIO_LAUNCH("k_batch_persistent", st, (v3::k_batch_persistent<v3::kTcBF16><<<grid, v3::NT, sm, st>>>(
                                                 la, ra, udesc, rdesc, items, nitems, head, ctr, spin_limit)));
    else
        FIO_LAUNCH("k_batch_persistent", st, (v3::k_batch_persistent<v3::kSimt><<<grid, v3::NT, sm, st>>>(
                                                 la, ra, udesc, rdesc, items, nitems, head, ctr, spin_limit)));
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}

// ---------------------------------------------------------------- grouped
// Host tables of a grouped half-pass launch over several operators.
void bf_group_tables(const std::vector<BfGroupOp>& ops, int adjoint, std::vector<unsigned char>& left_args,
                     std::vector<int4>& left_items, std::vector<unsigned char>& right_args,
                     std::vector<int4>& right_items) {
    left_args.assign(ops.size() * sizeof(HalfArgs), 0);
    right_args.assign(ops.size() * sizeof(HalfArgs), 0);
    left_items.clear();
    right_items.clear();
    for (size_t o = 0; o < ops.size(); ++o) {
        const fio_bf* bf = ops[o].bf;
        HalfArgs a{};
        a.ldx = a.ldy = bf->n;
        a.mid = ops[o].mid;
        a.VP = bf->VP.as<float2>();
        a.UP = bf->UP.as<float2>();
        a.M = bf->M.as<float2>();
        a.P = bf->P.as<float>();
        a.pu_off = int(bf->pu_off());
        a.pc_off = int(bf->pc_off());
        a.n = bf->n;
        a.L = bf->L;
        a.h = bf->h;
        a.sU = bf->sU;
        a.sV = bf->sV;
        a.k = ops[o].k;
        a.mode = bf_fused_mode(bf, -1);
        HalfArgs al = a, ar = a;
        for (size_t i = 0; i < bf->B.size() && i < 24; ++i) al.tab.t[i] = bf->B[i].as<float2>();
        for (size_t i = 0; i < bf->C.size() && i < 24; ++i) ar.tab.t[i] = bf->C[i].as<float2>();
        const int dir = adjoint ? 1 : 0;
        for (size_t i = 0; i < bf->Bst[dir].size() && i < 24; ++i) al.tabs.t[i] = bf->Bst[dir][i].as<float2>();
        for (size_t i = 0; i < bf->Cst[dir].size() && i < 24; ++i) ar.tabs.t[i] = bf->Cst[dir][i].as<float2>();
        al.Ms = nullptr;
        ar.Ms = (!adjoint && bf->Mst.p) ? bf->Mst.as<float2>() : nullptr;
        // adjoint: left reads X, writes mid; right reads mid, writes Y.  forward: the reverse.
        if (adjoint) {
            al.X = ops[o].X;
            ar.Y = ops[o].Y;
        } else {
            ar.X = ops[o].X;
            al.Y = ops[o].Y;
        }
        std::memcpy(left_args.data() + o * sizeof(HalfArgs), &al, sizeof(HalfArgs));
        std::memcpy(right_args.data() + o * sizeof(HalfArgs), &ar, sizeof(HalfArgs));
        const int Pl = 1 << (bf->L - bf->h), Pr = 1 << bf->h;
        const int KCl = v3::NT / Pl, KCr = v3::NT / Pr;
        for (int c0 = 0; c0 < ops[o].k; c0 += KCl)
            for (int b = 0; b < (1 << bf->h); ++b) left_items.push_back(make_int4(int(o), b, c0, 0));
        for (int c0 = 0; c0 < ops[o].k; c0 += KCr)
            for (int b = 0; b < (1 << (bf->L - bf->h)); ++b) right_items.push_back(make_int4(int(o), b, c0, 0));
    }
}

size_t bf_group_args_size() { return sizeof(HalfArgs); }

// Launch the two grouped halves (device copies of the tables of bf_group_tables); `mode`
// is the transfer-level mode shared by every operator of the launch (bf_fused_mode).
fio_status bf_group_launch(const void* dleft_args, const int4* dleft_items, int nleft, const void* dright_args,
                           const int4* dright_items, int nright, int adjoint, int mode, cudaStream_t st) {
    FIO_TRY(v3::set_attrs3());
    const HalfArgs* la = static_cast<const HalfArgs*>(dleft_args);
    const HalfArgs* ra = static_cast<const HalfArgs*>(dright_args);
    const size_t sm = v3::kSmem3Max;
    const int NT = v3::NT;
    auto left = [&](auto kern, const char* nm) -> fio_status {
        if (nleft) FIO_LAUNCH(nm, st, kern<<<nleft, NT, sm, st>>>(la, dleft_items));
        return FIO_OK;
    };
    auto right = [&](auto kern, const char* nm) -> fio_status {
        if (nright) FIO_LAUNCH(nm, st, kern<<<nright, NT, sm, st>>>(ra, dright_items));
        return FIO_OK;
    };
    using namespace v3;
    if (adjoint) {
        if (mode == kTcF16) {
            FIO_TRY(left(k_left3_group<true, kTcF16>, "k_bf_left_adj_group"));
            FIO_TRY(right(k_right3_group<true, kTcF16>, "k_bf_right_adj_group"));
        } else if (mode == kTcBF16) {
            FIO_TRY(left(k_left3_group<true, kTcBF16>, "k_bf_left_adj_group"));
            FIO_TRY(right(k_right3_group<true, kTcBF16>, "k_bf_right_adj_group"));
        } else {
            FIO_TRY(left(k_left3_group<true, kSimt>, "k_bf_left_adj_group"));
            FIO_TRY(right(k_right3_group<true, kSimt>, "k_bf_right_adj_group"));
        }
    } else {
        if (mode == kTcF16) {
            FIO_TRY(right(k_right3_group<false, kTcF16>, "k_bf_right_fwd_group"));
            FIO_TRY(left(k_left3_group<false, kTcF16>, "k_bf_left_fwd_group"));
        } else if (mode == kTcBF16) {
            FIO_TRY(right(k_right3_group<false, kTcBF16>, "k_bf_right_fwd_group"));
            FIO_TRY(left(k_left3_group<false, kTcBF16>, "k_bf_left_fwd_group"));
        } else {
            FIO_TRY(right(k_right3_group<false, kSimt>, "k_bf_right_fwd_group"));
            FIO_TRY(left(k_left3_group<false, kSimt>, "k_bf_left_fwd_group"));
        }
    }
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}

// Transfer-level mode of the staged fused kernels for this handle: split precision ->
// BF16 parts on the tensor cores; the FP32 setting -> FP16 parts on the tensor cores,
// or CUDA-core FP32 when the handle asks for it.  prec: -1 the handle's precision,
// 0 FP32, 1 split BF16.
int bf_fused_mode(const fio_bf* bf, int prec) {
    const bool split = prec < 0 ? bf->split : prec == 1;
    if (split) return v3::kTcBF16;
    return bf->simt ? v3::kSimt : v3::kTcF16;
}

fio_status bf_prestage(fio_bf* bf, cudaStream_t st) {
    using namespace v3;
    if (!bf_v3_ok(bf)) return FIO_OK;
    const int64_t bytes = int64_t(bf->n) / 2 * 4 * R * 8;   // one level's table
    for (int side = 0; side < 2; ++side) {                   // 0 right (C levels), 1 left (B levels)
        Geo g;
        g.L = bf->L; g.h = bf->h; g.sU = bf->sU; g.sV = bf->sV; g.n = bf->n;
        g.lgP = side ? bf->L - bf->h : bf->h;
        g.P = 1 << g.lgP;
        g.KC = NT >> g.lgP;
        const int nbox = side ? 1 << bf->h : 1 << (bf->L - bf->h);
        std::vector<DevBuf>* dst = side ? bf->Bst : bf->Cst;
        const std::vector<DevBuf>& src = side ? bf->B : bf->C;
        const int s0 = side ? bf->h : bf->sV;
        for (int adj = 0; adj < 2; ++adj) {
            dst[adj].resize(src.size());
            for (size_t i = 0; i < src.size(); ++i) {
                FIO_TRY(dst[adj][i].ensure(size_t(bytes)));
                float4* d = dst[adj][i].as<float4>();
                const float2* t = src[i].as<float2>();
                const int s = s0 + int(i);
                if (side && adj) k_prestage<true, true><<<nbox, 256, 0, st>>>(d, t, g, s);
                else if (side) k_prestage<true, false><<<nbox, 256, 0, st>>>(d, t, g, s);
                else if (adj) k_prestage<false, true><<<nbox, 256, 0, st>>>(d, t, g, s);
                else k_prestage<false, false><<<nbox, 256, 0, st>>>(d, t, g, s);
            }
        }
    }
    {   // the forward middle factor for the right half
        Geo g;
        g.L = bf->L; g.h = bf->h; g.sU = bf->sU; g.sV = bf->sV; g.n = bf->n;
        g.lgP = bf->h;
        g.P = 1 << g.lgP;
        g.KC = NT >> g.lgP;
        FIO_TRY(bf->Mst.ensure(bf->M.bytes));
        k_prestage_m<<<dim3(1 << (bf->L - bf->h), 8), 256, 0, st>>>(bf->Mst.as<float4>(), bf->M.as<float2>(), g);
    }
    FIO_CUDA(cudaGetLastError());
    bf->table_bytes += 2 * int64_t(bf->C.size() + bf->B.size()) * bytes + int64_t(bf->M.bytes);
    return FIO_OK;
}

int tc_wait_timeouts() {
    int v = 0, w = 0;
    if (cudaMemcpyFromSymbol(&v, v3::g_tc_wait_timeout, sizeof(int)) != cudaSuccess) return -1;
    if (cudaMemcpyFromSymbol(&w, v3::g_persist_timeout, sizeof(int)) != cudaSuccess) return -1;
    const int z = 0;
    if (v) cudaMemcpyToSymbol(v3::g_tc_wait_timeout, &z, sizeof(int));
    if (w) cudaMemcpyToSymbol(v3::g_persist_timeout, &z, sizeof(int));
    return v | w;
}

bool bf_v3_ok(const fio_bf* bf) {
    const int Pl = 1 << (bf->L - bf->h), Pr = 1 << bf->h;
    return bf->r == R && Pl >= 64 && Pl <= 512 && Pr >= 64 && Pr <= 512;
}

bool bf_fused_ok(const fio_bf* bf) {
    if (bf->r != R || bf->L < 6) return false;
    const int Pl = 1 << (bf->L - bf->h), Pr = 1 << bf->h;
    return Pl <= 512 && Pr <= 512 && bf->sU - bf->h <= 23 && bf->h - bf->sV <= 23;
}

// Columns per CTA: 64 KiB of in-place state (KC * P * 128 B) per CTA, two CTAs per SM.
int bf_fused_kc(const fio_bf* bf) {
    const int P = std::max(1 << (bf->L - bf->h), 1 << bf->h);
    return P <= 128 ? 4 : (P <= 256 ? 2 : 1);
}

fio_status bf_apply_fused(const fio_bf* bf, const float2* X, float2* Y, int64_t ld, int kcols, int adjoint,
                          float2* mid, cudaStream_t st, int prec) {
    HalfArgs a{};
    a.X = X;
    a.ldx = ld;
    a.Y = Y;
    a.ldy = ld;
    a.mid = mid;
    a.VP = bf->VP.as<float2>();
    a.UP = bf->UP.as<float2>();
    a.M = bf->M.as<float2>();
    a.P = bf->P.as<float>();
    a.pu_off = int(bf->pu_off());
    a.pc_off = int(bf->pc_off());
    a.n = bf->n;
    a.L = bf->L;
    a.h = bf->h;
    a.sU = bf->sU;
    a.sV = bf->sV;
    a.k = kcols;
    a.mode = bf_fused_mode(bf, prec);
    // the left kernels read E tables (B levels), the right kernels F tables (C levels)
    Tabs tl{}, tr{};
    for (size_t i = 0; i < bf->B.size() && i < 24; ++i) tl.t[i] = bf->B[i].as<float2>();
    for (size_t i = 0; i < bf->C.size() && i < 24; ++i) tr.t[i] = bf->C[i].as<float2>();
    if (bf_v3_ok(bf) && (!bf->fused_v2 || a.mode == v3::kTcBF16)) {
        HalfArgs al = a, ar = a;
        al.tab = tl;
        ar.tab = tr;
        al.tabs = Tabs{};
        ar.tabs = Tabs{};
        for (size_t i = 0; i < bf->Bst[adjoint ? 1 : 0].size() && i < 24; ++i) al.tabs.t[i] = bf->Bst[adjoint ? 1 : 0][i].as<float2>();
        for (size_t i = 0; i < bf->Cst[adjoint ? 1 : 0].size() && i < 24; ++i) ar.tabs.t[i] = bf->Cst[adjoint ? 1 : 0][i].as<float2>();
        al.Ms = nullptr;
        ar.Ms = (!adjoint && bf->Mst.p) ? bf->Mst.as<float2>() : nullptr;
        if (adjoint) {
            FIO_TRY(v3::left3<true>(bf, al, kcols, st));
            FIO_TRY(v3::right3<true>(bf, ar, kcols, st));
        } else {
            FIO_TRY(v3::right3<false>(bf, ar, kcols, st));
            FIO_TRY(v3::left3<false>(bf, al, kcols, st));
        }
        FIO_CUDA(cudaGetLastError());
        return FIO_OK;
    }
    const int KC = bf_fused_kc(bf);
    if (adjoint) {
        a.tab = tl;
        HalfArgs b = a;
        b.tab = tr;
        // left pass reads X, writes mid; right pass reads mid, writes Y
        if (KC == 4) FIO_TRY(launch_fused_pass<4>(bf, a, b, true, kcols, st));
        else if (KC == 2) FIO_TRY(launch_fused_pass<2>(bf, a, b, true, kcols, st));
        else FIO_TRY(launch_fused_pass<1>(bf, a, b, true, kcols, st));
    } else {
        a.tab = tr;
        HalfArgs b = a;
        b.tab = tl;
        if (KC == 4) FIO_TRY(launch_fused_pass<4>(bf, a, b, false, kcols, st));
        else if (KC == 2) FIO_TRY(launch_fused_pass<2>(bf, a, b, false, kcols, st));
        else FIO_TRY(launch_fused_pass<1>(bf, a, b, false, kcols, st));
    }
    return FIO_OK;
}

}  // namespace fio
