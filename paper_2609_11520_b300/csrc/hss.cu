// Randomized black-box HSS construction (Section 3.1-3.3), HSS matrix-vector
// product (Eq. 2.8) and handle management.
#include <algorithm>
#include <cmath>

#include "bf.cuh"
#include "cplx.cuh"
#include "hss.cuh"

namespace fio {
namespace {

constexpr int TB = 256;

// ----------------------------------------------------------- test matrices
// Philox4x32-10 (Salmon et al., SC 2011): 10 rounds, multipliers
// 0xD2511F53 / 0xCD9E8D57, Weyl key increments 0x9E3779B9 / 0xBB67AE85.
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
    for (int rnd = 0; rnd < 10; ++rnd) {
        if (rnd) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
        uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

// Omega (rows x cols, column-major): entry (i, j) from counter (i, j, level,
// attempt); Box-Muller on the first two words gives Re, Im ~ N(0, 1).
__global__ void k_gauss(float2* Om, int64_t rows, int cols, int level, int attempt, uint32_t k0, uint32_t k1) {
    int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= rows * cols) return;
    int64_t i = e % rows, j = e / rows;
    uint32_t c[4] = {uint32_t(i), uint32_t(j), uint32_t(level), uint32_t(attempt)};
    philox4x32_10(c, k0, k1);
    double u1 = (double(c[0]) + 0.5) * 0x1p-32, u2 = (double(c[1]) + 0.5) * 0x1p-32;
    double rad = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    Om[e] = make_float2(float(rad * cs), float(rad * sn));
}

// ----------------------------------------------------------- dense sampler
// Z = H X, H column-major N x N; 16 x 16 shared-memory tiles.
__global__ void k_dense_gemm(const float2* __restrict__ H, int64_t ldh, const float2* __restrict__ X, int64_t ldx,
                             float2* __restrict__ Z, int64_t ldz, int64_t N, int s) {
    __shared__ float2 sA[16][17], sB[16][17];
    int tx = threadIdx.x, ty = threadIdx.y;
    int64_t row = int64_t(blockIdx.x) * 16 + tx;
    int col = blockIdx.y * 16 + ty;
    float2 acc = make_float2(0.f, 0.f);
    for (int64_t k0 = 0; k0 < N; k0 += 16) {
        sA[ty][tx] = (row < N && k0 + ty < N) ? H[row + (k0 + ty) * ldh] : make_float2(0.f, 0.f);
        int colb = blockIdx.y * 16 + ty;
        sB[ty][tx] = (k0 + tx < N && colb < s) ? X[(k0 + tx) + colb * ldx] : make_float2(0.f, 0.f);
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) cfma(acc, sA[kk][tx], sB[ty][kk]);
        __syncthreads();
    }
    if (row < N && col < s) Z[row + col * ldz] = acc;
}

// ----------------------------------------------------------- node kernels
// LQ of Omega_t (m x s) by Householder reflectors applied from the right,
// the same reflectors applied to Y_t:
//   Omega_t H_1..H_m = [L, 0],   Y_t H_1..H_m = [Y Q1, Y Gamma].
// Gamma = last s-m columns of Q = H_1..H_m is an orthonormal basis of
// null(Omega_t) (Section 3.1).  Then W = Y Omega^+ = (Y Q1) L^{-1} overwrites
// Y Q1.  Workspace per node: row-major [2m][s] (Omega rows, then Y rows).
// thr[t] = tol * max_j ||Y_t(:, j)||.
template <class C>
__global__ void k_node_lq(const float2* __restrict__ Om, const float2* __restrict__ Y, int64_t ld, int m, int s,
                          C* __restrict__ WS, double* __restrict__ thr, double tol) {
    using R = typename RealOf<C>::T;
    extern __shared__ unsigned char smem_raw[];
    C* v = reinterpret_cast<C*>(smem_raw);
    __shared__ R red[32];
    const int t = blockIdx.x, tid = threadIdx.x, bd = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = bd >> 5;
    C* A = WS + int64_t(t) * 2 * m * s;
    for (int64_t e = tid; e < int64_t(m) * s; e += bd) {
        int i = int(e % m), j = int(e / m);
        A[int64_t(i) * s + j] = cvt<C>(Om[(int64_t(t) * m + i) + j * ld]);
        A[int64_t(m + i) * s + j] = cvt<C>(Y[(int64_t(t) * m + i) + j * ld]);
    }
    __syncthreads();
    R mx = 0;
    for (int j = tid; j < s; j += bd) {
        R a = 0;
        for (int i = 0; i < m; ++i) a += gabs2(A[int64_t(m + i) * s + j]);
        mx = a > mx ? a : mx;
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    if (tid == 0) {
        R g = 0;
        for (int w = 0; w < nw; ++w) g = fmax(g, red[w]);
        thr[t] = tol * sqrt(double(g));
    }
    __syncthreads();
    for (int k = 0; k < m; ++k) {
        C* Ak = A + int64_t(k) * s;
        R xn = 0;
        for (int j = k + 1 + tid; j < s; j += bd) xn += gabs2(Ak[j]);
        xn = block_sum(xn, red);
        C alpha = gconj(Ak[k]);
        R beta;
        C tau, scal;
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
        for (int j = k + tid; j < s; j += bd) v[j] = (j == k) ? mkc<C>(1, 0) : gmul(gconj(Ak[j]), scal);
        __syncthreads();
        for (int i = k + 1 + warp; i < 2 * m; i += nw) {
            C* Ai = A + int64_t(i) * s;
            C w = czero<C>();
            for (int j = k + lane; j < s; j += 32) gfma(w, Ai[j], v[j]);
            w.x = warp_sum(w.x);
            w.y = warp_sum(w.y);
            C tw = gmul(tau, w);
            for (int j = k + lane; j < s; j += 32) Ai[j] = gsub(Ai[j], gmul(tw, gconj(v[j])));
        }
        __syncthreads();
        for (int j = k + tid; j < s; j += bd) Ak[j] = (j == k) ? mkc<C>(beta, 0) : czero<C>();
        __syncthreads();
    }
    // W L = Y Q1, row by row (one warp per row, column sweep from the last column).
    for (int i = warp; i < m; i += nw) {
        C* y = A + int64_t(m + i) * s;
        for (int j = m - 1; j >= 0; --j) {
            C wj = gdiv(y[j], A[int64_t(j) * s + j]);
            __syncwarp();
            for (int l = lane; l < j; l += 32) y[l] = gsub(y[l], gmul(wj, A[int64_t(j) * s + l]));
            if (lane == 0) y[j] = wj;
            __syncwarp();
        }
    }
}

// Column-pivoted Householder QR (Businger-Golub) of Y_t Gamma (m x c, c = s-m,
// rows m.. of the workspace, columns m..), K steps.  |R_kk| = |beta_k|;
// khat = number of leading pivots above thr; sat = 1 when after K steps a
// remaining column still exceeds thr.  Reflector k: v (v_k = 1) stored below
// the diagonal of column k, tau in taus[t][k].
template <class C>
__global__ void k_node_qrcp(C* __restrict__ WS, int m, int s, int K, const double* __restrict__ thr, int* khat,
                            int* sat, C* __restrict__ taus) {
    using R = typename RealOf<C>::T;
    extern __shared__ unsigned char smem_raw[];
    const int c = s - m;
    R* cn = reinterpret_cast<R*>(smem_raw);                 // c
    C* v = reinterpret_cast<C*>(cn + ((c + 1) & ~1));       // m
    __shared__ R red[32];
    __shared__ R redv[32];
    __shared__ int redi[32];
    __shared__ int s_khat;
    const int t = blockIdx.x, tid = threadIdx.x, bd = blockDim.x;
    C* base = WS + int64_t(t) * 2 * m * s + int64_t(m) * s + m;   // A[i][j] = base[i*s + j]
    const R th = R(thr[t]);
    if (tid == 0) s_khat = -1;
    for (int k = 0; k < K; ++k) {
        for (int j = k + tid; j < c; j += bd) {
            R a = 0;
            for (int i = k; i < m; ++i) a += gabs2(base[int64_t(i) * s + j]);
            cn[j] = a;
        }
        __syncthreads();
        R bv = -1;
        int bi = 0x7fffffff;
        for (int j = k + tid; j < c; j += bd)
            if (cn[j] > bv) { bv = cn[j]; bi = j; }
        block_argmax(bv, bi, redv, redi);
        const int p = bi;
        if (p != k)
            for (int i = tid; i < m; i += bd) {
                C a = base[int64_t(i) * s + k];
                base[int64_t(i) * s + k] = base[int64_t(i) * s + p];
                base[int64_t(i) * s + p] = a;
            }
        __syncthreads();
        R xn = 0;
        for (int i = k + 1 + tid; i < m; i += bd) xn += gabs2(base[int64_t(i) * s + k]);
        xn = block_sum(xn, red);
        C alpha = base[int64_t(k) * s + k];
        R beta;
        C tau, scal;
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
        if (tid == 0 && s_khat < 0 && !(fabs(double(beta)) > double(th))) s_khat = k;
        for (int i = k + tid; i < m; i += bd) v[i] = (i == k) ? mkc<C>(1, 0) : gmul(base[int64_t(i) * s + k], scal);
        __syncthreads();
        for (int j = k + 1 + tid; j < c; j += bd) {
            C w = czero<C>();
            for (int i = k; i < m; ++i) gfmac(w, v[i], base[int64_t(i) * s + j]);
            C tw = gmulc(tau, w);   // conj(tau) * w
            for (int i = k; i < m; ++i) base[int64_t(i) * s + j] = gsub(base[int64_t(i) * s + j], gmul(v[i], tw));
        }
        for (int i = k + tid; i < m; i += bd) base[int64_t(i) * s + k] = (i == k) ? mkc<C>(beta, 0) : v[i];
        if (tid == 0) taus[int64_t(t) * K + k] = tau;
        __syncthreads();
    }
    // saturation: largest remaining column after K steps
    R rem = 0;
    if (K < m)
        for (int j = K + tid; j < c; j += bd) {
            R a = 0;
            for (int i = K; i < m; ++i) a += gabs2(base[int64_t(i) * s + j]);
            rem = a > rem ? a : rem;
        }
    for (int o = 16; o > 0; o >>= 1) rem = fmax(rem, __shfl_xor_sync(0xffffffffu, rem, o));
    if ((tid & 31) == 0) red[tid >> 5] = rem;
    __syncthreads();
    if (tid == 0) {
        R g = 0;
        for (int w = 0; w < (bd >> 5); ++w) g = fmax(g, red[w]);
        khat[t] = s_khat < 0 ? K : s_khat;
        sat[t] = (sqrt(double(g)) > double(th)) ? 1 : 0;
    }
}

// U_t = H_1 .. H_r [I_r; 0] (first r columns of the QRCP's Q), stored
// complex64 column-major m x r.  One warp per column.
template <class C>
__global__ void k_node_formU(const C* __restrict__ WS, int m, int s, int K, int r, const C* __restrict__ taus,
                             float2* __restrict__ Uout, C* __restrict__ E) {
    const int t = blockIdx.x, tid = threadIdx.x, bd = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = bd >> 5;
    const C* base = WS + int64_t(t) * 2 * m * s + int64_t(m) * s + m;
    C* Et = E + int64_t(t) * m * r;
    for (int e = tid; e < m * r; e += bd) {
        int i = e % m, cc = e / m;
        Et[e] = (i == cc) ? mkc<C>(1, 0) : czero<C>();
    }
    __syncthreads();
    for (int k = r - 1; k >= 0; --k) {
        C tau = taus[int64_t(t) * K + k];
        for (int cc = warp; cc < r; cc += nw) {
            C* col = Et + int64_t(cc) * m;
            C w = czero<C>();
            for (int i = k + lane; i < m; i += 32) {
                C vi = (i == k) ? mkc<C>(1, 0) : base[int64_t(i) * s + k];
                gfmac(w, vi, col[i]);
            }
            w.x = warp_sum(w.x);
            w.y = warp_sum(w.y);
            C tw = gmul(tau, w);
            for (int i = k + lane; i < m; i += 32) {
                C vi = (i == k) ? mkc<C>(1, 0) : base[int64_t(i) * s + k];
                col[i] = gsub(col[i], gmul(vi, tw));
            }
        }
        __syncthreads();
    }
    for (int e = tid; e < m * r; e += bd) Uout[int64_t(t) * m * r + e] = to_f2(Et[e]);
}

// D-check (Section 3.1): X = (I - U U^*) W,  D = X + U U^* X^*, with W the
// Y Omega^+ block of the workspace (row-major m x m).  Output complex64
// column-major m x m.  Scratch per node: T (r x m) then T2 (m x r).
template <class C>
__global__ void k_node_dcheck(C* __restrict__ WS, int m, int s, const float2* __restrict__ U, int r,
                              float2* __restrict__ Dout, C* __restrict__ scratch) {
    const int t = blockIdx.x, tid = threadIdx.x, bd = blockDim.x;
    C* Wm = WS + int64_t(t) * 2 * m * s + int64_t(m) * s;   // W[i][j] = Wm[i*s + j]
    const float2* Ut = U + int64_t(t) * m * r;              // Ut[i + c*m]
    C* T1 = scratch + int64_t(t) * 2 * m * r;               // T1[c][j] = T1[c*m + j]
    C* T2 = T1 + int64_t(m) * r;                            // T2[i][c] = T2[i*r + c]
    for (int e = tid; e < r * m; e += bd) {
        int cc = e / m, j = e % m;
        C a = czero<C>();
        for (int i = 0; i < m; ++i) gfmac(a, cvt<C>(Ut[i + int64_t(cc) * m]), Wm[int64_t(i) * s + j]);
        T1[e] = a;
    }
    __syncthreads();
    for (int e = tid; e < m * m; e += bd) {
        int i = e / m, j = e % m;
        C a = Wm[int64_t(i) * s + j];
        for (int cc = 0; cc < r; ++cc) a = gsub(a, gmul(cvt<C>(Ut[i + int64_t(cc) * m]), T1[int64_t(cc) * m + j]));
        Wm[int64_t(i) * s + j] = a;   // X
    }
    __syncthreads();
    for (int e = tid; e < m * r; e += bd) {
        int i = e / r, cc = e % r;
        C a = czero<C>();
        for (int j = 0; j < m; ++j) gfma(a, Wm[int64_t(i) * s + j], cvt<C>(Ut[j + int64_t(cc) * m]));
        T2[e] = a;
    }
    __syncthreads();
    for (int e = tid; e < m * m; e += bd) {
        int i = e % m, j = e / m;   // column-major output
        C a = Wm[int64_t(i) * s + j];
        for (int cc = 0; cc < r; ++cc) {
            C u = cvt<C>(Ut[i + int64_t(cc) * m]);
            a = gadd(a, gmul(u, gconj(T2[int64_t(j) * r + cc])));
        }
        Dout[int64_t(t) * m * m + e] = to_f2(a);
    }
}

// Root: H^[0] = Y^[0] Omega^[0]+ (the W block of the workspace), Hermitian
// part, into a column-major FP64 block.
template <class C>
__global__ void k_root_h0(const C* __restrict__ WS, int m, int s, double2* __restrict__ D0) {
    const C* Wm = WS + int64_t(m) * s;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        int i = e % m, j = e / m;
        C a = Wm[int64_t(i) * s + j], b = Wm[int64_t(j) * s + i];
        D0[e] = make_double2(0.5 * (double(a.x) + double(b.x)), 0.5 * (double(a.y) - double(b.y)));
    }
}

// Postprocessing (Section 3.3), node t of level l: Hermitian part of D_t
// (2rc x 2rc); B = A21; D_child = Dcheck_child + U_child A_cc U_child^*.
__global__ void k_post(const double2* __restrict__ Dcur, int rc, int mc, const float2* __restrict__ Uc,
                       const float2* __restrict__ Dchk, float2* __restrict__ Bout, double2* __restrict__ Dnext,
                       double2* __restrict__ scratch) {
    const int t = blockIdx.x, tid = threadIdx.x, bd = blockDim.x;
    const int mt = 2 * rc;
    const double2* Dt = Dcur + int64_t(t) * mt * mt;
    auto H = [&](int i, int j) {
        double2 a = Dt[i + int64_t(j) * mt], b = Dt[j + int64_t(i) * mt];
        return make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
    };
    for (int e = tid; e < rc * rc; e += bd) {
        int i = e % rc, j = e / rc;
        double2 v = H(rc + i, j);
        Bout[int64_t(t) * rc * rc + e] = make_float2(float(v.x), float(v.y));
    }
    for (int ch = 0; ch < 2; ++ch) {
        const int a = 2 * t + ch;
        const float2* Ua = Uc + int64_t(a) * mc * rc;
        double2* UA = scratch + int64_t(t) * mc * rc;      // U A  (mc x rc, column-major)
        __syncthreads();
        for (int e = tid; e < mc * rc; e += bd) {
            int i = e % mc, j = e / mc;
            double2 acc = make_double2(0, 0);
            for (int q = 0; q < rc; ++q) {
                float2 u = Ua[i + int64_t(q) * mc];
                zfma(acc, make_double2(u.x, u.y), H(ch * rc + q, ch * rc + j));
            }
            UA[e] = acc;
        }
        __syncthreads();
        for (int e = tid; e < mc * mc; e += bd) {
            int i = e % mc, j = e / mc;
            float2 dc = Dchk[int64_t(a) * mc * mc + e];
            double2 acc = make_double2(dc.x, dc.y);
            for (int q = 0; q < rc; ++q) {
                float2 u = Ua[j + int64_t(q) * mc];
                // + (U A)[i][q] * conj(U[j][q])
                double2 ua = UA[i + int64_t(q) * mc];
                acc.x += ua.x * u.x + ua.y * u.y;
                acc.y += ua.y * u.x - ua.x * u.y;
            }
            Dnext[int64_t(a) * mc * mc + e] = acc;
        }
    }
}

// Leaf D: Hermitian part of the final blocks, to complex64.
__global__ void k_leafD(const double2* __restrict__ Dn, int m, int64_t nodes, float2* __restrict__ D) {
    int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= nodes * m * m) return;
    int64_t t = e / (int64_t(m) * m);
    int w = int(e % (int64_t(m) * m)), i = w % m, j = w / m;
    double2 a = Dn[e], b = Dn[t * m * m + j + int64_t(i) * m];
    D[e] = make_float2(float(0.5 * (a.x + b.x)), float(0.5 * (a.y - b.y)));
}

// ----------------------------------------------------------- block products
__global__ void k_expand(const float2* __restrict__ U, int64_t nodes, int m, int r, const float2* __restrict__ in,
                         int64_t ldin, float2* __restrict__ out, int64_t ldout, bool acc) {
    int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= nodes * m) return;
    int col = blockIdx.y;
    int64_t t = e / m;
    int i = int(e % m);
    const float2* Ut = U + t * m * r;
    const float2* x = in + col * ldin + t * r;
    float2 a = acc ? out[col * ldout + e] : make_float2(0.f, 0.f);
    for (int c = 0; c < r; ++c) cfma(a, Ut[i + int64_t(c) * m], x[c]);
    out[col * ldout + e] = a;
}

__global__ void k_compress(const float2* __restrict__ U, int64_t nodes, int m, int r, const float2* __restrict__ in,
                           int64_t ldin, float2* __restrict__ out, int64_t ldout) {
    int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= nodes * r) return;
    int col = blockIdx.y;
    int64_t t = e / r;
    int c = int(e % r);
    const float2* Uc = U + t * m * r + int64_t(c) * m;
    const float2* x = in + col * ldin + t * m;
    float2 a = make_float2(0.f, 0.f);
    for (int i = 0; i < m; ++i) cfmac(a, Uc[i], x[i]);
    out[col * ldout + e] = a;
}

// matvec coupling at level l: y[2t] = B_t^* x[2t+1], y[2t+1] = B_t x[2t]
__global__ void k_couple(const float2* __restrict__ B, int64_t nodes, int r, const float2* __restrict__ x, int64_t ldx,
                         float2* __restrict__ y, int64_t ldy) {
    int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= nodes * 2 * r) return;
    int col = blockIdx.y;
    int64_t t = e / (2 * r);
    int w = int(e % (2 * r)), ch = w / r, i = w % r;
    const float2* Bt = B + t * r * r;
    const float2* xs = x + col * ldx + (2 * t + (1 - ch)) * r;
    float2 a = make_float2(0.f, 0.f);
    if (ch == 0)
        for (int j = 0; j < r; ++j) cfmac(a, Bt[j + int64_t(i) * r], xs[j]);   // (B^*)[i][j] = conj(B[j][i])
    else
        for (int j = 0; j < r; ++j) cfma(a, Bt[i + int64_t(j) * r], xs[j]);
    y[col * ldy + (2 * t + ch) * r + i] = a;
}

// leaf output: Y_t = D_t X_t + (U y)_t   (the U y part is already in Y)
__global__ void k_leaf_dx(const float2* __restrict__ D, int64_t nodes, int m, const float2* __restrict__ X, int64_t ldx,
                          float2* __restrict__ Y, int64_t ldy) {
    int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= nodes * m) return;
    int col = blockIdx.y;
    int64_t t = e / m;
    int i = int(e % m);
    const float2* Dt = D + t * m * m;
    const float2* x = X + col * ldx + t * m;
    float2 a = Y[col * ldy + e];
    for (int j = 0; j < m; ++j) cfma(a, Dt[i + int64_t(j) * m], x[j]);
    Y[col * ldy + e] = a;
}

}  // namespace

void launch_expand(const float2* U, int nodes, int m, int r, const float2* in, int64_t ldin, float2* out,
                   int64_t ldout, int k, bool accumulate, cudaStream_t st) {
    if (int64_t(nodes) * m == 0 || k == 0) return;
    if (r == 0) {
        if (!accumulate)
            for (int c = 0; c < k; ++c) cudaMemsetAsync(out + c * ldout, 0, size_t(nodes) * m * 8, st);
        return;
    }
    dim3 g(cdiv(int64_t(nodes) * m, TB), k);
    k_expand<<<g, TB, 0, st>>>(U, nodes, m, r, in, ldin, out, ldout, accumulate);
}

void launch_compress(const float2* U, int nodes, int m, int r, const float2* in, int64_t ldin, float2* out,
                     int64_t ldout, int k, cudaStream_t st) {
    if (int64_t(nodes) * r == 0 || k == 0) return;
    dim3 g(cdiv(int64_t(nodes) * r, TB), k);
    k_compress<<<g, TB, 0, st>>>(U, nodes, m, r, in, ldin, out, ldout);
}

namespace {

// H X for the sampler, X and Z: N x s, ld = N.  T is scratch (N x s).
fio_status sample(const fio_sampler* sm, int64_t N, const float2* X, float2* Z, float2* T, int s, cudaStream_t st) {
    if (sm->kind == FIO_SAMPLER_NORMAL) {
        // 2D: the HSS is built over the frequency index in quadtree (Morton) order
        fio_bf* bf = const_cast<fio_bf*>(sm->bf);
        FIO_TRY(bf_apply_ord(bf, X, T, N, s, 0, true, st));
        FIO_TRY(bf_apply_ord(bf, T, Z, N, s, 1, true, st));
        return FIO_OK;
    }
    dim3 g(cdiv(N, 16), cdiv(s, 16)), b(16, 16);
    k_dense_gemm<<<g, b, 0, st>>>(reinterpret_cast<const float2*>(sm->dense), sm->ld, X, N, Z, N, N, s);
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}

// Y^[l] = (U^[l+1]* .. U^[Lh]*) H (U^[Lh] .. U^[l+1]) Omega (Section 3.2).
// Omega has rows(l) rows; Y receives rows(l) rows; both column-major, s columns.
fio_status sample_level(fio_hss* h, const fio_sampler* sm, int l, const float2* Om, int s, float2* Y, DevBuf& xa,
                        DevBuf& xb, DevBuf& xc, cudaStream_t st) {
    const int64_t N = h->N;
    if (l == h->Lh) {   // leaf level: Omega already has N rows
        FIO_TRY(xc.ensure(size_t(N) * s * 8));
        return sample(sm, N, Om, Y, xc.as<float2>(), s, st);
    }
    FIO_TRY(xa.ensure(size_t(N) * s * 8));
    FIO_TRY(xb.ensure(size_t(N) * s * 8));
    FIO_TRY(xc.ensure(size_t(N) * s * 8));
    float2* buf[2] = {xa.as<float2>(), xb.as<float2>()};
    // expand through U^[l+1], ..., U^[Lh]
    const float2* cur = Om;
    int64_t ldcur = h->rows(l);
    int wi = 0;
    for (int j = l + 1; j <= h->Lh; ++j) {
        launch_expand(h->U[j].as<float2>(), 1 << j, h->m(j), h->ranks[j], cur, ldcur, buf[wi], h->rows(j), s, false, st);
        cur = buf[wi];
        ldcur = h->rows(j);
        wi ^= 1;
    }
    // cur = buf[wi ^ 1] holds X (N rows); buf[wi] is free
    float2* Z = buf[wi];
    FIO_TRY(sample(sm, N, cur, Z, xc.as<float2>(), s, st));
    // compress through U^[Lh]*, ..., U^[l+1]*
    float2* src = Z;
    float2* spare = buf[wi ^ 1];
    int64_t ldsrc = N;
    for (int j = h->Lh; j > l; --j) {
        float2* dst = (j == l + 1) ? Y : spare;
        launch_compress(h->U[j].as<float2>(), 1 << j, h->m(j), h->ranks[j], src, ldsrc, dst, h->rrows(j), s, st);
        spare = src;
        src = dst;
        ldsrc = h->rrows(j);
    }
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}

// Opt a kernel into `bytes` of dynamic shared memory (above the 48 KB default).
constexpr size_t kMaxDynSmem = 227 * 1024;
template <class Kern>
fio_status dyn_smem(Kern kernel, size_t bytes, const char* what) {
    if (bytes > kMaxDynSmem)
        return fail(FIO_EINVAL, std::string(what) + ": node needs " + std::to_string(bytes) +
                                    " bytes of shared memory (227 KB per CTA); sample count or rank too large");
    if (bytes > 48 * 1024) FIO_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes)));
    return FIO_OK;
}

template <class C>
fio_status level_nodes(fio_hss* h, int l, int m, int s, int rhat, const float2* Om, const float2* Y, double tol,
                       DevBuf& ws, DevBuf& thr, DevBuf& khat, DevBuf& sat, DevBuf& taus, std::vector<int>& hk,
                       std::vector<int>& hs, cudaStream_t st) {
    const int nn = 1 << l;
    FIO_TRY(ws.ensure(size_t(nn) * 2 * m * s * sizeof(C)));
    FIO_TRY(thr.ensure(size_t(nn) * 8));
    FIO_TRY(khat.ensure(size_t(nn) * 4));
    FIO_TRY(sat.ensure(size_t(nn) * 4));
    FIO_TRY(taus.ensure(size_t(nn) * std::max(1, rhat) * sizeof(C)));
    FIO_TRY(dyn_smem(k_node_lq<C>, size_t(s) * sizeof(C), "hss_build_from_samples"));
    k_node_lq<C><<<nn, TB, size_t(s) * sizeof(C), st>>>(Om, Y, h->rows(l), m, s, ws.as<C>(), thr.as<double>(), tol);
    size_t shq = (size_t((s - m + 1) & ~1)) * sizeof(typename RealOf<C>::T) + size_t(m) * sizeof(C);
    FIO_TRY(dyn_smem(k_node_qrcp<C>, shq, "hss_build_from_samples"));
    k_node_qrcp<C><<<nn, TB, shq, st>>>(ws.as<C>(), m, s, rhat, thr.as<double>(), khat.as<int>(), sat.as<int>(),
                                       taus.as<C>());
    FIO_CUDA(cudaGetLastError());
    hk.resize(nn);
    hs.resize(nn);
    FIO_CUDA(cudaMemcpyAsync(hk.data(), khat.p, nn * 4, cudaMemcpyDeviceToHost, st));
    FIO_CUDA(cudaMemcpyAsync(hs.data(), sat.p, nn * 4, cudaMemcpyDeviceToHost, st));
    FIO_CUDA(cudaStreamSynchronize(st));
    return FIO_OK;
}

template <class C>
fio_status level_finish(fio_hss* h, int l, int m, int s, int rhat, int rl, DevBuf& ws, DevBuf& taus, DevBuf& scratch,
                        DevBuf& Dchk, cudaStream_t st) {
    const int nn = 1 << l;
    FIO_TRY(h->U[l].ensure(std::max<size_t>(8, size_t(nn) * m * rl * 8)));
    FIO_TRY(Dchk.ensure(size_t(nn) * m * m * 8));
    FIO_TRY(scratch.ensure(std::max<size_t>(16, size_t(nn) * 2 * m * std::max(rl, 1) * sizeof(C))));
    if (rl > 0)
        k_node_formU<C><<<nn, TB, 0, st>>>(ws.as<C>(), m, s, rhat, rl, taus.as<C>(), h->U[l].as<float2>(),
                                           scratch.as<C>());
    k_node_dcheck<C><<<nn, TB, 0, st>>>(ws.as<C>(), m, s, h->U[l].as<float2>(), rl, Dchk.as<float2>(), scratch.as<C>());
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}

// FP32 node arithmetic on the wide levels, FP64 where a level has few nodes.
constexpr int kFp64Nodes = 16;

}  // namespace
}  // namespace fio

using namespace fio;

static fio_status hss_alloc_generators(fio_hss* h) {
    h->U.resize(h->Lh + 1);
    h->B.resize(h->Lh);
    h->W.resize(h->Lh + 1);
    return FIO_OK;
}

extern "C" fio_status hss_build_from_samples(const fio_sampler* sm, int64_t N, int leaf, int p, double tol, uint64_t seed,
                                             void* stream, fio_hss** out) {
    if (!sm || !out) return fail(FIO_EINVAL, "hss_build_from_samples: null pointer");
    *out = nullptr;
    if (leaf < 1 || leaf > 256 || N % leaf) return fail(FIO_EINVAL, "hss_build_from_samples: need 1 <= leaf <= 256, leaf | N");
    int Lh = ilog2_exact(N / leaf);
    if (Lh < 1) return fail(FIO_EINVAL, "hss_build_from_samples: N / leaf must be a power of two >= 2");
    if (p < 1 || p > 64) return fail(FIO_EINVAL, "hss_build_from_samples: oversample must be in [1, 64]");
    if (!(tol > 0)) return fail(FIO_EINVAL, "hss_build_from_samples: tol must be > 0");
    if (sm->kind == FIO_SAMPLER_NORMAL) {
        if (!sm->bf || sm->bf->N() != N) return fail(FIO_EINVAL, "hss_build_from_samples: bf missing or N mismatch");
    } else if (sm->kind == FIO_SAMPLER_DENSE) {
        if (!sm->dense || sm->ld < N) return fail(FIO_EINVAL, "hss_build_from_samples: dense sampler needs ld >= N");
    } else {
        return fail(FIO_EINVAL, "hss_build_from_samples: unknown sampler kind");
    }
    cudaStream_t st = as_stream(stream);
    fio_hss* h = new fio_hss();
    h->N = N;
    h->leaf = leaf;
    h->Lh = Lh;
    h->ranks.assign(Lh + 1, 0);
    hss_alloc_generators(h);
    auto bail = [&](fio_status s) { hss_free(h); return s; };
    std::vector<DevBuf> Dchk(Lh + 1);
    DevBuf Om, Yb, xa, xb, xc, ws, thr, khat, sat, taus, scratch, Dcur, Dnext;
    BigScratch* big = big_scratch_new();
    auto release = [&]() {
        for (auto& d : Dchk) d.release();
        for (DevBuf* b : {&Om, &Yb, &xa, &xb, &xc, &ws, &thr, &khat, &sat, &taus, &scratch, &Dcur, &Dnext}) b->release();
        big_scratch_free(big);
        big = nullptr;
    };
    const uint32_t k0 = uint32_t(seed & 0xffffffffu), k1 = uint32_t(seed >> 32);
    std::vector<int> hk, hsat;
    fio_status s;
    for (int l = Lh; l >= 1; --l) {
        const int m = h->m(l), nn = 1 << l;
        if (m == 0) {
            h->ranks[l] = 0;
            continue;
        }
        int rhat = std::max(1, std::min(m, (m + 1) / 2));
        int attempt = 0;
        int s_cols = 0;
        const bool f64 = nn <= kFp64Nodes;
        while (true) {
            s_cols = rhat + m + p;
            const int64_t rows = h->rows(l);
            if ((s = Om.ensure(size_t(rows) * s_cols * 8)) != FIO_OK) { release(); return bail(s); }
            if ((s = Yb.ensure(size_t(rows) * s_cols * 8)) != FIO_OK) { release(); return bail(s); }
            k_gauss<<<cdiv(rows * s_cols, TB), TB, 0, st>>>(Om.as<float2>(), rows, s_cols, l, attempt, k0, k1);
            if ((s = sample_level(h, sm, l, Om.as<float2>(), s_cols, Yb.as<float2>(), xa, xb, xc, st)) != FIO_OK) {
                release();
                return bail(s);
            }
            h->samples += s_cols;
            if (large_level(nn, m))
                s = big_level_nodes(*big, nn, m, s_cols, rhat, Om.as<float2>(), Yb.as<float2>(), rows, tol, hk, hsat, st);
            else
                s = f64 ? level_nodes<double2>(h, l, m, s_cols, rhat, Om.as<float2>(), Yb.as<float2>(), tol, ws, thr, khat,
                                               sat, taus, hk, hsat, st)
                        : level_nodes<float2>(h, l, m, s_cols, rhat, Om.as<float2>(), Yb.as<float2>(), tol, ws, thr, khat,
                                              sat, taus, hk, hsat, st);
            if (s != FIO_OK) { release(); return bail(s); }
            bool saturated = false;
            int rl = 0;
            for (int t = 0; t < nn; ++t) {
                rl = std::max(rl, hk[t]);
                saturated |= hsat[t] != 0;
            }
            if (saturated && rhat < m) {
                rhat = std::min(m, 2 * rhat);
                ++attempt;
                continue;
            }
            h->ranks[l] = rl;
            break;
        }
        if (large_level(nn, m)) {
            const int rl = h->ranks[l];
            if ((s = h->U[l].ensure(std::max<size_t>(8, size_t(nn) * m * rl * 8))) != FIO_OK) { release(); return bail(s); }
            if ((s = Dchk[l].ensure(size_t(nn) * m * m * 8)) != FIO_OK) { release(); return bail(s); }
            s = big_level_finish(*big, nn, m, rl, h->U[l].as<float2>(), Dchk[l].as<float2>(), st);
        } else {
            s = f64 ? level_finish<double2>(h, l, m, s_cols, rhat, h->ranks[l], ws, taus, scratch, Dchk[l], st)
                    : level_finish<float2>(h, l, m, s_cols, rhat, h->ranks[l], ws, taus, scratch, Dchk[l], st);
        }
        if (s != FIO_OK) { release(); return bail(s); }
    }
    // root: H^[0] = Y^[0] Omega^[0]+
    const int m0 = 2 * h->ranks[1];
    if ((s = Dcur.ensure(std::max<size_t>(16, size_t(m0) * m0 * 16))) != FIO_OK) { release(); return bail(s); }
    if (m0 > 0) {
        const int s0 = m0 + p;
        if ((s = Om.ensure(size_t(m0) * s0 * 8)) != FIO_OK) { release(); return bail(s); }
        if ((s = Yb.ensure(size_t(m0) * s0 * 8)) != FIO_OK) { release(); return bail(s); }
        k_gauss<<<cdiv(int64_t(m0) * s0, TB), TB, 0, st>>>(Om.as<float2>(), m0, s0, 0, 0, k0, k1);
        if ((s = sample_level(h, sm, 0, Om.as<float2>(), s0, Yb.as<float2>(), xa, xb, xc, st)) != FIO_OK) {
            release();
            return bail(s);
        }
        h->samples += s0;
        if (large_level(1, m0)) {
            if ((s = big_root(*big, m0, s0, Om.as<float2>(), Yb.as<float2>(), Dcur.as<double2>(), st)) != FIO_OK) {
                release();
                return bail(s);
            }
        } else {
            if ((s = ws.ensure(size_t(2) * m0 * s0 * 16)) != FIO_OK) { release(); return bail(s); }
            if ((s = thr.ensure(16)) != FIO_OK) { release(); return bail(s); }
            if ((s = dyn_smem(k_node_lq<double2>, size_t(s0) * 16, "hss_build_from_samples (root)")) != FIO_OK) {
                release();
                return bail(s);
            }
            k_node_lq<double2><<<1, TB, size_t(s0) * 16, st>>>(Om.as<float2>(), Yb.as<float2>(), m0, m0, s0,
                                                             ws.as<double2>(), thr.as<double>(), tol);
            k_root_h0<double2><<<1, TB, 0, st>>>(ws.as<double2>(), m0, s0, Dcur.as<double2>());
        }
    }
    // postprocessing, top-down (Section 3.3)
    for (int l = 0; l < Lh; ++l) {
        const int rc = h->ranks[l + 1], mc = h->m(l + 1), nn = 1 << l;
        if ((s = h->B[l].ensure(std::max<size_t>(8, size_t(nn) * rc * rc * 8))) != FIO_OK) { release(); return bail(s); }
        if ((s = Dnext.ensure(size_t(2 * nn) * mc * mc * 16)) != FIO_OK) { release(); return bail(s); }
        if ((s = scratch.ensure(std::max<size_t>(16, size_t(nn) * mc * std::max(rc, 1) * 16))) != FIO_OK) {
            release();
            return bail(s);
        }
        if (mc > 0 && large_level(1, mc)) {
            if ((s = big_post(*big, nn, rc, mc, Dcur.as<double2>(), h->U[l + 1].as<float2>(), Dchk[l + 1].as<float2>(),
                              h->B[l].as<float2>(), Dnext.as<double2>(), st)) != FIO_OK) {
                release();
                return bail(s);
            }
        } else if (mc > 0) {
            k_post<<<nn, TB, 0, st>>>(Dcur.as<double2>(), rc, mc, h->U[l + 1].as<float2>(), Dchk[l + 1].as<float2>(),
                                      h->B[l].as<float2>(), Dnext.as<double2>(), scratch.as<double2>());
        }
        std::swap(Dcur, Dnext);
    }
    if ((s = h->D.ensure(size_t(1 << Lh) * leaf * leaf * 8)) != FIO_OK) { release(); return bail(s); }
    {
        int64_t tot = (int64_t(1) << Lh) * leaf * leaf;
        k_leafD<<<cdiv(tot, TB), TB, 0, st>>>(Dcur.as<double2>(), leaf, int64_t(1) << Lh, h->D.as<float2>());
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    release();
    if (e != cudaSuccess) return bail(cuda_status(e, "hss_build_from_samples"));
    *out = h;
    return FIO_OK;
}

extern "C" fio_status hss_from_generators(int64_t N, int leaf, const int* ranks, const void* U, const void* B,
                                          const void* D, void* stream, fio_hss** out) {
    if (!out || !ranks || !D) return fail(FIO_EINVAL, "hss_from_generators: null pointer");
    *out = nullptr;
    if (leaf < 1 || leaf > 256 || N % leaf) return fail(FIO_EINVAL, "hss_from_generators: bad leaf");
    int Lh = ilog2_exact(N / leaf);
    if (Lh < 1) return fail(FIO_EINVAL, "hss_from_generators: N / leaf must be a power of two >= 2");
    fio_hss* h = new fio_hss();
    h->N = N;
    h->leaf = leaf;
    h->Lh = Lh;
    h->ranks.assign(ranks, ranks + Lh + 1);
    h->ranks[0] = 0;
    for (int l = 1; l <= Lh; ++l)
        if (h->ranks[l] < 0 || h->ranks[l] > h->m(l)) {
            hss_free(h);
            return fail(FIO_EINVAL, "hss_from_generators: rank exceeds block size");
        }
    hss_alloc_generators(h);
    cudaStream_t st = as_stream(stream);
    const char* u = static_cast<const char*>(U);
    const char* b = static_cast<const char*>(B);
    fio_status s;
    for (int l = 1; l <= Lh; ++l) {
        size_t bytes = size_t(1 << l) * h->m(l) * h->ranks[l] * 8;
        if ((s = h->U[l].ensure(std::max<size_t>(8, bytes))) != FIO_OK) { hss_free(h); return s; }
        if (bytes) {
            if (!U) { hss_free(h); return fail(FIO_EINVAL, "hss_from_generators: U missing"); }
            cudaMemcpyAsync(h->U[l].p, u, bytes, cudaMemcpyHostToDevice, st);
            u += bytes;
        }
    }
    for (int l = 0; l < Lh; ++l) {
        size_t bytes = size_t(1 << l) * h->ranks[l + 1] * h->ranks[l + 1] * 8;
        if ((s = h->B[l].ensure(std::max<size_t>(8, bytes))) != FIO_OK) { hss_free(h); return s; }
        if (bytes) {
            if (!B) { hss_free(h); return fail(FIO_EINVAL, "hss_from_generators: B missing"); }
            cudaMemcpyAsync(h->B[l].p, b, bytes, cudaMemcpyHostToDevice, st);
            b += bytes;
        }
    }
    size_t dbytes = size_t(1 << Lh) * leaf * leaf * 8;
    if ((s = h->D.ensure(dbytes)) != FIO_OK) { hss_free(h); return s; }
    cudaMemcpyAsync(h->D.p, D, dbytes, cudaMemcpyHostToDevice, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { hss_free(h); return cuda_status(e, "hss_from_generators"); }
    *out = h;
    return FIO_OK;
}

extern "C" fio_status hss_info(const fio_hss* h, int64_t* out, int max_out, int64_t* samples) {
    if (!h || !out) return fail(FIO_EINVAL, "hss_info: null pointer");
    if (max_out < 3 + h->Lh + 1) return fail(FIO_EINVAL, "hss_info: output too small");
    out[0] = h->N;
    out[1] = h->leaf;
    out[2] = h->Lh;
    for (int l = 0; l <= h->Lh; ++l) out[3 + l] = h->ranks[l];
    if (samples) *samples = h->samples;
    return FIO_OK;
}

extern "C" fio_status hss_matvec(const fio_hss* hc, const void* Xv, void* Yv, int64_t ld, int k, void* stream) {
    if (!hc) return fail(FIO_EINVAL, "hss_matvec: null handle");
    if (k < 0 || ld < hc->N) return fail(FIO_EINVAL, "hss_matvec: need k >= 0 and ld >= N");
    if (k == 0) return FIO_OK;
    fio_hss* h = const_cast<fio_hss*>(hc);
    cudaStream_t st = as_stream(stream);
    const float2* X = static_cast<const float2*>(Xv);
    float2* Y = static_cast<float2*>(Yv);
    const int Lh = h->Lh;
    // per level l = 1..Lh: x_l (rrows(l)), y_l (rrows(l))
    std::vector<int64_t> off(Lh + 2, 0);
    for (int l = 1; l <= Lh; ++l) off[l + 1] = off[l] + h->rrows(l);
    const int64_t tot = off[Lh + 1];
    FIO_TRY(h->mv_ws.ensure(std::max<size_t>(16, size_t(2) * tot * k * 8)));
    float2* xs = h->mv_ws.as<float2>();
    float2* ys = xs + tot * k;
    auto xl = [&](int l) { return xs + off[l] * k; };
    auto yl = [&](int l) { return ys + off[l] * k; };
    // up
    launch_compress(h->U[Lh].as<float2>(), 1 << Lh, h->leaf, h->ranks[Lh], X, ld, xl(Lh), h->rrows(Lh), k, st);
    for (int l = Lh - 1; l >= 1; --l)
        launch_compress(h->U[l].as<float2>(), 1 << l, h->m(l), h->ranks[l], xl(l + 1), h->rrows(l + 1), xl(l),
                        h->rrows(l), k, st);
    // coupling
    for (int l = 0; l < Lh; ++l) {
        int r = h->ranks[l + 1];
        if (r == 0) continue;
        dim3 g(cdiv(int64_t(1 << l) * 2 * r, TB), k);
        k_couple<<<g, TB, 0, st>>>(h->B[l].as<float2>(), 1 << l, r, xl(l + 1), h->rrows(l + 1), yl(l + 1),
                                   h->rrows(l + 1));
    }
    // down
    for (int l = 1; l < Lh; ++l)
        if (h->ranks[l] > 0)
            launch_expand(h->U[l].as<float2>(), 1 << l, h->m(l), h->ranks[l], yl(l), h->rrows(l), yl(l + 1),
                          h->rrows(l + 1), k, true, st);
    // leaves
    if (h->ranks[Lh] > 0)
        launch_expand(h->U[Lh].as<float2>(), 1 << Lh, h->leaf, h->ranks[Lh], yl(Lh), h->rrows(Lh), Y, ld, k, false, st);
    else
        for (int c = 0; c < k; ++c) cudaMemsetAsync(Y + c * ld, 0, size_t(h->N) * 8, st);
    dim3 g(cdiv(h->N, TB), k);
    k_leaf_dx<<<g, TB, 0, st>>>(h->D.as<float2>(), 1 << Lh, h->leaf, X, ld, Y, ld);
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}

extern "C" void hss_free(fio_hss* h) {
    if (!h) return;
    for (auto& b : h->U) b.release();
    for (auto& b : h->B) b.release();
    for (auto& b : h->W) b.release();
    for (auto& b : h->Wmx) b.release();
    h->D.release();
    h->Rinv.release();
    h->solve_ws.release();
    h->solve_part.release();
    h->mv_ws.release();
    h->fio_ws.release();
    delete h;
}
