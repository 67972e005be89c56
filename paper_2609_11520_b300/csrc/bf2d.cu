// Butterfly factorization of a 2D FIO (Section 2.2 with d = 2, Section 5.2):
// quadtree boxes, tensor Chebyshev grids of r1 x r1 nodes (r1 = 3 .. 7; the
// kernels are instantiated per r1), the same factor sequence as Eq. 2.1.
//
// Geometry (per dimension as in 1D).  n points per dimension, N = n^2,
// L = log2 n, h = floor(L/2), sU = max(L-3, h), sV = min(3, h).  A box at
// level s is (a1, a2) with id a = a1 2^s + a2; its children are
// (2 a1 + c1, 2 a2 + c2), child number c = 2 c1 + c2.  Node t = t1 r1 + t2 of
// a box is the tensor product of the 1D first-kind Chebyshev points.  A pair
// at space level s is (tau at space level s, sigma at frequency level L-s),
// index tau 4^(L-s) + sigma.  Vectors are lexicographic (x_i = (i1, i2)/n
// with i = i1 n + i2; xi_j = (j1 - n/2, j2 - n/2) with j = j1 n + j2); the
// frequency side can instead be taken in quadtree (Morton) order, the order
// in which the HSS of K~^* K~ is built.
//
// Phase-folded factored tables, as in 1D (the state between stages carries
// e^{+2 pi i Phi(y_tau, gamma_sigma_j)} on the right side and
// e^{-2 pi i Phi(z_tau_i, eta_sigma)} on the left side):
//   VP[a][j]          e^{2 pi i Phi(y_a, xi_j)}                      a at level sV
//   F_s[g][o][c][t]   e^{2 pi i (Phi(y_tau_o, gamma_beta_c,t) - Phi(y_tau, gamma_beta_c,t))}   C level s
//   M[p][i][j]        e^{2 pi i (Phi(z_i, gamma_j) - Phi(z_i, eta) - Phi(y, gamma_j))}
//   E_s[g][o][c][i]   e^{2 pi i (Phi(z_tau_o,i, eta_beta_c) - Phi(z_tau_o,i, eta_sigma'))}      B level s
//   UP[x][b]          e^{2 pi i Phi(x, eta_b)}                       b at frequency level L-sU
// with the group g = (tau at space level s, sigma' at frequency level L-s-1):
// the inputs are the pairs (tau, beta_c = child c of sigma'), the outputs the
// pairs (tau_o = child o of tau, sigma').  Real tables: Pc[c][j][t] =
// l_j(child c node t) (the parent's Lagrange basis at a child's nodes; the
// same matrix serves the frequency boxes of C and the space boxes of B),
// its transpose, and the leaf bases QV[t][q], QU[x][i].
#include <cmath>
#include <cstring>

#include "bf.cuh"

namespace fio {
namespace {

constexpr int TB = 256;
constexpr int kMinR1 = 3, kMaxR1 = 7;

// Per-grid constants: R = r1^2 coefficients per pair, RP = R padded to whole float4 rows, PHG
// transfer groups whose phase rows a CTA stages in shared memory, MP middle-level pairs per CTA
// (the static shared memory of the transfer kernel and the M block of the middle kernel shrink
// with R so that r1 = 7 still fits).
template <int R1>
struct G2 {
    static constexpr int R = R1 * R1;
    static constexpr int RP = (R + 3) / 4 * 4;
    static constexpr int PHG = R <= 25 ? 8 : (R <= 36 ? 2 : 1);
    static constexpr int MP = R <= 36 ? 16 : 8;
    // r1 >= 6: the middle level splits each pair's R outputs into r1 chunks of r1 (one thread per
    // chunk, MQ = MQP pairs x 16 columns x r1 threads per CTA), which keeps the registers low
    static constexpr bool CHUNK_M = R1 >= 6;
    static constexpr int MQP = 8;
    static constexpr int MQ = MQP * 16 * R1;
};

// first-kind Chebyshev points on [-1, 1] of the handle's r1
struct Cheb2 {
    double t[kMaxR1];
};

// Nonlinear part Phi(x, xi) - x . xi of the 2D families (Sections 5.2 and 5.3; 0 for the DFT).
__device__ __forceinline__ double phi2_nl(int kind, double s, double x1, double x2, double k1, double k2) {
    if (kind == FIO_PHASE_2D_ELLIPTIC) {
        const double c1 = (2.0 + sinpi(2.0 * x1) * sinpi(2.0 * x2)) * 0.0625;
        const double c2 = (2.0 + cospi(2.0 * x1) * cospi(2.0 * x2)) * 0.0625;
        return sqrt(c1 * c1 * k1 * k1 + c2 * c2 * k2 * k2);
    }
    if (kind == FIO_PHASE_2D_ISO) return (3.0 + s * sinpi(2.0 * x1) * sinpi(2.0 * x2)) * 0.125 * sqrt(k1 * k1 + k2 * k2);
    return 0.0;
}
// The handle's 2D phase (kind and modulation depth s), by value in kernel parameters.
struct Ph2 {
    int kind;
    double s;
};
// Phi(x, xi) of the 2D families.
__device__ __forceinline__ double phi2(const Ph2& p, double x1, double x2, double k1, double k2) {
    return x1 * k1 + x2 * k2 + phi2_nl(p.kind, p.s, x1, x2, k1, k2);
}

// Hankel amplitude of Section 5.3: a = H0^(1)(2 pi phi) e^{-2 pi i phi}, H0^(1) = J0 + i Y0.
__device__ __forceinline__ float2 hankel_amp(double ph) {
    const double z = 2.0 * M_PI * ph;
    const double jr = j0(z), yi = y0(z);
    double sn, cs;
    sincospi(2.0 * ph, &sn, &cs);
    return make_float2(float(jr * cs + yi * sn), float(yi * cs - jr * sn));
}

// e^{2 pi i ph}: reduce modulo 1 in FP64, then sin/cos of the remainder.
__device__ __forceinline__ float2 expi(double ph) {
    const double fr = ph - rint(ph);
    float sn, cs;
    sincospif(2.0f * float(fr), &sn, &cs);
    return make_float2(cs, sn);
}

__host__ __device__ __forceinline__ int64_t child_id(int s, int64_t a, int c) {
    const int64_t a1 = a >> s, a2 = a & ((int64_t(1) << s) - 1);
    return ((2 * a1 + (c >> 1)) << (s + 1)) + 2 * a2 + (c & 1);
}
// coordinate d (0, 1) of the centre of space box a at level s
__device__ __forceinline__ double sctr(int s, int64_t a, int d) {
    const int64_t ad = d == 0 ? (a >> s) : (a & ((int64_t(1) << s) - 1));
    return ldexp(double(ad) + 0.5, -s);
}
__device__ __forceinline__ double snode(const Cheb2& ch, int s, int64_t a, int d, int k) {
    return sctr(s, a, d) + ldexp(0.5, -s) * ch.t[k];
}
__device__ __forceinline__ double fctr(int n, int l, int64_t b, int d) {
    const int64_t bd = d == 0 ? (b >> l) : (b & ((int64_t(1) << l) - 1));
    return -0.5 * n + (double(bd) + 0.5) * ldexp(double(n), -l);
}
__device__ __forceinline__ double fnode(const Cheb2& ch, int n, int l, int64_t b, int d, int k) {
    return fctr(n, l, b, d) + ldexp(double(n), -l - 1) * ch.t[k];
}

// Morton position of the frequency (j1, j2): bits of j2 at even, of j1 at odd positions.
__device__ __forceinline__ int64_t morton(int j1, int j2, int L) {
    int64_t m = 0;
    for (int k = 0; k < L; ++k) m |= (int64_t((j2 >> k) & 1) << (2 * k)) | (int64_t((j1 >> k) & 1) << (2 * k + 1));
    return m;
}
__device__ __forceinline__ int64_t fidx(int j1, int j2, int n, int L, bool mort) {
    return mort ? morton(j1, j2, L) : int64_t(j1) * n + j2;
}

// ---------------------------------------------------------------- tables
__global__ void k2_tab_VP(float2* VP, Ph2 kind, int n, int sV) {
    const int64_t N = int64_t(n) * n;
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= (int64_t(1) << (2 * sV)) * N) return;
    const int64_t a = e / N, j = e % N;
    VP[e] = expi(phi2(kind, sctr(sV, a, 0), sctr(sV, a, 1), double(j / n) - 0.5 * n, double(j % n) - 0.5 * n));
}

// groups g = tau 4^(L-s-1) + sigma', entries [g][o][c][t]
template <int R1>
__global__ void k2_tab_F(float2* F, Ph2 kind, Cheb2 ch, int n, int L, int s) {
    constexpr int R = G2<R1>::R;
    const int64_t N = int64_t(n) * n;
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= N / 4 * 16 * R) return;
    const int t = int(e % R);
    const int64_t rest = e / R;
    const int c = int(rest & 3), o = int((rest >> 2) & 3);
    const int64_t g = rest >> 4;
    const int64_t nbq = int64_t(1) << (2 * (L - s - 1));
    const int64_t tau = g / nbq, sq = g % nbq;
    const int64_t to = child_id(s, tau, o), beta = child_id(L - s - 1, sq, c);
    const double g1 = fnode(ch, n, L - s, beta, 0, t / R1), g2 = fnode(ch, n, L - s, beta, 1, t % R1);
    F[e] = expi(phi2(kind, sctr(s + 1, to, 0), sctr(s + 1, to, 1), g1, g2) -
                phi2(kind, sctr(s, tau, 0), sctr(s, tau, 1), g1, g2));
}

template <int R1>
__global__ void k2_tab_M(float2* M, Ph2 kind, int amp_kind, Cheb2 ch, int n, int L, int h) {
    constexpr int R = G2<R1>::R;
    const int64_t N = int64_t(n) * n;
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= N * R * R) return;
    const int j = int(e % R), i = int((e / R) % R);
    const int64_t p = e / (R * R);
    const int64_t nb = int64_t(1) << (2 * (L - h));
    const int64_t tau = p / nb, sg = p % nb;
    const double z1 = snode(ch, h, tau, 0, i / R1), z2 = snode(ch, h, tau, 1, i % R1);
    const double y1 = sctr(h, tau, 0), y2 = sctr(h, tau, 1);
    const double g1 = fnode(ch, n, L - h, sg, 0, j / R1), g2 = fnode(ch, n, L - h, sg, 1, j % R1);
    const double e1 = fctr(n, L - h, sg, 0), e2 = fctr(n, L - h, sg, 1);
    const float2 m = expi(phi2(kind, z1, z2, g1, g2) - phi2(kind, z1, z2, e1, e2) - phi2(kind, y1, y2, g1, g2));
    M[e] = amp_kind == FIO_AMP_HANKEL ? cmul(hankel_amp(phi2_nl(kind.kind, kind.s, z1, z2, g1, g2)), m) : m;
}

template <int R1>
__global__ void k2_tab_E(float2* E, Ph2 kind, Cheb2 ch, int n, int L, int s) {
    constexpr int R = G2<R1>::R;
    const int64_t N = int64_t(n) * n;
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= N / 4 * 16 * R) return;
    const int i = int(e % R);
    const int64_t rest = e / R;
    const int c = int(rest & 3), o = int((rest >> 2) & 3);
    const int64_t g = rest >> 4;
    const int64_t nbq = int64_t(1) << (2 * (L - s - 1));
    const int64_t al = g / nbq, sq = g % nbq;
    const int64_t to = child_id(s, al, o), beta = child_id(L - s - 1, sq, c);
    const double z1 = snode(ch, s + 1, to, 0, i / R1), z2 = snode(ch, s + 1, to, 1, i % R1);
    E[e] = expi(phi2(kind, z1, z2, fctr(n, L - s, beta, 0), fctr(n, L - s, beta, 1)) -
                phi2(kind, z1, z2, fctr(n, L - s - 1, sq, 0), fctr(n, L - s - 1, sq, 1)));
}

__global__ void k2_tab_UP(float2* UP, Ph2 kind, int n, int L, int sU) {
    const int64_t N = int64_t(n) * n;
    const int64_t nsg = int64_t(1) << (2 * (L - sU));
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= N * nsg) return;
    const int64_t x = e / nsg, sg = e % nsg;
    UP[e] = expi(phi2(kind, double(x / n) / n, double(x % n) / n, fctr(n, L - sU, sg, 0), fctr(n, L - sU, sg, 1)));
}

// ---------------------------------------------------------------- apply
// Column block: X, Y (N x kc, ld); coefficient states S[col][pair][t] with
// SN = N * R complex per column.

// R-term real-by-complex dot product of a padded smem row with a register vector.
template <int R>
__device__ __forceinline__ float2 rowdot(const float* __restrict__ row, const float2 (&x)[R]) {
    const float4* r4 = reinterpret_cast<const float4*>(row);
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < R / 4; ++q) {
        const float4 a = r4[q];
        acc.x = fmaf(a.x, x[4 * q].x, acc.x); acc.y = fmaf(a.x, x[4 * q].y, acc.y);
        acc.x = fmaf(a.y, x[4 * q + 1].x, acc.x); acc.y = fmaf(a.y, x[4 * q + 1].y, acc.y);
        acc.x = fmaf(a.z, x[4 * q + 2].x, acc.x); acc.y = fmaf(a.z, x[4 * q + 2].y, acc.y);
        acc.x = fmaf(a.w, x[4 * q + 3].x, acc.x); acc.y = fmaf(a.w, x[4 * q + 3].y, acc.y);
    }
#pragma unroll
    for (int t = R / 4 * 4; t < R; ++t) {
        acc.x = fmaf(row[t], x[t].x, acc.x);
        acc.y = fmaf(row[t], x[t].y, acc.y);
    }
    return acc;
}

// V (forward): c(a, b, t) = sum_q QV[t][q] VP[a][xi(b, q)] f(xi(b, q)).
// CTA: one frequency leaf b, 4 columns; thread (a, column).
template <int R1>
__global__ void __launch_bounds__(TB) k2_V_fwd(const float2* __restrict__ X, int64_t ld, float2* __restrict__ S,
                                               int64_t SN, const float2* __restrict__ VP, const float* __restrict__ QV,
                                               int n, int L, int sV, int kc, int mort) {
    constexpr int R = G2<R1>::R;
    __shared__ float2 vps[64][65];
    __shared__ float2 fs[4][64];
    __shared__ float qv[R][64];
    const int NA = 1 << (2 * sV), m = 1 << sV, lb = L - sV;
    const int64_t N = int64_t(n) * n, NB = int64_t(1) << (2 * lb);
    const int64_t b = blockIdx.x;
    const int col0 = blockIdx.y * 4;
    const int b1 = int(b >> lb), b2 = int(b & ((int64_t(1) << lb) - 1));
    for (int idx = threadIdx.x; idx < NA * NA; idx += TB) {
        const int a = idx / NA, q = idx % NA;
        vps[a][q] = VP[a * N + int64_t(b1 * m + q / m) * n + b2 * m + q % m];
    }
    for (int idx = threadIdx.x; idx < 4 * NA; idx += TB) {
        const int cl = idx / NA, q = idx % NA;
        if (col0 + cl < kc) fs[cl][q] = X[(col0 + cl) * ld + fidx(b1 * m + q / m, b2 * m + q % m, n, L, mort)];
    }
    for (int idx = threadIdx.x; idx < R * NA; idx += TB) qv[idx / NA][idx % NA] = QV[idx];
    __syncthreads();
    const int a = threadIdx.x & 63, cl = threadIdx.x >> 6;
    if (a >= NA || col0 + cl >= kc) return;
    float2 acc[R];
#pragma unroll
    for (int t = 0; t < R; ++t) acc[t] = make_float2(0.f, 0.f);
    for (int q = 0; q < NA; ++q) {
        const float2 v = cmul(vps[a][q], fs[cl][q]);
#pragma unroll
        for (int t = 0; t < R; ++t) {
            acc[t].x = fmaf(qv[t][q], v.x, acc[t].x);
            acc[t].y = fmaf(qv[t][q], v.y, acc[t].y);
        }
    }
    float2* out = S + (col0 + cl) * SN + (a * NB + b) * R;
#pragma unroll
    for (int t = 0; t < R; ++t) out[t] = acc[t];
}

// V^*: f(xi(b, q)) = sum_a conj(VP[a][xi]) sum_t QV[t][q] c(a, b, t).  Thread (q, column).
template <int R1>
__global__ void __launch_bounds__(TB) k2_V_adj(const float2* __restrict__ S, int64_t SN, float2* __restrict__ Y,
                                               int64_t ld, const float2* __restrict__ VP, const float* __restrict__ QV,
                                               int n, int L, int sV, int kc, int mort) {
    constexpr int R = G2<R1>::R;
    extern __shared__ float4 smem_v[];
    float2(*vps)[65] = reinterpret_cast<float2(*)[65]>(smem_v);                 // [64][65]
    float2* cs = reinterpret_cast<float2*>(smem_v) + 64 * 65;                     // [4][64][R]
    float* qv = reinterpret_cast<float*>(cs + 4 * 64 * R);                        // [R][64]
    const int NA = 1 << (2 * sV), m = 1 << sV, lb = L - sV;
    const int64_t N = int64_t(n) * n, NB = int64_t(1) << (2 * lb);
    const int64_t b = blockIdx.x;
    const int col0 = blockIdx.y * 4;
    const int b1 = int(b >> lb), b2 = int(b & ((int64_t(1) << lb) - 1));
    for (int idx = threadIdx.x; idx < NA * NA; idx += TB) {
        const int a = idx / NA, q = idx % NA;
        vps[a][q] = VP[a * N + int64_t(b1 * m + q / m) * n + b2 * m + q % m];
    }
    for (int idx = threadIdx.x; idx < 4 * NA * R; idx += TB) {
        const int cl = idx / (NA * R), rem = idx % (NA * R), a = rem / R, t = rem % R;
        if (col0 + cl < kc) cs[(cl * 64 + a) * R + t] = S[(col0 + cl) * SN + (a * NB + b) * R + t];
    }
    for (int idx = threadIdx.x; idx < R * NA; idx += TB) qv[(idx / NA) * 64 + idx % NA] = QV[idx];
    __syncthreads();
    const int q = threadIdx.x & 63, cl = threadIdx.x >> 6;
    if (q >= NA || col0 + cl >= kc) return;
    float qq[R];
#pragma unroll
    for (int t = 0; t < R; ++t) qq[t] = qv[t * 64 + q];
    float2 acc = make_float2(0.f, 0.f);
    for (int a = 0; a < NA; ++a) {
        const float2* c = cs + (cl * 64 + a) * R;
        float2 tmp = make_float2(0.f, 0.f);
#pragma unroll
        for (int t = 0; t < R; ++t) {
            tmp.x = fmaf(qq[t], c[t].x, tmp.x);
            tmp.y = fmaf(qq[t], c[t].y, tmp.y);
        }
        cfmac(acc, vps[a][q], tmp);
    }
    Y[(col0 + cl) * ld + fidx(b1 * m + q / m, b2 * m + q % m, n, L, mort)] = acc;
}

// One transfer level between pair levels s and s+1 (C: SM = true forward,
// false adjoint; B: SM = false forward, true adjoint).  Group g couples the
// level-s pairs low(c) = (tau, child c of sigma') and the level-(s+1) pairs
// high(o) = (child o of tau, sigma').  Forward reads low (w = c) and writes
// high (u = o); the adjoint reads high (w = o) and writes low (u = c).
//   SM: out[u][v] = sum_w sum_t A_w[v][t] (Ph[u,w,t] x[w][t])          A = Pc
//   MS: out[u][v] = sum_w Ph[u,w,v] sum_t A_u[v][t] x[w][t]            A = Pc^T
// Ph[u,w,.] = table[g][o][c][.] (conjugated for the adjoint).
// Thread (group, column, u); 64 (group, column) items per CTA.
template <int R1, bool SM, bool ADJ>
__global__ void __launch_bounds__(TB, R1 <= 5 ? 2 : 1) k2_trans(const float2* __restrict__ Sin, float2* __restrict__ Sout, int64_t SN,
                                                  const float2* __restrict__ Ph, const float* __restrict__ Am, int L,
                                                  int s, int kc) {
    constexpr int R = G2<R1>::R, RP = G2<R1>::RP, kPhGroups = G2<R1>::PHG;
    __shared__ __align__(16) float A[4 * R * RP];
    __shared__ float2 phs[kPhGroups * 16 * R];   // phase rows of the CTA's groups (when they fit)
    for (int i = threadIdx.x; i < 4 * R * RP; i += TB) A[i] = Am[i];
    const int64_t ngroups = int64_t(1) << (2 * L - 2);
    const int64_t item0 = int64_t(blockIdx.x) * (TB / 4);
    const int64_t g0 = item0 / kc;
    const int ng = int(std::min<int64_t>(ngroups - 1, (item0 + TB / 4 - 1) / kc) - g0 + 1);
    // MS reads one phase per output inside the product loop: stage them; SM reads its
    // phases ahead of the products, where the global loads already overlap
    const bool staged = !SM && ng <= kPhGroups;
    if (staged)
        for (int i = threadIdx.x; i < ng * 16 * R; i += TB) phs[i] = Ph[g0 * 16 * R + i];
    __syncthreads();
    const int u = threadIdx.x & 3;
    const int64_t item = item0 + (threadIdx.x >> 2);
    if (item >= ngroups * kc) return;
    const int col = int(item % kc);
    const int64_t g = item / kc;
    const int64_t nbq = int64_t(1) << (2 * (L - s - 1));
    const int64_t tau = g / nbq, sq = g % nbq;
    auto low = [&](int c) { return tau * (nbq * 4) + child_id(L - s - 1, sq, c); };
    auto high = [&](int o) { return child_id(s, tau, o) * nbq + sq; };
    const float2* xin = Sin + col * SN;
    float2 acc[R];
#pragma unroll
    for (int v = 0; v < R; ++v) acc[v] = make_float2(0.f, 0.f);
    for (int w = 0; w < 4; ++w) {
        const float2* x = xin + (ADJ ? high(w) : low(w)) * R;
        const int o = ADJ ? w : u, c = ADJ ? u : w;
        const float2* ph = staged ? phs + ((g - g0) * 16 + o * 4 + c) * R : Ph + ((g * 4 + o) * 4 + c) * R;
        auto phv = [&](int i) { return staged ? ph[i] : __ldg(ph + i); };
        float2 xv[R];
#pragma unroll
        for (int t = 0; t < R; ++t) xv[t] = __ldg(x + t);
        if (SM) {
#pragma unroll
            for (int t = 0; t < R; ++t) xv[t] = ADJ ? cmulc(phv(t), xv[t]) : cmul(phv(t), xv[t]);
            const float* Aw = A + w * R * RP;
#pragma unroll
            for (int v = 0; v < R; ++v) acc[v] = cadd(acc[v], rowdot<R>(Aw + v * RP, xv));
        } else {
            const float* Au = A + u * R * RP;
#pragma unroll
            for (int v = 0; v < R; ++v) {
                const float2 tmp = rowdot<R>(Au + v * RP, xv);
                if (ADJ) cfmac(acc[v], phv(v), tmp);
                else cfma(acc[v], phv(v), tmp);
            }
        }
    }
    float2* out = Sout + col * SN + (ADJ ? low(u) : high(u)) * R;
#pragma unroll
    for (int v = 0; v < R; ++v) out[v] = acc[v];
}

// The same transfer level for r1 >= 6: thread (group, column, u) as above, but the R outputs in two
// halves of VH, one after the other, and the inner index t in blocks of four (one float4 of A per
// output row per block), so that a thread holds VH (SM) or 2 VH (MS) complex accumulators instead
// of 2 R values and two CTAs fit on an SM.  The SM form recomputes the phase products per half,
// the MS form reloads the inputs.
template <int R1, bool SM, bool ADJ>
__global__ void __launch_bounds__(TB, 2) k2_trans_h(const float2* __restrict__ Sin, float2* __restrict__ Sout,
                                                    int64_t SN, const float2* __restrict__ Ph,
                                                    const float* __restrict__ Am, int L, int s, int kc) {
    constexpr int R = G2<R1>::R, RP = G2<R1>::RP, VH = (R + 1) / 2;
    __shared__ __align__(16) float A[4 * R * RP];
    for (int i = threadIdx.x; i < 4 * R * RP; i += TB) A[i] = Am[i];
    __syncthreads();
    const int u = threadIdx.x & 3;
    const int64_t ngroups = int64_t(1) << (2 * L - 2);
    const int64_t item = int64_t(blockIdx.x) * (TB / 4) + (threadIdx.x >> 2);
    if (item >= ngroups * kc) return;
    const int col = int(item % kc);
    const int64_t g = item / kc;
    const int64_t nbq = int64_t(1) << (2 * (L - s - 1));
    const int64_t tau = g / nbq, sq = g % nbq;
    auto low = [&](int c) { return tau * (nbq * 4) + child_id(L - s - 1, sq, c); };
    auto high = [&](int o) { return child_id(s, tau, o) * nbq + sq; };
    const float2* xin = Sin + col * SN;
    float2* out = Sout + col * SN + (ADJ ? low(u) : high(u)) * R;
#pragma unroll 1
    for (int v0 = 0; v0 < R; v0 += VH) {
        const int nv = min(VH, R - v0);
        float2 acc[VH];
#pragma unroll
        for (int v = 0; v < VH; ++v) acc[v] = make_float2(0.f, 0.f);
#pragma unroll 1
        for (int w = 0; w < 4; ++w) {
            const float2* x = xin + (ADJ ? high(w) : low(w)) * R;
            const int o = ADJ ? w : u, c = ADJ ? u : w;
            const float2* ph = Ph + ((g * 4 + o) * 4 + c) * R;
            float2 tmp[SM ? 1 : VH];
            if (!SM)
#pragma unroll
                for (int v = 0; v < VH; ++v) tmp[v] = make_float2(0.f, 0.f);
            const float* Ab = A + ((SM ? w : u) * R + v0) * RP;   // rows v0 .. v0 + VH - 1
#pragma unroll 1
            for (int t0 = 0; t0 < R; t0 += 4) {
                float2 y[4];
#pragma unroll
                for (int d = 0; d < 4; ++d) {
                    const int t = min(t0 + d, R - 1);
                    const float2 xv = __ldg(x + t);
                    float2 v = xv;
                    if (SM) {
                        const float2 pv = __ldg(ph + t);
                        v = ADJ ? cmulc(pv, xv) : cmul(pv, xv);
                    }
                    y[d] = t0 + d < R ? v : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int v = 0; v < VH; ++v) {
                    if (v >= nv) break;
                    const float4 a = *reinterpret_cast<const float4*>(Ab + v * RP + t0);
                    float2& dst = SM ? acc[v] : tmp[SM ? 0 : v];
                    dst.x = fmaf(a.x, y[0].x, dst.x); dst.y = fmaf(a.x, y[0].y, dst.y);
                    dst.x = fmaf(a.y, y[1].x, dst.x); dst.y = fmaf(a.y, y[1].y, dst.y);
                    dst.x = fmaf(a.z, y[2].x, dst.x); dst.y = fmaf(a.z, y[2].y, dst.y);
                    dst.x = fmaf(a.w, y[3].x, dst.x); dst.y = fmaf(a.w, y[3].y, dst.y);
                }
            }
            if (!SM)
#pragma unroll
                for (int v = 0; v < VH; ++v) {
                    if (v >= nv) break;
                    const float2 pv = __ldg(ph + v0 + v);
                    if (ADJ) cfmac(acc[v], pv, tmp[v]);
                    else cfma(acc[v], pv, tmp[v]);
                }
        }
#pragma unroll
        for (int v = 0; v < VH; ++v) {
            if (v >= nv) break;
            out[v0 + v] = acc[v];
        }
    }
}

// Middle level: y[i] = sum_j M[p][i][j] x[j] (adjoint: x[j] = sum_i conj(M[p][i][j]) y[i]).
// CTA: MP pairs x TB / MP columns; thread (pair, column).
template <int R1, bool ADJ>
__global__ void __launch_bounds__(TB) k2_M(const float2* __restrict__ Sin, float2* __restrict__ Sout, int64_t SN,
                                           const float2* __restrict__ M, int64_t npairs, int kc) {
    constexpr int R = G2<R1>::R, MP = G2<R1>::MP, CPB = TB / MP;
    extern __shared__ float4 smem_m[];
    float2* Ms = reinterpret_cast<float2*>(smem_m);   // [MP][R*R]
    const int64_t p0 = int64_t(blockIdx.x) * MP;
    const int np = int(std::min<int64_t>(MP, npairs - p0));
    const float4* src = reinterpret_cast<const float4*>(M + p0 * R * R);
    float4* dst = reinterpret_cast<float4*>(Ms);
    for (int i = threadIdx.x; i < np * R * R / 2; i += TB) dst[i] = src[i];   // p0 even: 16-byte aligned
    if (np * R * R % 2) Ms[np * R * R - 1] = M[(p0 + np) * R * R - 1];
    __syncthreads();
    const int pl = threadIdx.x / CPB, col = blockIdx.y * CPB + threadIdx.x % CPB;
    if (pl >= np || col >= kc) return;
    const float2* m = Ms + pl * R * R;
    const float2* x = Sin + col * SN + (p0 + pl) * R;
    float2 acc[R];
#pragma unroll
    for (int v = 0; v < R; ++v) acc[v] = make_float2(0.f, 0.f);
    for (int w = 0; w < R; ++w) {
        const float2 xw = __ldg(x + w);
        if (ADJ) {
#pragma unroll
            for (int v = 0; v < R; ++v) cfmac(acc[v], m[w * R + v], xw);
        } else {
#pragma unroll
            for (int v = 0; v < R; ++v) cfma(acc[v], m[v * R + w], xw);
        }
    }
    float2* y = Sout + col * SN + (p0 + pl) * R;
#pragma unroll
    for (int v = 0; v < R; ++v) y[v] = acc[v];
}

// Middle level for r1 >= 6: CTA = MQP pairs x 16 columns x r1 chunks of r1 outputs; thread
// (chunk, pair, column); the M blocks of the MQP pairs staged in shared memory.
template <int R1, bool ADJ>
__global__ void __launch_bounds__(G2<R1>::MQ) k2_Mq(const float2* __restrict__ Sin, float2* __restrict__ Sout,
                                                    int64_t SN, const float2* __restrict__ M, int64_t npairs, int kc) {
    constexpr int R = G2<R1>::R, MP = G2<R1>::MQP, MQ = G2<R1>::MQ;
    extern __shared__ float4 smem_m[];
    float2* Ms = reinterpret_cast<float2*>(smem_m);   // [MQP][R*R]
    const int64_t p0 = int64_t(blockIdx.x) * MP;
    const int np = int(std::min<int64_t>(MP, npairs - p0));
    const float4* src = reinterpret_cast<const float4*>(M + p0 * R * R);
    float4* dst = reinterpret_cast<float4*>(Ms);
    for (int i = threadIdx.x; i < np * R * R / 2; i += MQ) dst[i] = src[i];   // p0 even: 16-byte aligned
    if (np * R * R % 2 && threadIdx.x == 0) Ms[np * R * R - 1] = M[(p0 + np) * R * R - 1];
    __syncthreads();
    const int q = threadIdx.x % R1, rest = threadIdx.x / R1, pl = rest % MP;
    const int col = blockIdx.y * 16 + rest / MP;
    if (pl >= np || col >= kc) return;
    const float2* m = Ms + pl * R * R;
    const float2* x = Sin + col * SN + (p0 + pl) * R;
    float2 acc[R1];
#pragma unroll
    for (int vv = 0; vv < R1; ++vv) acc[vv] = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int w = 0; w < R; ++w) {
        const float2 xw = __ldg(x + w);
#pragma unroll
        for (int vv = 0; vv < R1; ++vv) {
            const int v = q * R1 + vv;
            if (ADJ) cfmac(acc[vv], m[w * R + v], xw);
            else cfma(acc[vv], m[v * R + w], xw);
        }
    }
    float2* y = Sout + col * SN + (p0 + pl) * R + q * R1;
#pragma unroll
    for (int vv = 0; vv < R1; ++vv) y[vv] = acc[vv];
}

// U (forward): y(x) = sum_b UP[x][b] sum_i QU[x_loc][i] d(tau, b, i).
// CTA: one space leaf tau, 4 columns; thread (x_loc, column).
template <int R1>
__global__ void __launch_bounds__(TB) k2_U_fwd(const float2* __restrict__ S, int64_t SN, float2* __restrict__ Y,
                                               int64_t ld, const float2* __restrict__ UP, const float* __restrict__ QU,
                                               int n, int L, int sU, int kc) {
    constexpr int R = G2<R1>::R;
    extern __shared__ float4 smem_u[];
    float2(*ups)[65] = reinterpret_cast<float2(*)[65]>(smem_u);
    float2* ds = reinterpret_cast<float2*>(smem_u) + 64 * 65;      // [4][64][R]
    float* qu = reinterpret_cast<float*>(ds + 4 * 64 * R);          // [64][R]
    const int NP = 1 << (2 * (L - sU)), m = 1 << (L - sU);          // points per leaf = frequency boxes
    const int64_t tau = blockIdx.x;
    const int col0 = blockIdx.y * 4;
    const int t1 = int(tau >> sU), t2 = int(tau & ((int64_t(1) << sU) - 1));
    auto gx = [&](int x) { return int64_t(t1 * m + x / m) * n + t2 * m + x % m; };
    for (int idx = threadIdx.x; idx < NP * NP; idx += TB) ups[idx / NP][idx % NP] = UP[gx(idx / NP) * NP + idx % NP];
    for (int idx = threadIdx.x; idx < 4 * NP * R; idx += TB) {
        const int cl = idx / (NP * R), rem = idx % (NP * R);
        if (col0 + cl < kc) ds[cl * 64 * R + rem] = S[(col0 + cl) * SN + tau * NP * R + rem];
    }
    for (int idx = threadIdx.x; idx < NP * R; idx += TB) qu[idx] = QU[idx];
    __syncthreads();
    const int x = threadIdx.x & 63, cl = threadIdx.x >> 6;
    if (x >= NP || col0 + cl >= kc) return;
    float qq[R];
#pragma unroll
    for (int i = 0; i < R; ++i) qq[i] = qu[x * R + i];
    float2 acc = make_float2(0.f, 0.f);
    for (int b = 0; b < NP; ++b) {
        const float2* d = ds + (cl * 64 + b) * R;
        float2 tmp = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < R; ++i) {
            tmp.x = fmaf(qq[i], d[i].x, tmp.x);
            tmp.y = fmaf(qq[i], d[i].y, tmp.y);
        }
        cfma(acc, ups[x][b], tmp);
    }
    Y[(col0 + cl) * ld + gx(x)] = acc;
}

// U^*: d(tau, b, i) = sum_x QU[x_loc][i] conj(UP[x][b]) g(x).  Thread (b, column).
template <int R1>
__global__ void __launch_bounds__(TB) k2_U_adj(const float2* __restrict__ X, int64_t ld, float2* __restrict__ S,
                                               int64_t SN, const float2* __restrict__ UP, const float* __restrict__ QU,
                                               int n, int L, int sU, int kc) {
    constexpr int R = G2<R1>::R;
    __shared__ float2 ups[64][65];
    __shared__ float2 gs[4][64];
    __shared__ float qu[64 * R];
    const int NP = 1 << (2 * (L - sU)), m = 1 << (L - sU);
    const int64_t tau = blockIdx.x;
    const int col0 = blockIdx.y * 4;
    const int t1 = int(tau >> sU), t2 = int(tau & ((int64_t(1) << sU) - 1));
    auto gx = [&](int x) { return int64_t(t1 * m + x / m) * n + t2 * m + x % m; };
    for (int idx = threadIdx.x; idx < NP * NP; idx += TB) ups[idx / NP][idx % NP] = UP[gx(idx / NP) * NP + idx % NP];
    for (int idx = threadIdx.x; idx < 4 * NP; idx += TB) {
        const int cl = idx / NP, x = idx % NP;
        if (col0 + cl < kc) gs[cl][x] = X[(col0 + cl) * ld + gx(x)];
    }
    for (int idx = threadIdx.x; idx < NP * R; idx += TB) qu[idx] = QU[idx];
    __syncthreads();
    const int b = threadIdx.x & 63, cl = threadIdx.x >> 6;
    if (b >= NP || col0 + cl >= kc) return;
    float2 acc[R];
#pragma unroll
    for (int i = 0; i < R; ++i) acc[i] = make_float2(0.f, 0.f);
    for (int x = 0; x < NP; ++x) {
        const float2 v = cmulc(ups[x][b], gs[cl][x]);
#pragma unroll
        for (int i = 0; i < R; ++i) {
            acc[i].x = fmaf(qu[x * R + i], v.x, acc[i].x);
            acc[i].y = fmaf(qu[x * R + i], v.y, acc[i].y);
        }
    }
    float2* out = S + (col0 + cl) * SN + (tau * NP + b) * R;
#pragma unroll
    for (int i = 0; i < R; ++i) out[i] = acc[i];
}

// ---------------------------------------------------------------- sampled entries (FP64)
__device__ __forceinline__ double2 expi_d(double ph) {
    const double fr = ph - rint(ph);
    double sn, cs;
    sincospi(2.0 * fr, &sn, &cs);
    return make_double2(cs, sn);
}
__device__ __forceinline__ double2 zmul2(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// 1D Lagrange polynomial l_k on the r1 Chebyshev points, at the box coordinate v in [-1, 1]
__device__ double lag1_d(const Cheb2& ch, int r1, int k, double v) {
    double p = 1.0;
    for (int m = 0; m < r1; ++m)
        if (m != k) p *= (v - ch.t[m]) / (ch.t[k] - ch.t[m]);
    return p;
}
// the Hankel amplitude of Section 5.3 in FP64
__device__ __forceinline__ double2 hankel_amp_d(double ph) {
    const double z = 2.0 * M_PI * ph;
    const double2 w = expi_d(-ph);
    return zmul2(make_double2(j0(z), y0(z)), w);
}
// box of space level s holding the point (i1, i2) / n, and of frequency level l holding (j1, j2)
__device__ __forceinline__ int64_t box_at(int64_t i1, int64_t i2, int L, int s) {
    return ((i1 >> (L - s)) << s) + (i2 >> (L - s));
}

// One sampled entry per thread, as the 1D k_entry_chain: K~(i, j) in FP64 from the factor entries
// (tensor Chebyshev grids of r1 x r1 points, four children per box) along the single chain of pairs
// (box of space level s holding x_i, box of frequency level L - s holding xi_j), and the exact K(i, j).
// A Hankel sample at xi = 0 (where the amplitude is infinite) is written as zeros.
template <int R1>
__global__ void k2_entry_chain(const int64_t* __restrict__ rows, const int64_t* __restrict__ cols, int S, Ph2 kind,
                               int amp_kind, Cheb2 ch, int n, int L, int h, int sU, int sV, double2* __restrict__ out) {
    constexpr int R = G2<R1>::R;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= S) return;
    const int64_t i = rows[e], j = cols[e];
    const int64_t i1 = i / n, i2 = i % n, j1 = j / n, j2 = j % n;
    const double x1 = double(i1) / n, x2 = double(i2) / n, k1 = double(j1) - 0.5 * n, k2 = double(j2) - 0.5 * n;
    if (amp_kind == FIO_AMP_HANKEL && k1 == 0.0 && k2 == 0.0) {
        out[2 * e] = out[2 * e + 1] = make_double2(0.0, 0.0);
        return;
    }
    double2 c[R], d[R];
    auto fhalf = [&](int l) { return ldexp(double(n), -l - 1); };
    auto amp = [&](double a1, double a2, double b1, double b2) {
        return amp_kind == FIO_AMP_HANKEL ? hankel_amp_d(phi2_nl(kind.kind, kind.s, a1, a2, b1, b2)) : make_double2(1.0, 0.0);
    };
    {   // V at space level sV
        const int l = L - sV;
        const int64_t tau = box_at(i1, i2, L, sV), sg = box_at(j1, j2, L, l);
        const double y1 = sctr(sV, tau, 0), y2 = sctr(sV, tau, 1);
        const double v1 = (k1 - fctr(n, l, sg, 0)) / fhalf(l), v2 = (k2 - fctr(n, l, sg, 1)) / fhalf(l);
        for (int t = 0; t < R; ++t) {
            const double g1 = fnode(ch, n, l, sg, 0, t / R1), g2 = fnode(ch, n, l, sg, 1, t % R1);
            const double2 w = expi_d(phi2(kind, y1, y2, k1, k2) - phi2(kind, y1, y2, g1, g2));
            const double q = lag1_d(ch, R1, t / R1, v1) * lag1_d(ch, R1, t % R1, v2);
            c[t] = make_double2(w.x * q, w.y * q);
        }
    }
    for (int s = sV; s < h; ++s) {   // C, pair level s -> s+1
        const int l1 = L - s - 1;
        const int64_t tau1 = box_at(i1, i2, L, s + 1), sg1 = box_at(j1, j2, L, l1), beta = box_at(j1, j2, L, L - s);
        const double y1 = sctr(s + 1, tau1, 0), y2 = sctr(s + 1, tau1, 1);
        const double f1 = fctr(n, l1, sg1, 0), f2 = fctr(n, l1, sg1, 1);
        for (int jj = 0; jj < R; ++jj) {
            const double gj1 = fnode(ch, n, l1, sg1, 0, jj / R1), gj2 = fnode(ch, n, l1, sg1, 1, jj % R1);
            double2 acc = make_double2(0.0, 0.0);
            for (int t = 0; t < R; ++t) {
                const double gb1 = fnode(ch, n, L - s, beta, 0, t / R1), gb2 = fnode(ch, n, L - s, beta, 1, t % R1);
                const double2 w = zmul2(expi_d(phi2(kind, y1, y2, gb1, gb2) - phi2(kind, y1, y2, gj1, gj2)), c[t]);
                const double q = lag1_d(ch, R1, jj / R1, (gb1 - f1) / fhalf(l1)) * lag1_d(ch, R1, jj % R1, (gb2 - f2) / fhalf(l1));
                acc.x += q * w.x;
                acc.y += q * w.y;
            }
            d[jj] = acc;
        }
        for (int t = 0; t < R; ++t) c[t] = d[t];
    }
    {   // M at level h
        const int64_t tau = box_at(i1, i2, L, h), sg = box_at(j1, j2, L, L - h);
        for (int ii = 0; ii < R; ++ii) {
            const double z1 = snode(ch, h, tau, 0, ii / R1), z2 = snode(ch, h, tau, 1, ii % R1);
            double2 acc = make_double2(0.0, 0.0);
            for (int t = 0; t < R; ++t) {
                const double g1 = fnode(ch, n, L - h, sg, 0, t / R1), g2 = fnode(ch, n, L - h, sg, 1, t % R1);
                const double2 w = zmul2(zmul2(amp(z1, z2, g1, g2), expi_d(phi2(kind, z1, z2, g1, g2))), c[t]);
                acc.x += w.x;
                acc.y += w.y;
            }
            d[ii] = acc;
        }
    }
    for (int s = h; s < sU; ++s) {   // B, pair level s -> s+1
        const int64_t al = box_at(i1, i2, L, s), tau1 = box_at(i1, i2, L, s + 1), beta = box_at(j1, j2, L, L - s);
        const double e1 = fctr(n, L - s, beta, 0), e2 = fctr(n, L - s, beta, 1);
        const double ya1 = sctr(s, al, 0), ya2 = sctr(s, al, 1);
        for (int ii = 0; ii < R; ++ii) {
            const double z1 = snode(ch, s + 1, tau1, 0, ii / R1), z2 = snode(ch, s + 1, tau1, 1, ii % R1);
            const double p1 = ldexp(1.0, s + 1) * (z1 - ya1), p2 = ldexp(1.0, s + 1) * (z2 - ya2);
            double2 acc = make_double2(0.0, 0.0);
            for (int t = 0; t < R; ++t) {
                const double za1 = snode(ch, s, al, 0, t / R1), za2 = snode(ch, s, al, 1, t % R1);
                const double2 w = zmul2(expi_d(phi2(kind, z1, z2, e1, e2) - phi2(kind, za1, za2, e1, e2)), d[t]);
                const double p = lag1_d(ch, R1, t / R1, p1) * lag1_d(ch, R1, t % R1, p2);
                acc.x += p * w.x;
                acc.y += p * w.y;
            }
            c[ii] = acc;
        }
        for (int t = 0; t < R; ++t) d[t] = c[t];
    }
    double2 y = make_double2(0.0, 0.0);
    {   // U at space level sU
        const int64_t tau = box_at(i1, i2, L, sU), sg = box_at(j1, j2, L, L - sU);
        const double e1 = fctr(n, L - sU, sg, 0), e2 = fctr(n, L - sU, sg, 1);
        const double p1 = ldexp(1.0, sU + 1) * (x1 - sctr(sU, tau, 0)), p2 = ldexp(1.0, sU + 1) * (x2 - sctr(sU, tau, 1));
        for (int t = 0; t < R; ++t) {
            const double z1 = snode(ch, sU, tau, 0, t / R1), z2 = snode(ch, sU, tau, 1, t % R1);
            const double2 w = zmul2(expi_d(phi2(kind, x1, x2, e1, e2) - phi2(kind, z1, z2, e1, e2)), d[t]);
            const double p = lag1_d(ch, R1, t / R1, p1) * lag1_d(ch, R1, t % R1, p2);
            y.x += p * w.x;
            y.y += p * w.y;
        }
    }
    out[2 * e] = y;
    out[2 * e + 1] = zmul2(amp(x1, x2, k1, k2), expi_d(phi2(kind, x1, x2, k1, k2)));
}

// Lexicographic <- Morton reordering of frequency vectors: X[j] = Xm[morton(j)].
__global__ void k2_unmorton(const float2* __restrict__ Xm, float2* __restrict__ X, int n, int L, int64_t ld) {
    const int64_t N = int64_t(n) * n;
    const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const int col = blockIdx.y;
    X[col * ld + j] = Xm[col * ld + morton(int(j / n), int(j % n), L)];
}

template <int R1>
constexpr size_t smem_leaf() {   // V^* and U: 64 x 65 phases, 4 columns x 64 x R states, 64 x R basis values
    return (64 * 65 + 4 * 64 * G2<R1>::R) * sizeof(float2) + G2<R1>::R * 64 * sizeof(float);
}
template <int R1>
constexpr size_t smem_mid() {
    return size_t(G2<R1>::CHUNK_M ? G2<R1>::MQP : G2<R1>::MP) * G2<R1>::R * G2<R1>::R * sizeof(float2);
}

// real tables: Pc | Pc^T (4 children x R rows of RP) | QV (R x NA) | QU (NP x R)
size_t off_P() { return 0; }
size_t off_PT(int R, int RP) { return size_t(4) * R * RP; }
size_t off_QV(int R, int RP) { return size_t(8) * R * RP; }
size_t off_QU(int R, int RP, int NA) { return off_QV(R, RP) + size_t(R) * NA; }

}  // namespace

bool bf2d_ok_kind(int kind) {
    return kind == FIO_PHASE_DFT || kind == FIO_PHASE_2D_ELLIPTIC || kind == FIO_PHASE_2D_ISO;
}

bool bf2d_ok_r1(int r1) { return r1 >= kMinR1 && r1 <= kMaxR1; }

namespace {

template <int R1>
fio_status build2(fio_bf* bf, cudaStream_t st) {
    constexpr int R = G2<R1>::R, RP = G2<R1>::RP;
    const int n = bf->nside, L = bf->L;
    const int NA = 1 << (2 * bf->sV), NP = 1 << (2 * (L - bf->sU));
    const int mV = 1 << bf->sV, mU = 1 << (L - bf->sU);
    Cheb2 ch{};
    for (int k = 0; k < R1; ++k) ch.t[k] = std::cos((2.0 * k + 1.0) * M_PI / (2.0 * R1));
    // real tables: Pc, Pc^T, QV, QU
    std::vector<float> P(off_QU(R, RP, NA) + size_t(NP) * R, 0.f);
    auto l1 = [&](int k, double u) { return lagrange_host(ch.t, R1, k, u); };
    for (int c = 0; c < 4; ++c)
        for (int j = 0; j < R; ++j)
            for (int t = 0; t < R; ++t) {
                const double v = l1(j / R1, (c >> 1) - 0.5 + 0.5 * ch.t[t / R1]) * l1(j % R1, (c & 1) - 0.5 + 0.5 * ch.t[t % R1]);
                P[off_P() + (c * R + j) * RP + t] = float(v);
                P[off_PT(R, RP) + (c * R + t) * RP + j] = float(v);
            }
    for (int t = 0; t < R; ++t)
        for (int q = 0; q < NA; ++q)
            P[off_QV(R, RP) + t * NA + q] =
                float(l1(t / R1, 2.0 * (q / mV) / mV - 1.0) * l1(t % R1, 2.0 * (q % mV) / mV - 1.0));
    for (int x = 0; x < NP; ++x)
        for (int i = 0; i < R; ++i)
            P[off_QU(R, RP, NA) + x * R + i] =
                float(l1(i / R1, 2.0 * (x / mU) / mU - 1.0) * l1(i % R1, 2.0 * (x % mU) / mU - 1.0));
    FIO_TRY(bf->P.ensure(P.size() * sizeof(float)));
    FIO_CUDA(cudaMemcpyAsync(bf->P.p, P.data(), P.size() * sizeof(float), cudaMemcpyHostToDevice, st));
    const int64_t N = int64_t(n) * n;
    const Ph2 kind{bf->phase.kind, bf->phase.s};
    const int64_t nVP = int64_t(NA) * N, nUP = N * NP, nM = N * R * R, nT = N / 4 * 16 * R;
    FIO_TRY(bf->VP.ensure(nVP * 8));
    FIO_TRY(bf->UP.ensure(nUP * 8));
    FIO_TRY(bf->M.ensure(nM * 8));
    k2_tab_VP<<<cdiv(nVP, TB), TB, 0, st>>>(bf->VP.as<float2>(), kind, n, bf->sV);
    k2_tab_UP<<<cdiv(nUP, TB), TB, 0, st>>>(bf->UP.as<float2>(), kind, n, L, bf->sU);
    k2_tab_M<R1><<<cdiv(nM, TB), TB, 0, st>>>(bf->M.as<float2>(), kind, bf->amp.kind, ch, n, L, bf->h);
    bf->C.resize(bf->h - bf->sV);
    for (int s = bf->sV; s < bf->h; ++s) {
        FIO_TRY(bf->C[s - bf->sV].ensure(nT * 8));
        k2_tab_F<R1><<<cdiv(nT, TB), TB, 0, st>>>(bf->C[s - bf->sV].as<float2>(), kind, ch, n, L, s);
    }
    bf->B.resize(bf->sU - bf->h);
    for (int s = bf->h; s < bf->sU; ++s) {
        FIO_TRY(bf->B[s - bf->h].ensure(nT * 8));
        k2_tab_E<R1><<<cdiv(nT, TB), TB, 0, st>>>(bf->B[s - bf->h].as<float2>(), kind, ch, n, L, s);
    }
    FIO_CUDA(cudaGetLastError());
    FIO_CUDA(cudaStreamSynchronize(st));
    bf->table_bytes = (nVP + nUP + nM + nT * int64_t(bf->C.size() + bf->B.size())) * 8 + int64_t(P.size()) * 4;
    static PerDeviceOnce attrs;
    FIO_CUDA(attrs.run([] {
        constexpr int sl = int(smem_leaf<R1>()), sm = int(smem_mid<R1>());
        cudaError_t e = cudaFuncSetAttribute(k2_V_adj<R1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sl);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k2_U_fwd<R1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sl);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k2_M<R1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k2_M<R1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        if (e == cudaSuccess && G2<R1>::CHUNK_M)
            e = cudaFuncSetAttribute(k2_Mq<R1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        if (e == cudaSuccess && G2<R1>::CHUNK_M)
            e = cudaFuncSetAttribute(k2_Mq<R1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        return e;
    }));
    return FIO_OK;
}

// kc columns; states s0, s1 of N * R * kc complex each.
template <int R1>
fio_status apply2(const fio_bf* bf, const float2* X, float2* Y, int64_t ld, int kc, int adjoint, bool mort, float2* s0,
                  float2* s1, cudaStream_t st) {
    constexpr int R = G2<R1>::R, RP = G2<R1>::RP, MP = G2<R1>::MP;
    constexpr size_t sl = smem_leaf<R1>(), sm = smem_mid<R1>();
    const int n = bf->nside, L = bf->L, h = bf->h, sU = bf->sU, sV = bf->sV;
    const int64_t N = int64_t(n) * n, SN = N * R;
    const int NA = 1 << (2 * sV);
    const float* Pm = bf->P.as<float>();
    const float* QV = Pm + off_QV(R, RP);
    const float* QU = Pm + off_QU(R, RP, NA);
    const float* Pc = Pm + off_P();
    const float* PcT = Pm + off_PT(R, RP);
    const int64_t ngroups = N / 4;
    const unsigned gtr = cdiv(ngroups * kc, TB / 4);
    const dim3 gV(unsigned(int64_t(1) << (2 * (L - sV))), cdiv(kc, 4));
    const dim3 gU(unsigned(int64_t(1) << (2 * sU)), cdiv(kc, 4));
    const dim3 gM(cdiv(N, MP), cdiv(kc, TB / MP)), gMq(cdiv(N, G2<R1>::MQP), cdiv(kc, 16));
    // transfer kernels: all outputs per thread, or for the scale-then-mix form at r1 >= 6 in two
    // halves (measured at n = 256, r1 = 7: 527 against 487 GB/s; the mix-then-scale form is faster
    // with all outputs per thread, 509 against 373 GB/s)
    using TransK = void (*)(const float2*, float2*, int64_t, const float2*, const float*, int, int, int);
    constexpr bool HALF = G2<R1>::CHUNK_M;
    const TransK kCf = HALF ? k2_trans_h<R1, true, false> : k2_trans<R1, true, false>;
    const TransK kBf = k2_trans<R1, false, false>;
    const TransK kBa = HALF ? k2_trans_h<R1, true, true> : k2_trans<R1, true, true>;
    const TransK kCa = k2_trans<R1, false, true>;
    float2* cur = s0;
    float2* oth = s1;
    const int m = mort ? 1 : 0;
    if (!adjoint) {
        FIO_LAUNCH("k2_V_fwd", st, k2_V_fwd<R1><<<gV, TB, 0, st>>>(X, ld, cur, SN, bf->VP.as<float2>(), QV, n, L, sV, kc, m));
        for (int s = sV; s < h; ++s) {
            FIO_LAUNCH("k2_C_fwd", st, (kCf<<<gtr, TB, 0, st>>>(cur, oth, SN, bf->C[s - sV].as<float2>(),
                                                                                     Pc, L, s, kc)));
            std::swap(cur, oth);
        }
        if (G2<R1>::CHUNK_M)
            FIO_LAUNCH("k2_M_fwd", st, (k2_Mq<R1, false><<<gMq, G2<R1>::MQ, sm, st>>>(cur, oth, SN, bf->M.as<float2>(), N, kc)));
        else
            FIO_LAUNCH("k2_M_fwd", st, (k2_M<R1, false><<<gM, TB, sm, st>>>(cur, oth, SN, bf->M.as<float2>(), N, kc)));
        std::swap(cur, oth);
        for (int s = h; s < sU; ++s) {
            FIO_LAUNCH("k2_B_fwd", st, (kBf<<<gtr, TB, 0, st>>>(cur, oth, SN, bf->B[s - h].as<float2>(),
                                                                                      PcT, L, s, kc)));
            std::swap(cur, oth);
        }
        FIO_LAUNCH("k2_U_fwd", st, k2_U_fwd<R1><<<gU, TB, sl, st>>>(cur, SN, Y, ld, bf->UP.as<float2>(), QU, n, L, sU, kc));
    } else {
        FIO_LAUNCH("k2_U_adj", st, k2_U_adj<R1><<<gU, TB, 0, st>>>(X, ld, cur, SN, bf->UP.as<float2>(), QU, n, L, sU, kc));
        for (int s = sU - 1; s >= h; --s) {
            FIO_LAUNCH("k2_B_adj", st, (kBa<<<gtr, TB, 0, st>>>(cur, oth, SN, bf->B[s - h].as<float2>(),
                                                                                    Pc, L, s, kc)));
            std::swap(cur, oth);
        }
        if (G2<R1>::CHUNK_M)
            FIO_LAUNCH("k2_M_adj", st, (k2_Mq<R1, true><<<gMq, G2<R1>::MQ, sm, st>>>(cur, oth, SN, bf->M.as<float2>(), N, kc)));
        else
            FIO_LAUNCH("k2_M_adj", st, (k2_M<R1, true><<<gM, TB, sm, st>>>(cur, oth, SN, bf->M.as<float2>(), N, kc)));
        std::swap(cur, oth);
        for (int s = h - 1; s >= sV; --s) {
            FIO_LAUNCH("k2_C_adj", st, (kCa<<<gtr, TB, 0, st>>>(cur, oth, SN, bf->C[s - sV].as<float2>(),
                                                                                     PcT, L, s, kc)));
            std::swap(cur, oth);
        }
        FIO_LAUNCH("k2_V_adj", st, k2_V_adj<R1><<<gV, TB, sl, st>>>(cur, SN, Y, ld, bf->VP.as<float2>(), QV, n, L, sV, kc, m));
    }
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}

int r1_of(const fio_bf* bf) {
    int r1 = 1;
    while ((r1 + 1) * (r1 + 1) <= bf->r) ++r1;
    return r1;
}

}  // namespace

fio_status bf2d_build(fio_bf* bf, cudaStream_t st) {
    switch (r1_of(bf)) {
        case 3: return build2<3>(bf, st);
        case 4: return build2<4>(bf, st);
        case 5: return build2<5>(bf, st);
        case 6: return build2<6>(bf, st);
        case 7: return build2<7>(bf, st);
    }
    return fail(FIO_EINVAL, "bf_build: 2D needs r = r1^2 with 3 <= r1 <= 7");
}

fio_status bf2d_apply_cols(const fio_bf* bf, const float2* X, float2* Y, int64_t ld, int kc, int adjoint, bool mort,
                           float2* s0, float2* s1, cudaStream_t st) {
    switch (r1_of(bf)) {
        case 3: return apply2<3>(bf, X, Y, ld, kc, adjoint, mort, s0, s1, st);
        case 4: return apply2<4>(bf, X, Y, ld, kc, adjoint, mort, s0, s1, st);
        case 5: return apply2<5>(bf, X, Y, ld, kc, adjoint, mort, s0, s1, st);
        case 6: return apply2<6>(bf, X, Y, ld, kc, adjoint, mort, s0, s1, st);
        case 7: return apply2<7>(bf, X, Y, ld, kc, adjoint, mort, s0, s1, st);
    }
    return fail(FIO_EINVAL, "bf_apply: 2D handle with an unsupported rank");
}

namespace {
template <int R1>
fio_status entries2(const fio_phase& phase, int amp_kind, int n, const int64_t* rows, const int64_t* cols, int S,
                    double2* out, cudaStream_t st) {
    const int L = ilog2_exact(n);
    const int h = L / 2, sU = std::max(L - 3, h), sV = std::min(3, h);
    Cheb2 ch{};
    for (int k = 0; k < R1; ++k) ch.t[k] = std::cos((2.0 * k + 1.0) * M_PI / (2.0 * R1));
    const Ph2 kind{phase.kind, phase.s};
    FIO_LAUNCH("k2_entry_chain", st,
               (k2_entry_chain<R1><<<cdiv(S, 64), 64, 0, st>>>(rows, cols, S, kind, amp_kind, ch, n, L, h, sU, sV, out)));
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}
}  // namespace

fio_status bf2d_entries(const fio_phase& phase, int amp_kind, int n, int r1, const int64_t* rows, const int64_t* cols,
                        int S, double2* out, cudaStream_t st) {
    switch (r1) {
        case 3: return entries2<3>(phase, amp_kind, n, rows, cols, S, out, st);
        case 4: return entries2<4>(phase, amp_kind, n, rows, cols, S, out, st);
        case 5: return entries2<5>(phase, amp_kind, n, rows, cols, S, out, st);
        case 6: return entries2<6>(phase, amp_kind, n, rows, cols, S, out, st);
        case 7: return entries2<7>(phase, amp_kind, n, rows, cols, S, out, st);
    }
    return fail(FIO_EINVAL, "2D rank r1 must be in [3, 7]");
}

fio_status bf2d_unmorton(const fio_bf* bf, const float2* Xm, float2* X, int64_t ld, int k, cudaStream_t st) {
    const int64_t N = int64_t(bf->nside) * bf->nside;
    for (int c0 = 0; c0 < k; c0 += 65535) {
        const int cc = std::min(65535, k - c0);
        FIO_LAUNCH("k2_unmorton", st, (k2_unmorton<<<dim3(cdiv(N, TB), cc), TB, 0, st>>>(Xm + c0 * ld, X + c0 * ld,
                                                                                        bf->nside, bf->L, ld)));
    }
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}

}  // namespace fio
