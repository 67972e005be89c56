// Butterfly factorization: device evaluation of the factors (bf_build) and
// the forward / adjoint products (bf_apply), Section 2.2, Eq. 2.1.
#include <cmath>
#include <cstring>

#include "bf.cuh"
#include "hss.cuh"

namespace fio {
namespace {

constexpr int kMaxR = 16;   // rank bound of the warp-per-quad transfer kernels

struct PhaseDev {
    int kind;
    double s;
};
struct Cheb {
    double t[32];
};

// Phi(x, xi) of the 1D families (Eq. 1.1 with the phases of the workloads).
__device__ __forceinline__ double phi(const PhaseDev& p, double x, double xi) {
    double v = x * xi;
    if (p.kind == FIO_PHASE_1D_CABS) v += (2.0 + p.s * sinpi(2.0 * x)) * 0.0625 * fabs(xi);
    if (p.kind == FIO_PHASE_1D_CABS8) v += (2.0 + p.s * sinpi(2.0 * x)) * 0.125 * fabs(xi);
    return v;
}

// a(x, xi) of the 1D amplitudes (Gaussian bumps of Section 5.1, or 1).
__device__ __forceinline__ double amp1d(const AmpDev& a, double x, double xi) {
    if (a.kind != FIO_AMP_BUMPS) return 1.0;
    double v = 0.0;
    for (int k = 0; k < a.m; ++k) {
        const double dx = x - a.c[2 * k], dxi = (xi - a.c[2 * k + 1]) / a.N;
        v += exp(-(dx * dx + dxi * dxi) / a.sigma2);
    }
    return v;
}

// e^{2 pi i ph} for an FP64 phase: reduce modulo 1 in FP64, then sin/cos of
// the small remainder.
__device__ __forceinline__ float2 expi2pi(double ph) {
    double fr = ph - rint(ph);
    float sn, cs;
    sincospif(2.0f * float(fr), &sn, &cs);
    return make_float2(cs, sn);
}

__device__ __forceinline__ double space_center(int s, int64_t a) { return ldexp(double(a) + 0.5, -s); }
__device__ __forceinline__ double space_node(const Cheb& c, int s, int64_t a, int k) {
    return space_center(s, a) + ldexp(0.5, -s) * c.t[k];
}
__device__ __forceinline__ double freq_center(int n, int l, int64_t b) {
    return -0.5 * n + (double(b) + 0.5) * ldexp(double(n), -l);
}
__device__ __forceinline__ double freq_node(const Cheb& c, int n, int l, int64_t b, int k) {
    return freq_center(n, l, b) + ldexp(double(n), -l - 1) * c.t[k];
}

// ---------------------------------------------------------------- tables
__global__ void k_tab_VP(float2* VP, PhaseDev ph, int n, int sV) {
    int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    int64_t total = (int64_t(1) << sV) * n;
    if (e >= total) return;
    int64_t a = e / n, j = e % n;
    VP[e] = expi2pi(phi(ph, space_center(sV, a), double(j) - 0.5 * n));
}

__global__ void k_tab_UP(float2* UP, PhaseDev ph, int n, int L, int sU) {
    int nb = 1 << (L - sU);
    int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= int64_t(n) * nb) return;
    int64_t i = e / nb, b = e % nb;
    UP[e] = expi2pi(phi(ph, double(i) / n, freq_center(n, L - sU, b)));
}

// F_s[q][c][beta][t], quad (tau at space level s, b' at frequency level L-s-1)
// stored at q = box 2^(h-1) + tau 2^(h-s-1) + (b' mod 2^(h-s-1)), box = the
// frequency box of level L-h holding b' (contiguous per box for the fused apply).
__device__ __forceinline__ int64_t fquad(int64_t tau, int64_t bq, int h, int s) {
    int64_t box = bq >> (h - s - 1), sl = bq & ((int64_t(1) << (h - s - 1)) - 1);
    return (box << (h - 1)) + (tau << (h - s - 1)) + sl;
}

__global__ void k_tab_F(float2* F, PhaseDev ph, Cheb ch, int n, int L, int h, int s, int r) {
    int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    int64_t nquad = int64_t(n) / 2;
    if (e >= nquad * 4 * r) return;
    int t = int(e % r);
    int64_t rest = e / r;
    int be = int(rest & 1), c = int((rest >> 1) & 1);
    int64_t qR = rest >> 2;
    int64_t box = qR >> (h - 1), rem = qR & ((int64_t(1) << (h - 1)) - 1);
    int64_t tau = rem >> (h - s - 1), bq = (box << (h - s - 1)) + (rem & ((int64_t(1) << (h - s - 1)) - 1));
    double g = freq_node(ch, n, L - s, 2 * bq + be, t);
    double yc = space_center(s + 1, 2 * tau + c), yp = space_center(s, tau);
    F[e] = expi2pi(phi(ph, yc, g) - phi(ph, yp, g));
}

// E_s[q][c][beta][i], quad q = (alpha at space level s, b' at frequency level L-s-1).
__global__ void k_tab_E(float2* E, PhaseDev ph, Cheb ch, int n, int L, int s, int r) {
    int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    int64_t nquad = int64_t(n) / 2;
    if (e >= nquad * 4 * r) return;
    int i = int(e % r);
    int64_t rest = e / r;
    int be = int(rest & 1), c = int((rest >> 1) & 1);
    int64_t q = rest >> 2;
    int64_t nbq = int64_t(1) << (L - s - 1);
    int64_t al = q / nbq, bq = q % nbq;
    double z = space_node(ch, s + 1, 2 * al + c, i);
    E[e] = expi2pi(phi(ph, z, freq_center(n, L - s, 2 * bq + be)) - phi(ph, z, freq_center(n, L - s - 1, bq)));
}

// M[p][i][j], pair p = tau * 2^(L-h) + sigma at the middle level h; the amplitude
// a(z_i, gamma_j) multiplies the entry (it enters no other factor).
__global__ void k_tab_M(float2* M, PhaseDev ph, AmpDev amp, Cheb ch, int n, int L, int h, int r) {
    int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= int64_t(n) * r * r) return;
    int j = int(e % r), i = int((e / r) % r);
    int64_t p = e / (int64_t(r) * r);
    int64_t nb = int64_t(1) << (L - h);
    int64_t tau = p / nb, sg = p % nb;
    double z = space_node(ch, h, tau, i), y = space_center(h, tau);
    double g = freq_node(ch, n, L - h, sg, j), eta = freq_center(n, L - h, sg);
    const float2 m = expi2pi(phi(ph, z, g) - phi(ph, z, eta) - phi(ph, y, g));
    M[e] = amp.kind == FIO_AMP_ONE ? m : cscale(m, float(amp1d(amp, z, g)));
}

// ---------------------------------------------------------------- apply
// V: c(a,b,j) = sum_q PV[q][j] VP[a][b ls + q] x(b ls + q)
__global__ void k_V_fwd(const float2* __restrict__ X, int64_t ld, float2* __restrict__ S, const float2* __restrict__ VP,
                        const float* __restrict__ PV, int n, int L, int sV, int r) {
    extern __shared__ float sP[];
    int ls = 1 << sV, nb = 1 << (L - sV);
    for (int e = threadIdx.x; e < ls * r; e += blockDim.x) sP[e] = PV[e];
    __syncthreads();
    int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    int col = blockIdx.y;
    if (e >= int64_t(n) * r) return;
    int j = int(e % r);
    int64_t p = e / r, a = p / nb, b = p % nb;
    const float2* x = X + col * ld + b * ls;
    const float2* vp = VP + a * n + b * ls;
    float2 acc = make_float2(0.f, 0.f);
    for (int q = 0; q < ls; ++q) {
        float2 v = cmul(vp[q], x[q]);
        acc.x = fmaf(sP[q * r + j], v.x, acc.x);
        acc.y = fmaf(sP[q * r + j], v.y, acc.y);
    }
    S[int64_t(col) * n * r + e] = acc;
}

// V^*: f(j) = sum_a conj(VP[a][j]) sum_t PV[q][t] c(a,b,t),  j = b ls + q
__global__ void k_V_adj(const float2* __restrict__ S, float2* __restrict__ Y, int64_t ld, const float2* __restrict__ VP,
                        const float* __restrict__ PV, int n, int L, int sV, int r) {
    extern __shared__ float sP[];
    int ls = 1 << sV, nb = 1 << (L - sV), na = 1 << sV;
    for (int e = threadIdx.x; e < ls * r; e += blockDim.x) sP[e] = PV[e];
    __syncthreads();
    int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    int col = blockIdx.y;
    if (j >= n) return;
    int64_t b = j / ls;
    int q = int(j % ls);
    const float2* st = S + int64_t(col) * n * r;
    float2 out = make_float2(0.f, 0.f);
    for (int a = 0; a < na; ++a) {
        const float2* c = st + (int64_t(a) * nb + b) * r;
        float2 acc = make_float2(0.f, 0.f);
        for (int t = 0; t < r; ++t) {
            acc.x = fmaf(sP[q * r + t], c[t].x, acc.x);
            acc.y = fmaf(sP[q * r + t], c[t].y, acc.y);
        }
        cfmac(out, VP[int64_t(a) * n + j], acc);
    }
    Y[col * ld + j] = out;
}

// U: y(x) = sum_b UP[x][b] sum_i PU[q][i] d(a,b,i),  x = a ls + q
__global__ void k_U_fwd(const float2* __restrict__ S, float2* __restrict__ Y, int64_t ld, const float2* __restrict__ UP,
                        const float* __restrict__ PU, int n, int L, int sU, int r) {
    extern __shared__ float sP[];
    int ls = 1 << (L - sU), nb = ls;
    for (int e = threadIdx.x; e < ls * r; e += blockDim.x) sP[e] = PU[e];
    __syncthreads();
    int64_t x = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    int col = blockIdx.y;
    if (x >= n) return;
    int64_t a = x / ls;
    int q = int(x % ls);
    const float2* st = S + int64_t(col) * n * r;
    float2 out = make_float2(0.f, 0.f);
    for (int b = 0; b < nb; ++b) {
        const float2* d = st + (a * nb + b) * r;
        float2 acc = make_float2(0.f, 0.f);
        for (int i = 0; i < r; ++i) {
            acc.x = fmaf(sP[q * r + i], d[i].x, acc.x);
            acc.y = fmaf(sP[q * r + i], d[i].y, acc.y);
        }
        cfma(out, UP[x * nb + b], acc);
    }
    Y[col * ld + x] = out;
}

// U^*: d(a,b,i) = sum_q PU[q][i] conj(UP[a ls + q][b]) g(a ls + q)
__global__ void k_U_adj(const float2* __restrict__ X, int64_t ld, float2* __restrict__ S, const float2* __restrict__ UP,
                        const float* __restrict__ PU, int n, int L, int sU, int r) {
    extern __shared__ float sP[];
    int ls = 1 << (L - sU), nb = ls;
    for (int e = threadIdx.x; e < ls * r; e += blockDim.x) sP[e] = PU[e];
    __syncthreads();
    int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    int col = blockIdx.y;
    if (e >= int64_t(n) * r) return;
    int i = int(e % r);
    int64_t p = e / r, a = p / nb, b = p % nb;
    const float2* g = X + col * ld + a * ls;
    float2 acc = make_float2(0.f, 0.f);
    for (int q = 0; q < ls; ++q) {
        float2 v = cmulc(UP[(a * ls + q) * nb + b], g[q]);
        acc.x = fmaf(sP[q * r + i], v.x, acc.x);
        acc.y = fmaf(sP[q * r + i], v.y, acc.y);
    }
    S[int64_t(col) * n * r + e] = acc;
}

// M (forward): d(p,i) = sum_j M[p][i][j] c(p,j);  M^*: c(p,j) = sum_i conj(M[p][i][j]) d(p,i)
template <bool ADJ>
__global__ void k_M(const float2* __restrict__ Sin, float2* __restrict__ Sout, const float2* __restrict__ M, int n, int r) {
    int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    int col = blockIdx.y;
    if (e >= int64_t(n) * r) return;
    int o = int(e % r);
    int64_t p = e / r;
    const float2* x = Sin + int64_t(col) * n * r + p * r;
    const float2* m = M + p * r * r;
    float2 acc = make_float2(0.f, 0.f);
    if (!ADJ) {
        for (int j = 0; j < r; ++j) cfma(acc, m[o * r + j], x[j]);
    } else {
        for (int i = 0; i < r; ++i) cfmac(acc, m[i * r + o], x[i]);
    }
    Sout[int64_t(col) * n * r + e] = acc;
}

// Transfer factor on quads (warp per quad, r <= 16; lane = (half, index)).
//  MS ("mix, then scale"):  y[o][i] = sum_e Phi(o,e,i) sum_t Pc[o][i][t] x[e][t]
//        forward B (table E[q][o][e]) / adjoint C (conj F[q][e][o])
//  SM ("scale, then mix"):  y[o][j] = sum_e sum_t Pc[e][t][j] Phi(o,e,t) x[e][t]
//        forward C (table F[q][o][e]) / adjoint B (conj E[q][e][o])
//  Forward: inputs are the pairs (tau, 2b'+e) (adjacent), outputs (2tau+o, b').
//  Adjoint: the reverse.
template <bool MS, bool ADJ>
__global__ void k_quad(const float2* __restrict__ Sin, float2* __restrict__ Sout, const float2* __restrict__ T,
                       const float* __restrict__ Pc, int n, int L, int h, int s, int r) {
    // MS lanes read row i of Pc[o] across t, SM lanes read column j of Pc[e]
    // across t: store Pc so that the lanes of a warp hit consecutive banks
    // (MS: transposed, sPc[o][t][i]; SM: as is, sPc[e][t][j]).
    __shared__ float sPc[2 * kMaxR * kMaxR];
    __shared__ float2 sx[8][2 * kMaxR];
    __shared__ float2 sg[8][4 * kMaxR];
    for (int e = threadIdx.x; e < 2 * r * r; e += blockDim.x) {
        if (MS) {
            int c = e / (r * r), rem = e % (r * r), t = rem / r, i = rem % r;
            sPc[e] = Pc[(c * r + i) * r + t];
        } else {
            sPc[e] = Pc[e];
        }
    }
    __syncthreads();
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t q = int64_t(blockIdx.x) * 8 + w;
    int col = blockIdx.y;
    int64_t nquad = int64_t(n) / 2;
    if (q >= nquad) return;
    int64_t nbq = int64_t(1) << (L - s - 1);
    int64_t tau = q / nbq, bq = q % nbq;
    const float2* in = Sin + int64_t(col) * n * r;
    float2* out = Sout + int64_t(col) * n * r;
    int hl = lane >> 4, idx = lane & 15;
    bool act = idx < r;
    // pair indices
    int64_t pin, pout;
    if (!ADJ) {
        pin = tau * 2 * nbq + 2 * bq + hl;
        pout = (2 * tau + hl) * nbq + bq;
    } else {
        pin = (2 * tau + hl) * nbq + bq;
        pout = tau * 2 * nbq + 2 * bq + hl;
    }
    if (act) sx[w][hl * r + idx] = in[pin * r + idx];
    __syncwarp();
    // C levels (forward SM / adjoint MS) use the box-ordered F layout
    const int64_t qt = (MS == ADJ) ? fquad(tau, bq, h, s) : q;
    const float2* tq = T + qt * 4 * r;
    float2 y = make_float2(0.f, 0.f);
    if (MS) {
        // lane = (o = hl, i = idx)
        if (act) {
            const float* P = sPc + hl * r * r + idx;
            float2 h0 = make_float2(0.f, 0.f), h1 = make_float2(0.f, 0.f);
            for (int t = 0; t < r; ++t) {
                float pv = P[t * r];
                float2 x0 = sx[w][t], x1 = sx[w][r + t];
                h0.x = fmaf(pv, x0.x, h0.x); h0.y = fmaf(pv, x0.y, h0.y);
                h1.x = fmaf(pv, x1.x, h1.x); h1.y = fmaf(pv, x1.y, h1.y);
            }
            if (!ADJ) {
                cfma(y, tq[(hl * 2 + 0) * r + idx], h0);
                cfma(y, tq[(hl * 2 + 1) * r + idx], h1);
            } else {
                cfmac(y, tq[(0 * 2 + hl) * r + idx], h0);
                cfmac(y, tq[(1 * 2 + hl) * r + idx], h1);
            }
            out[pout * r + idx] = y;
        }
    } else {
        // g[o][e][t] = Phi(o,e,t) x[e][t]; lane (e = hl, t = idx) computes both o
        if (act) {
            float2 xv = sx[w][hl * r + idx];
            for (int o = 0; o < 2; ++o) {
                float2 g;
                if (!ADJ) g = cmul(tq[(o * 2 + hl) * r + idx], xv);
                else g = cmulc(tq[(hl * 2 + o) * r + idx], xv);
                sg[w][(o * 2 + hl) * r + idx] = g;
            }
        }
        __syncwarp();
        // lane = (o = hl, j = idx)
        if (act) {
            for (int e2 = 0; e2 < 2; ++e2) {
                const float* P = sPc + e2 * r * r;
                for (int t = 0; t < r; ++t) {
                    float pv = P[t * r + idx];
                    float2 g = sg[w][(hl * 2 + e2) * r + t];
                    y.x = fmaf(pv, g.x, y.x);
                    y.y = fmaf(pv, g.y, y.y);
                }
            }
            out[pout * r + idx] = y;
        }
    }
}

// ---------------------------------------------------------------- sampled entries (FP64)
// e^{2 pi i ph} in FP64.
__device__ __forceinline__ double2 expi2pi_d(double ph) {
    const double fr = ph - rint(ph);
    double sn, cs;
    sincospi(2.0 * fr, &sn, &cs);
    return make_double2(cs, sn);
}
__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// Lagrange polynomial l_k on the r Chebyshev points of a box, at the box coordinate v in [-1, 1].
__device__ double lag_d(const Cheb& ch, int r, int k, double v) {
    double p = 1.0;
    for (int m = 0; m < r; ++m)
        if (m != k) p *= (v - ch.t[m]) / (ch.t[k] - ch.t[m]);
    return p;
}

// One sampled entry (x_i, xi_j) per thread: K~(i, j) in FP64 straight from the factor entries of
// Eq. 2.1 (the interpolation functions of Section 2.2, not the stored FP32 tables) and the exact
// K(i, j) = a(x_i, xi_j) e^{2 pi i Phi(x_i, xi_j)}.  Only one chain of pairs couples x_i with
// xi_j -- at space level s the pair (tau = the box of level s holding x_i, sigma = the box of
// frequency level L - s holding xi_j) -- so the entry is a product of one r x r block per level:
// r coefficients carried from V through C, M and B to U.
__global__ void k_entry_chain(const int64_t* __restrict__ rows, const int64_t* __restrict__ cols, int S, PhaseDev ph,
                              AmpDev amp, Cheb ch, int n, int L, int h, int sU, int sV, int r, double2* __restrict__ out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= S) return;
    const int64_t i = rows[e], j = cols[e];
    const double x = double(i) / n, xi = double(j) - 0.5 * n;
    double2 c[kMaxR], d[kMaxR];
    auto fhalf = [&](int l) { return ldexp(double(n), -l - 1); };   // half width of a frequency box of level l
    {   // V at space level sV: c_t = e^{2 pi i (Phi(y, xi) - Phi(y, gamma_t))} q_t(xi)
        const int64_t tau = i >> (L - sV), sg = j >> sV;
        const int l = L - sV;
        const double y = space_center(sV, tau), fc = freq_center(n, l, sg);
        for (int t = 0; t < r; ++t) {
            const double g = freq_node(ch, n, l, sg, t);
            const double2 w = expi2pi_d(phi(ph, y, xi) - phi(ph, y, g));
            const double q = lag_d(ch, r, t, (xi - fc) / fhalf(l));
            c[t] = make_double2(w.x * q, w.y * q);
        }
    }
    for (int s = sV; s < h; ++s) {   // C, pair level s -> s+1
        const int64_t tau1 = i >> (L - s - 1), sg1 = j >> (s + 1), beta = j >> s;
        const double y1 = space_center(s + 1, tau1), fc1 = freq_center(n, L - s - 1, sg1);
        for (int jj = 0; jj < r; ++jj) {
            const double gj = freq_node(ch, n, L - s - 1, sg1, jj);
            double2 acc = make_double2(0.0, 0.0);
            for (int t = 0; t < r; ++t) {
                const double gb = freq_node(ch, n, L - s, beta, t);
                const double2 w = expi2pi_d(phi(ph, y1, gb) - phi(ph, y1, gj));
                const double q = lag_d(ch, r, jj, (gb - fc1) / fhalf(L - s - 1));
                const double2 v = zmul(w, c[t]);
                acc.x += q * v.x;
                acc.y += q * v.y;
            }
            d[jj] = acc;
        }
        for (int t = 0; t < r; ++t) c[t] = d[t];
    }
    {   // M at level h: d_i = sum_j a(z_i, gamma_j) e^{2 pi i Phi(z_i, gamma_j)} c_j
        const int64_t tau = i >> (L - h), sg = j >> h;
        for (int ii = 0; ii < r; ++ii) {
            const double z = space_node(ch, h, tau, ii);
            double2 acc = make_double2(0.0, 0.0);
            for (int t = 0; t < r; ++t) {
                const double g = freq_node(ch, n, L - h, sg, t);
                const double2 w = zmul(expi2pi_d(phi(ph, z, g)), c[t]);
                const double a = amp1d(amp, z, g);
                acc.x += a * w.x;
                acc.y += a * w.y;
            }
            d[ii] = acc;
        }
    }
    for (int s = h; s < sU; ++s) {   // B, pair level s -> s+1
        const int64_t al = i >> (L - s), tau1 = i >> (L - s - 1), beta = j >> s;
        const double eta = freq_center(n, L - s, beta), ya = space_center(s, al);
        for (int ii = 0; ii < r; ++ii) {
            const double z = space_node(ch, s + 1, tau1, ii);
            const double pz = ldexp(1.0, s + 1) * (z - ya);   // coordinate of z in the box of alpha
            double2 acc = make_double2(0.0, 0.0);
            for (int t = 0; t < r; ++t) {
                const double za = space_node(ch, s, al, t);
                const double2 w = zmul(expi2pi_d(phi(ph, z, eta) - phi(ph, za, eta)), d[t]);
                const double p = lag_d(ch, r, t, pz);
                acc.x += p * w.x;
                acc.y += p * w.y;
            }
            c[ii] = acc;
        }
        for (int t = 0; t < r; ++t) d[t] = c[t];
    }
    double2 y = make_double2(0.0, 0.0);
    {   // U at space level sU: y = sum_i e^{2 pi i (Phi(x, eta) - Phi(z_i, eta))} p_i(x) d_i
        const int64_t tau = i >> (L - sU), sg = j >> sU;
        const double eta = freq_center(n, L - sU, sg), px = ldexp(1.0, sU + 1) * (x - space_center(sU, tau));
        for (int t = 0; t < r; ++t) {
            const double z = space_node(ch, sU, tau, t);
            const double2 w = zmul(expi2pi_d(phi(ph, x, eta) - phi(ph, z, eta)), d[t]);
            const double p = lag_d(ch, r, t, px);
            y.x += p * w.x;
            y.y += p * w.y;
        }
    }
    const double2 k = expi2pi_d(phi(ph, x, xi));
    const double a = amp1d(amp, x, xi);
    out[2 * e] = y;
    out[2 * e + 1] = make_double2(a * k.x, a * k.y);
}

}  // namespace

// ---------------------------------------------------------------- host helpers
double lagrange_host(const double* t, int r, int k, double u) {
    double v = 1.0;
    for (int kk = 0; kk < r; ++kk)
        if (kk != k) v *= (u - t[kk]) / (t[k] - t[kk]);
    return v;
}

fio_status bf_apply_cols(const fio_bf* bf, const float2* X, float2* Y, int64_t ld, int kc, int adjoint,
                         float2* s0, float2* s1, cudaStream_t st) {
    const int n = bf->n, r = bf->r, L = bf->L;
    const float* P = bf->P.as<float>();
    const float* PV = P + bf->pv_off();
    const float* PU = P + bf->pu_off();
    const float* Pc = P + bf->pc_off();
    const int TB = 256;
    dim3 gNr(cdiv(int64_t(n) * r, TB), kc), gN(cdiv(n, TB), kc), gQ(cdiv(int64_t(n) / 2, 8), kc);
    size_t shV = size_t(bf->lsV) * r * sizeof(float), shU = size_t(bf->lsU) * r * sizeof(float);
    float2* a = s0;
    float2* b = s1;
    if (!adjoint) {
        FIO_LAUNCH("k_V_fwd", st, k_V_fwd<<<gNr, TB, shV, st>>>(X, ld, a, bf->VP.as<float2>(), PV, n, L, bf->sV, r));
        for (int s = bf->sV; s < bf->h; ++s) {
            FIO_LAUNCH("k_quad_C_fwd", st, k_quad<false, false><<<gQ, TB, 0, st>>>(a, b, bf->C[s - bf->sV].as<float2>(), Pc, n, L, bf->h, s, r));
            std::swap(a, b);
        }
        FIO_LAUNCH("k_M_fwd", st, k_M<false><<<gNr, TB, 0, st>>>(a, b, bf->M.as<float2>(), n, r));
        std::swap(a, b);
        for (int s = bf->h; s < bf->sU; ++s) {
            FIO_LAUNCH("k_quad_B_fwd", st, k_quad<true, false><<<gQ, TB, 0, st>>>(a, b, bf->B[s - bf->h].as<float2>(), Pc, n, L, bf->h, s, r));
            std::swap(a, b);
        }
        FIO_LAUNCH("k_U_fwd", st, k_U_fwd<<<gN, TB, shU, st>>>(a, Y, ld, bf->UP.as<float2>(), PU, n, L, bf->sU, r));
    } else {
        FIO_LAUNCH("k_U_adj", st, k_U_adj<<<gNr, TB, shU, st>>>(X, ld, a, bf->UP.as<float2>(), PU, n, L, bf->sU, r));
        for (int s = bf->sU - 1; s >= bf->h; --s) {
            FIO_LAUNCH("k_quad_B_adj", st, k_quad<false, true><<<gQ, TB, 0, st>>>(a, b, bf->B[s - bf->h].as<float2>(), Pc, n, L, bf->h, s, r));
            std::swap(a, b);
        }
        FIO_LAUNCH("k_M_adj", st, k_M<true><<<gNr, TB, 0, st>>>(a, b, bf->M.as<float2>(), n, r));
        std::swap(a, b);
        for (int s = bf->h - 1; s >= bf->sV; --s) {
            FIO_LAUNCH("k_quad_C_adj", st, k_quad<true, true><<<gQ, TB, 0, st>>>(a, b, bf->C[s - bf->sV].as<float2>(), Pc, n, L, bf->h, s, r));
            std::swap(a, b);
        }
        FIO_LAUNCH("k_V_adj", st, k_V_adj<<<gN, TB, shV, st>>>(a, Y, ld, bf->VP.as<float2>(), PV, n, L, bf->sV, r));
    }
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}

// Sampled entries of a 1D BF of rank r (K~ then K per sample, device double2[2 S]).
fio_status bf1d_entries(const fio_phase& phase, const AmpDev& amp, int n, int r, const int64_t* rows,
                        const int64_t* cols, int S, double2* out, cudaStream_t st) {
    const int L = ilog2_exact(n);
    const int h = L / 2, sU = std::max(L - 3, h), sV = std::min(3, h);
    Cheb ch{};
    for (int k = 0; k < r; ++k) ch.t[k] = std::cos((2.0 * k + 1.0) * M_PI / (2.0 * r));
    const PhaseDev ph{phase.kind, phase.s};
    FIO_LAUNCH("k_entry_chain", st,
               (k_entry_chain<<<cdiv(S, 64), 64, 0, st>>>(rows, cols, S, ph, amp, ch, n, L, h, sU, sV, r, out)));
    FIO_CUDA(cudaGetLastError());
    return FIO_OK;
}

}  // namespace fio

using namespace fio;

extern "C" fio_status bf_build(const fio_phase* phase, int n, int d, int r, void* stream, fio_bf** out) {
    return bf_build_amp(phase, nullptr, n, d, r, stream, out);
}

// The device form of an amplitude, checked against the dimension and phase it is used with.
static fio_status amp_dev(const fio_phase* phase, const fio_amp* amp, int n, int d, AmpDev& ad) {
    ad = AmpDev{};
    if (amp && amp->kind != FIO_AMP_ONE) {
        if (amp->kind == FIO_AMP_BUMPS) {
            if (d != 1) return fail(FIO_EINVAL, "bf_build_amp: the Gaussian-bump amplitude is 1D");
            if (amp->m < 1 || amp->m > FIO_AMP_MAX_BUMPS || !amp->centers || !(amp->sigma2 > 0.0))
                return fail(FIO_EINVAL, "bf_build_amp: bumps need 1 <= m <= FIO_AMP_MAX_BUMPS, centers and sigma2 > 0");
            ad.kind = FIO_AMP_BUMPS;
            ad.m = amp->m;
            ad.sigma2 = amp->sigma2;
            ad.N = double(n);
            for (int k = 0; k < 2 * amp->m; ++k) ad.c[k] = amp->centers[k];
        } else if (amp->kind == FIO_AMP_HANKEL) {
            if (d != 2 || phase->kind != FIO_PHASE_2D_ISO)
                return fail(FIO_EINVAL, "bf_build_amp: the Hankel amplitude needs d = 2 and FIO_PHASE_2D_ISO");
            ad.kind = FIO_AMP_HANKEL;
        } else {
            return fail(FIO_EINVAL, "bf_build_amp: unknown amplitude kind");
        }
    }
    return FIO_OK;
}

extern "C" fio_status bf_build_amp(const fio_phase* phase, const fio_amp* amp, int n, int d, int r, void* stream,
                                   fio_bf** out) {
    if (!out || !phase) return fail(FIO_EINVAL, "bf_build: null pointer");
    *out = nullptr;
    AmpDev ad;
    FIO_TRY(amp_dev(phase, amp, n, d, ad));
    if (d == 2) {
        const int L2 = ilog2_exact(n);
        if (L2 < 3 || L2 > 10) return fail(FIO_EINVAL, "bf_build: 2D needs n a power of two in [8, 1024]");
        int r1 = 1;
        while ((r1 + 1) * (r1 + 1) <= r) ++r1;
        if (r1 * r1 != r || !bf2d_ok_r1(r1))
            return fail(FIO_EINVAL, "bf_build: 2D needs r = r1^2 with 3 <= r1 <= 7 (r1 x r1 tensor Chebyshev grid)");
        if (!bf2d_ok_kind(phase->kind)) return fail(FIO_EINVAL, "bf_build: 2D phase must be DFT, 2D elliptic or 2D iso");
        fio_bf* bf = new fio_bf();
        bf->phase = *phase;
        bf->amp = ad;
        bf->nside = n; bf->n = n * n; bf->d = 2; bf->r = r; bf->L = L2;
        bf->h = L2 / 2;
        bf->sU = std::max(L2 - 3, bf->h);
        bf->sV = std::min(3, bf->h);
        fio_status s2 = bf2d_build(bf, as_stream(stream));
        if (s2 != FIO_OK) {
            bf_free(bf);
            return s2;
        }
        *out = bf;
        return FIO_OK;
    }
    if (d != 1) return fail(FIO_EINVAL, "bf_build: d must be 1 or 2");
    if (phase->kind == FIO_PHASE_2D_ELLIPTIC || phase->kind == FIO_PHASE_2D_ISO)
        return fail(FIO_EINVAL, "bf_build: that phase is 2D (d = 2)");
    int L = ilog2_exact(n);
    if (L < 4 || L > 24) return fail(FIO_EINVAL, "bf_build: n must be a power of two in [16, 2^24]");
    if (r < 1 || r > kMaxR) return fail(FIO_EINVAL, "bf_build: r must be in [1, 16]");
    if (phase->kind != FIO_PHASE_DFT && phase->kind != FIO_PHASE_1D_CABS && phase->kind != FIO_PHASE_1D_CABS8)
        return fail(FIO_EINVAL, "bf_build: unknown phase kind");
    cudaStream_t st = as_stream(stream);
    fio_bf* bf = new fio_bf();
    bf->phase = *phase;
    bf->amp = ad;
    bf->n = n; bf->nside = n; bf->d = d; bf->r = r; bf->L = L;
    bf->h = L / 2;
    bf->sU = std::max(L - 3, bf->h);
    bf->sV = std::min(3, bf->h);
    bf->lsV = 1 << bf->sV;
    bf->lsU = 1 << (L - bf->sU);
    for (int k = 0; k < 32; ++k) bf->tcheb[k] = k < r ? std::cos((2.0 * k + 1.0) * M_PI / (2.0 * r)) : 0.0;
    PhaseDev ph{phase->kind, phase->s};
    Cheb ch;
    std::memcpy(ch.t, bf->tcheb, sizeof(ch.t));
    auto cleanup = [&](fio_status s) { bf_free(bf); return s; };
    // real Lagrange tables
    std::vector<float> P(size_t(bf->lsV) * r + size_t(bf->lsU) * r + 2 * size_t(r) * r);
    for (int q = 0; q < bf->lsV; ++q)
        for (int j = 0; j < r; ++j) P[bf->pv_off() + q * r + j] = float(lagrange_host(bf->tcheb, r, j, 2.0 * q / bf->lsV - 1.0));
    for (int q = 0; q < bf->lsU; ++q)
        for (int i = 0; i < r; ++i) P[bf->pu_off() + q * r + i] = float(lagrange_host(bf->tcheb, r, i, 2.0 * q / bf->lsU - 1.0));
    for (int c = 0; c < 2; ++c)
        for (int i = 0; i < r; ++i)
            for (int t = 0; t < r; ++t)
                P[bf->pc_off() + (c * r + i) * r + t] = float(lagrange_host(bf->tcheb, r, t, (c - 0.5) + 0.5 * bf->tcheb[i]));
    fio_status s;
    if ((s = bf->P.ensure(P.size() * sizeof(float))) != FIO_OK) return cleanup(s);
    if (cudaMemcpyAsync(bf->P.p, P.data(), P.size() * sizeof(float), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return cleanup(cuda_status(cudaGetLastError(), "bf_build: copy of Lagrange tables"));
    const int TB = 256;
    int64_t nVP = (int64_t(1) << bf->sV) * n, nUP = int64_t(n) * bf->lsU;
    int64_t nM = int64_t(n) * r * r, nT = int64_t(n) / 2 * 4 * r;
    if ((s = bf->VP.ensure(nVP * 8)) != FIO_OK) return cleanup(s);
    if ((s = bf->UP.ensure(nUP * 8)) != FIO_OK) return cleanup(s);
    if ((s = bf->M.ensure(nM * 8)) != FIO_OK) return cleanup(s);
    k_tab_VP<<<cdiv(nVP, TB), TB, 0, st>>>(bf->VP.as<float2>(), ph, n, bf->sV);
    k_tab_UP<<<cdiv(nUP, TB), TB, 0, st>>>(bf->UP.as<float2>(), ph, n, L, bf->sU);
    k_tab_M<<<cdiv(nM, TB), TB, 0, st>>>(bf->M.as<float2>(), ph, bf->amp, ch, n, L, bf->h, r);
    bf->C.resize(bf->h - bf->sV);
    for (int lv = bf->sV; lv < bf->h; ++lv) {
        if ((s = bf->C[lv - bf->sV].ensure(nT * 8)) != FIO_OK) return cleanup(s);
        k_tab_F<<<cdiv(nT, TB), TB, 0, st>>>(bf->C[lv - bf->sV].as<float2>(), ph, ch, n, L, bf->h, lv, r);
    }
    bf->B.resize(bf->sU - bf->h);
    for (int lv = bf->h; lv < bf->sU; ++lv) {
        if ((s = bf->B[lv - bf->h].ensure(nT * 8)) != FIO_OK) return cleanup(s);
        k_tab_E<<<cdiv(nT, TB), TB, 0, st>>>(bf->B[lv - bf->h].as<float2>(), ph, ch, n, L, lv, r);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cleanup(cuda_status(e, "bf_build: table kernels"));
    bf->table_bytes = (nVP + nUP + nM + nT * int64_t(bf->C.size() + bf->B.size())) * 8 + int64_t(P.size()) * 4;
    if ((s = bf_prestage(bf, st)) != FIO_OK) return cleanup(s);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cleanup(cuda_status(e, "bf_build: staged tables"));
    *out = bf;
    return FIO_OK;
}

namespace fio {
fio_status bf_apply_ord(const fio_bf* bfc, const float2* X, float2* Y, int64_t ld, int k, int adjoint, bool morton,
                        cudaStream_t st, int prec) {
    if (!bfc) return fail(FIO_EINVAL, "bf_apply: null handle");
    if (bfc->d == 1) return bf_apply_prec(bfc, X, Y, ld, k, adjoint, prec, st);
    fio_bf* bf = const_cast<fio_bf*>(bfc);   // the 2D path only grows the handle's scratch
    if (k < 0 || ld < bf->n) return fail(FIO_EINVAL, "bf_apply: need k >= 0 and ld >= N");
    if (k == 0) return FIO_OK;
    if (!X || !Y) return fail(FIO_EINVAL, "bf_apply: null vector");
    const int64_t stateN = int64_t(bf->n) * bf->r;
    const int kc = int(std::min<int64_t>(k, std::max<int64_t>(1, std::min<int64_t>(32, (int64_t(1) << 30) / (2 * stateN * 8)))));
    FIO_TRY(bf->ws.ensure(size_t(2) * stateN * kc * 8));
    float2* s0 = bf->ws.as<float2>();
    float2* s1 = s0 + stateN * kc;
    for (int c0 = 0; c0 < k; c0 += kc) {
        const int cc = std::min(kc, k - c0);
        FIO_TRY(bf2d_apply_cols(bf, X + c0 * ld, Y + c0 * ld, ld, cc, adjoint, morton, s0, s1, st));
    }
    return FIO_OK;
}
}  // namespace fio

namespace fio {
// bf_apply with an explicit precision request (-1: the handle's setting); the handle's
// settings are not modified, only its scratch grows.
fio_status bf_apply_prec(const fio_bf* bfc, const float2* X, float2* Y, int64_t ld, int k, int adjoint, int prec,
                         cudaStream_t st) {
    if (!bfc) return fail(FIO_EINVAL, "bf_apply: null handle");
    if (k < 0 || ld < bfc->n) return fail(FIO_EINVAL, "bf_apply: need k >= 0 and ld >= N");
    if (k == 0) return FIO_OK;
    if (!X || !Y) return fail(FIO_EINVAL, "bf_apply: null vector");
    if (bfc->d == 2) return bf_apply_ord(bfc, X, Y, ld, k, adjoint, false, st, prec);
    fio_bf* bf = const_cast<fio_bf*>(bfc);
    const bool split = prec < 0 ? bf->split : prec == 1;
    const int64_t stateN = int64_t(bf->n) * bf->r;
    const bool fused = bf_fused_ok(bf) && (!bf->force_unfused || split);
    // column chunk: at most 64 columns or 1 GiB of state, whichever is smaller
    const int nstate = fused ? 1 : 2;
    int kc = int(std::min<int64_t>(k, std::max<int64_t>(1, std::min<int64_t>(64, (int64_t(1) << 30) / (nstate * stateN * 8)))));
    FIO_TRY(bf->ws.ensure(size_t(nstate) * stateN * kc * 8));
    float2* s0 = bf->ws.as<float2>();
    float2* s1 = s0 + stateN * kc;
    for (int c0 = 0; c0 < k; c0 += kc) {
        int cc = std::min(kc, k - c0);
        const float2* Xc = X + c0 * ld;
        float2* Yc = Y + c0 * ld;
        if (fused) FIO_TRY(bf_apply_fused(bf, Xc, Yc, ld, cc, adjoint, s0, st, prec));
        else FIO_TRY(bf_apply_cols(bf, Xc, Yc, ld, cc, adjoint, s0, s1, st));
    }
    return FIO_OK;
}
}  // namespace fio

// ---------------------------------------------------------------- sampled entries, adaptive rank
namespace {
// Entries (rows[e], cols[e]) of the BF of rank r (FP64 chain) and of K, to the host.
fio_status entries_host(const fio_phase& phase, const AmpDev& ad, int nside, int d, int r, const int64_t* rows,
                        const int64_t* cols, int S, cudaStream_t st, std::vector<double2>& out) {
    if (!rows || !cols) return fail(FIO_EINVAL, "bf_entries: null index array");
    if (S < 1 || S > (1 << 22)) return fail(FIO_EINVAL, "bf_entries: need 1 <= S <= 2^22 samples");
    const int64_t N = d == 2 ? int64_t(nside) * nside : int64_t(nside);
    for (int e = 0; e < S; ++e)
        if (rows[e] < 0 || rows[e] >= N || cols[e] < 0 || cols[e] >= N)
            return fail(FIO_EINVAL, "bf_entries: index out of range");
    DevBuf buf;
    fio_status s = buf.ensure(size_t(S) * (2 * sizeof(int64_t) + 2 * sizeof(double2)));
    if (s != FIO_OK) return s;
    int64_t* drows = buf.as<int64_t>();
    int64_t* dcols = drows + S;
    double2* dout = reinterpret_cast<double2*>(dcols + S);
    out.assign(size_t(2) * S, make_double2(0.0, 0.0));
    cudaError_t e = cudaMemcpyAsync(drows, rows, size_t(S) * sizeof(int64_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dcols, cols, size_t(S) * sizeof(int64_t), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
        buf.release();
        return cuda_status(e, "bf_entries: index copy");
    }
    if (d == 2) {
        int r1 = 1;
        while ((r1 + 1) * (r1 + 1) <= r) ++r1;
        s = bf2d_entries(phase, ad.kind, nside, r1, drows, dcols, S, dout, st);
    } else {
        s = bf1d_entries(phase, ad, nside, r, drows, dcols, S, dout, st);
    }
    if (s == FIO_OK) {
        e = cudaMemcpyAsync(out.data(), dout, size_t(2) * S * sizeof(double2), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = cuda_status(e, "bf_entries");
    }
    buf.release();
    return s;
}

// sqrt(sum |K~ - K|^2 / sum |K|^2) over the samples
fio_status entry_error(const std::vector<double2>& v, double* err) {
    double num = 0.0, den = 0.0;
    for (size_t e = 0; e + 1 < v.size(); e += 2) {
        const double dr = v[e].x - v[e + 1].x, di = v[e].y - v[e + 1].y;
        num += dr * dr + di * di;
        den += v[e + 1].x * v[e + 1].x + v[e + 1].y * v[e + 1].y;
    }
    if (!(den > 0.0)) return fail(FIO_EINVAL, "bf_entry_error: no sample with a finite nonzero entry of K");
    *err = std::sqrt(num / den);
    return FIO_OK;
}

fio_status check_geometry(const fio_phase* phase, int n, int d, int r) {
    if (!phase) return fail(FIO_EINVAL, "null phase");
    if (d == 2) {
        const int L2 = ilog2_exact(n);
        int r1 = 1;
        while ((r1 + 1) * (r1 + 1) <= r) ++r1;
        if (L2 < 3 || L2 > 10 || r1 * r1 != r || !bf2d_ok_r1(r1) || !bf2d_ok_kind(phase->kind))
            return fail(FIO_EINVAL, "2D needs n = 2^3..2^10, r = r1^2 with 3 <= r1 <= 7 and a 2D phase");
        return FIO_OK;
    }
    if (d != 1) return fail(FIO_EINVAL, "d must be 1 or 2");
    const int L = ilog2_exact(n);
    if (L < 4 || L > 24 || r < 1 || r > kMaxR) return fail(FIO_EINVAL, "1D needs n = 2^4..2^24 and 1 <= r <= 16");
    if (phase->kind != FIO_PHASE_DFT && phase->kind != FIO_PHASE_1D_CABS && phase->kind != FIO_PHASE_1D_CABS8)
        return fail(FIO_EINVAL, "1D needs a 1D phase");
    return FIO_OK;
}
}  // namespace

extern "C" fio_status bf_entries(const fio_bf* bf, const int64_t* rows, const int64_t* cols, int S, void* stream,
                                 double* out) {
    if (!bf || !out) return fail(FIO_EINVAL, "bf_entries: null pointer");
    std::vector<double2> v;
    FIO_TRY(entries_host(bf->phase, bf->amp, bf->nside, bf->d, bf->r, rows, cols, S, as_stream(stream), v));
    std::memcpy(out, v.data(), v.size() * sizeof(double2));
    return FIO_OK;
}

extern "C" fio_status bf_entry_error(const fio_phase* phase, const fio_amp* amp, int n, int d, int r,
                                     const int64_t* rows, const int64_t* cols, int S, void* stream, double* err) {
    if (!err) return fail(FIO_EINVAL, "bf_entry_error: null pointer");
    FIO_TRY(check_geometry(phase, n, d, r));
    AmpDev ad;
    FIO_TRY(amp_dev(phase, amp, n, d, ad));
    std::vector<double2> v;
    FIO_TRY(entries_host(*phase, ad, n, d, r, rows, cols, S, as_stream(stream), v));
    return entry_error(v, err);
}

extern "C" fio_status bf_build_tol(const fio_phase* phase, const fio_amp* amp, int n, int d, double tol,
                                   const int64_t* rows, const int64_t* cols, int S, void* stream, fio_bf** out,
                                   int* r_out, double* err_out) {
    if (!out || !phase) return fail(FIO_EINVAL, "bf_build_tol: null pointer");
    *out = nullptr;
    if (!(tol > 0.0)) return fail(FIO_EINVAL, "bf_build_tol: tol must be positive");
    std::vector<int> cand;
    if (d == 2)
        for (int r1 = 3; r1 <= 7; ++r1) cand.push_back(r1 * r1);
    else
        for (int r = 4; r <= kMaxR; r += 2) cand.push_back(r);
    AmpDev ad;
    FIO_TRY(amp_dev(phase, amp, n, d, ad));
    int r_pick = cand.back();
    double e_pick = 0.0;
    for (size_t c = 0; c < cand.size(); ++c) {
        FIO_TRY(check_geometry(phase, n, d, cand[c]));
        std::vector<double2> v;
        FIO_TRY(entries_host(*phase, ad, n, d, cand[c], rows, cols, S, as_stream(stream), v));
        double e = 0.0;
        FIO_TRY(entry_error(v, &e));
        r_pick = cand[c];
        e_pick = e;
        if (e <= tol) break;
    }
    if (r_out) *r_out = r_pick;
    if (err_out) *err_out = e_pick;
    return bf_build_amp(phase, amp, n, d, r_pick, stream, out);
}

extern "C" fio_status bf_apply(fio_bf* bf, const void* X, void* Y, int64_t ld, int k, int adjoint, void* stream) {
    return bf_apply_prec(bf, static_cast<const float2*>(X), static_cast<float2*>(Y), ld, k, adjoint, -1,
                         as_stream(stream));
}

extern "C" fio_status bf_set_path(fio_bf* bf, int path) {
    if (!bf || path < 0 || path > 4) return fail(FIO_EINVAL, "bf_set_path: bad handle or path");
    if (bf->d == 2 && path >= 2) return fail(FIO_EINVAL, "bf_set_path: 2D handles run the per-level kernels only");
    if (path >= 2 && !bf_fused_ok(bf)) return fail(FIO_EINVAL, "bf_set_path: fused apply needs r = 16 and n >= 64");
    if (path == 4 && !bf_v3_ok(bf)) return fail(FIO_EINVAL, "bf_set_path: staged fused kernels need 2^12 <= n <= 2^18");
    bf->force_unfused = (path == 1);
    bf->fused_v2 = (path == 3);
    bf->simt = (path == 4);
    return FIO_OK;
}

extern "C" fio_status fio_device_status(void) {
    const int v1 = tc_wait_timeouts(), v2 = ulv_tc_timeouts();
    if (v1 < 0 || v2 < 0) return fail(FIO_ECUDA, "fio_device_status: reading the device flag failed");
    const int v = v1 | v2;
    if (v > 0) return fail(FIO_ETIMEOUT, "a bounded wait of a tensor-core kernel ran out (results of that launch are invalid)");
    return FIO_OK;
}

extern "C" fio_status bf_set_precision(fio_bf* bf, int precision) {
    if (!bf || precision < 0 || precision > 1) return fail(FIO_EINVAL, "bf_set_precision: bad handle or precision");
    if (precision == 1 && !bf_v3_ok(bf))
        return fail(FIO_EINVAL, "bf_set_precision: split BF16 needs r = 16 and 2^12 <= n <= 2^18");
    bf->split = (precision == 1);
    return FIO_OK;
}

extern "C" fio_status bf_info(const fio_bf* bf, int64_t* o) {
    if (!bf || !o) return fail(FIO_EINVAL, "bf_info: null pointer");
    o[0] = bf->n; o[1] = bf->d; o[2] = bf->r; o[3] = bf->L; o[4] = bf->h; o[5] = bf->sU; o[6] = bf->sV;
    o[7] = bf->table_bytes;
    return FIO_OK;
}

extern "C" void bf_free(fio_bf* bf) {
    if (!bf) return;
    bf->VP.release(); bf->UP.release(); bf->M.release(); bf->P.release(); bf->ws.release();
    for (auto& b : bf->C) b.release();
    for (auto& b : bf->B) b.release();
    bf->Mst.release();
    for (int d = 0; d < 2; ++d) {
        for (auto& b : bf->Cst[d]) b.release();
        for (auto& b : bf->Bst[d]) b.release();
    }
    delete bf;
}
