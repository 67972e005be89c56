// Preconditioned conjugate gradients on the approximate normal equation
// (Section 4.1, Eq. 4.3):  K~^* K~ f = K~^* u, preconditioned by the ULV
// factorization F~ = G~^{-1} of the HSS approximation.  Every column of the
// block is an independent CG run (f_0 = 0, stop when the recurrence residual
// satisfies ||r_k|| <= tol ||K~^* u||); the columns share the operator
// applies, which run on the whole block.  Vectors are complex64 (the
// precision of the applies and the ULV solve); inner products and the CG
// scalars are accumulated and kept in FP64 on the device.
#include <algorithm>
#include <cmath>

#include "bf.cuh"
#include "hss.cuh"

namespace fio {
namespace {

constexpr int TB = 256;

__device__ __forceinline__ double2 block_sum2(double2 v, double2* sh) {
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    double2 s = make_double2(0.0, 0.0);
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : make_double2(0.0, 0.0);
        for (int o = 16; o > 0; o >>= 1) {
            s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
            s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
        }
    }
    return s;
}

// out[c] += sum_i conj(a[c][i]) b[c][i]   (grid: (blocks, k); out zeroed beforehand)
__global__ void k_cdot(const float2* __restrict__ a, const float2* __restrict__ b, int64_t n, int64_t ld,
                       double2* __restrict__ out) {
    __shared__ double2 sh[TB / 32];
    const int c = blockIdx.y;
    double2 acc = make_double2(0.0, 0.0);
    for (int64_t i = int64_t(blockIdx.x) * TB + threadIdx.x; i < n; i += int64_t(gridDim.x) * TB) {
        const float2 x = a[c * ld + i], y = b[c * ld + i];
        acc.x += double(x.x) * y.x + double(x.y) * y.y;
        acc.y += double(x.x) * y.y - double(x.y) * y.x;
    }
    const double2 s = block_sum2(acc, sh);
    if (threadIdx.x == 0) {
        atomicAdd(&out[c].x, s.x);
        atomicAdd(&out[c].y, s.y);
    }
}

// alpha = rz / pq for active columns, 0 otherwise
__global__ void k_alpha(const double2* rz, const double2* pq, const int* active, double2* alpha, int k) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= k) return;
    if (!active[c]) {
        alpha[c] = make_double2(0.0, 0.0);
        return;
    }
    const double2 a = rz[c], b = pq[c];
    const double d = b.x * b.x + b.y * b.y;
    alpha[c] = d > 0.0 ? make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d) : make_double2(0.0, 0.0);
}

// x += alpha p ; r -= alpha q
__global__ void k_update_xr(float2* __restrict__ x, float2* __restrict__ r, const float2* __restrict__ p,
                            const float2* __restrict__ q, const double2* __restrict__ alpha, int64_t n, int64_t ld) {
    const int c = blockIdx.y;
    const int64_t i = int64_t(blockIdx.x) * TB + threadIdx.x;
    if (i >= n) return;
    const double2 a = alpha[c];
    if (a.x == 0.0 && a.y == 0.0) return;
    const float2 pv = p[c * ld + i], qv = q[c * ld + i];
    float2 xv = x[c * ld + i], rv = r[c * ld + i];
    xv.x += float(a.x * pv.x - a.y * pv.y);
    xv.y += float(a.x * pv.y + a.y * pv.x);
    rv.x -= float(a.x * qv.x - a.y * qv.y);
    rv.y -= float(a.x * qv.y + a.y * qv.x);
    x[c * ld + i] = xv;
    r[c * ld + i] = rv;
}

// beta = rz_new / rz (active columns); p = z + beta p; rz = rz_new
__global__ void k_beta(double2* rz, const double2* rz_new, const int* active, double2* beta, int k) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= k) return;
    const double2 a = rz_new[c], b = rz[c];
    const double d = b.x * b.x + b.y * b.y;
    beta[c] = (active[c] && d > 0.0) ? make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d)
                                     : make_double2(0.0, 0.0);
    if (active[c]) rz[c] = a;
}
__global__ void k_update_p(float2* __restrict__ p, const float2* __restrict__ z, const double2* __restrict__ beta,
                           const int* __restrict__ active, int64_t n, int64_t ld) {
    const int c = blockIdx.y;
    const int64_t i = int64_t(blockIdx.x) * TB + threadIdx.x;
    if (i >= n || !active[c]) return;
    const double2 b = beta[c];
    const float2 zv = z[c * ld + i], pv = p[c * ld + i];
    p[c * ld + i] = make_float2(float(zv.x + b.x * pv.x - b.y * pv.y), float(zv.y + b.x * pv.y + b.y * pv.x));
}

fio_status cdot(const float2* a, const float2* b, int64_t n, int64_t ld, int k, double2* out, cudaStream_t st) {
    FIO_CUDA(cudaMemsetAsync(out, 0, sizeof(double2) * k, st));
    const unsigned nb = unsigned(std::min<int64_t>(cdiv(n, TB), 148 * 4));
    FIO_LAUNCH("k_cdot", st, k_cdot<<<dim3(nb, k), TB, 0, st>>>(a, b, n, ld, out));
    return FIO_OK;
}

}  // namespace
}  // namespace fio

using namespace fio;

extern "C" fio_status fio_pcg(const fio_bf* bf, const fio_hss* hc, const void* U, void* F, int64_t ld, int k,
                              double tol, int maxit, int* iters, double* relres, void* stream) {
    if (!bf || !hc) return fail(FIO_EINVAL, "fio_pcg: null handle");
    if (bf->N() != hc->N) return fail(FIO_EINVAL, "fio_pcg: BF and HSS sizes differ");
    if (k < 0 || ld < hc->N || maxit < 0 || !(tol >= 0.0)) return fail(FIO_EINVAL, "fio_pcg: bad k, ld, tol or maxit");
    if (!hc->factored) return fail(FIO_EINVAL, "fio_pcg: the HSS has no ULV factorization (hss_ulv_factor)");
    if (iters) *iters = 0;
    if (k == 0) return FIO_OK;
    if (!U || !F) return fail(FIO_EINVAL, "fio_pcg: null vector");
    fio_hss* h = const_cast<fio_hss*>(hc);
    cudaStream_t st = as_stream(stream);
    const int64_t N = h->N;
    const bool mort = bf->d == 2;   // 2D: the iteration runs in quadtree order (the HSS order)
    // workspace: X (Morton solution, 2D only), R, Z, P, Q, T, then the scalars
    const int nvec = 5 + (mort ? 1 : 0);
    const size_t vec_bytes = size_t(nvec) * ld * k * 8;
    const size_t scal_bytes = size_t(k) * (6 * sizeof(double2) + sizeof(double) + sizeof(int)) + 256;
    FIO_TRY(h->fio_ws.ensure(vec_bytes + scal_bytes));
    float2* R = h->fio_ws.as<float2>();
    float2* Z = R + ld * k;
    float2* P = Z + ld * k;
    float2* Q = P + ld * k;
    float2* T = Q + ld * k;
    float2* X = mort ? T + ld * k : static_cast<float2*>(F);
    double2* rz = reinterpret_cast<double2*>(reinterpret_cast<char*>(h->fio_ws.p) + vec_bytes);
    double2* rz_new = rz + k;
    double2* pq = rz_new + k;
    double2* alpha = pq + k;
    double2* beta = alpha + k;
    double2* nrm = beta + k;   // .x: ||r||^2 (from <r, r>)
    int* active = reinterpret_cast<int*>(nrm + k);
    const dim3 gv(cdiv(N, TB), k);

    // b = K~^* u (held in R: r_0 = b since f_0 = 0)
    FIO_TRY(bf_apply_ord(bf, static_cast<const float2*>(U), R, ld, k, 1, mort, st));
    FIO_CUDA(cudaMemsetAsync(X, 0, size_t(ld) * k * 8, st));
    FIO_TRY(cdot(R, R, N, ld, k, nrm, st));
    std::vector<double2> hb(k), hn(k);
    FIO_CUDA(cudaMemcpyAsync(hb.data(), nrm, sizeof(double2) * k, cudaMemcpyDeviceToHost, st));
    FIO_CUDA(cudaStreamSynchronize(st));
    std::vector<int> act(k);
    std::vector<double> rel(k, 0.0);
    int nact = 0;
    for (int c = 0; c < k; ++c) {
        act[c] = hb[c].x > 0.0 ? 1 : 0;
        nact += act[c];
    }
    FIO_CUDA(cudaMemcpyAsync(active, act.data(), sizeof(int) * k, cudaMemcpyHostToDevice, st));
    FIO_TRY(hss_solve(h, R, Z, ld, k, st));                       // z_0 = M r_0
    FIO_CUDA(cudaMemcpyAsync(P, Z, size_t(ld) * k * 8, cudaMemcpyDeviceToDevice, st));
    FIO_TRY(cdot(R, Z, N, ld, k, rz, st));
    int it = 0;
    while (nact > 0 && it < maxit) {
        FIO_TRY(bf_apply_ord(bf, P, T, ld, k, 0, mort, st));      // K~ p
        FIO_TRY(bf_apply_ord(bf, T, Q, ld, k, 1, mort, st));      // q = K~^* K~ p
        FIO_TRY(cdot(P, Q, N, ld, k, pq, st));
        FIO_LAUNCH("k_alpha", st, k_alpha<<<cdiv(k, 128), 128, 0, st>>>(rz, pq, active, alpha, k));
        FIO_LAUNCH("k_update_xr", st, k_update_xr<<<gv, TB, 0, st>>>(X, R, P, Q, alpha, N, ld));
        ++it;
        FIO_TRY(cdot(R, R, N, ld, k, nrm, st));
        FIO_CUDA(cudaMemcpyAsync(hn.data(), nrm, sizeof(double2) * k, cudaMemcpyDeviceToHost, st));
        FIO_CUDA(cudaStreamSynchronize(st));
        nact = 0;
        for (int c = 0; c < k; ++c) {
            if (!act[c]) continue;
            rel[c] = std::sqrt(std::max(hn[c].x, 0.0) / hb[c].x);
            act[c] = rel[c] > tol ? 1 : 0;
            nact += act[c];
        }
        if (nact == 0 || it >= maxit) break;
        FIO_CUDA(cudaMemcpyAsync(active, act.data(), sizeof(int) * k, cudaMemcpyHostToDevice, st));
        FIO_TRY(hss_solve(h, R, Z, ld, k, st));                   // z = M r
        FIO_TRY(cdot(R, Z, N, ld, k, rz_new, st));
        FIO_LAUNCH("k_beta", st, k_beta<<<cdiv(k, 128), 128, 0, st>>>(rz, rz_new, active, beta, k));
        FIO_LAUNCH("k_update_p", st, k_update_p<<<gv, TB, 0, st>>>(P, Z, beta, active, N, ld));
    }
    if (mort) FIO_TRY(bf2d_unmorton(bf, X, static_cast<float2*>(F), ld, k, st));
    FIO_CUDA(cudaGetLastError());
    if (iters) *iters = it;
    if (relres)
        for (int c = 0; c < k; ++c) relres[c] = rel[c];
    return FIO_OK;
}
