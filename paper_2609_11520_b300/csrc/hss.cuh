// HSS handle (Def. 2.1-2.2) with one rank per level, and its ULV factors
// (Section 2.4).  All generator blocks are complex64, column-major,
// node-major within a level.
#pragma once
#include "common.cuh"

struct fio_hss {
    int64_t N = 0;
    int leaf = 0, Lh = 0;
    std::vector<int> ranks;          // r_l, l = 0..Lh (r_0 = 0)
    std::vector<fio::DevBuf> U;      // U[l], l = 1..Lh: 2^l blocks m_l x r_l
    std::vector<fio::DevBuf> B;      // B[l], l = 0..Lh-1: 2^l blocks r_{l+1} x r_{l+1}
    fio::DevBuf D;                   // 2^Lh blocks leaf x leaf
    // ULV factors: W[l] (2^l blocks m_l x m_l, complex64), root inverse
    bool factored = false;
    std::vector<fio::DevBuf> W;
    std::vector<fio::DevBuf> Wmx;    // per level (32 <= m_l <= 512): largest |Re|, |Im| of each row of W_t, then of W_t^*
    fio::DevBuf Rinv;                // m_0 x m_0 (complex64)
    fio::DevBuf solve_ws;            // per-level vectors of the solve
    fio::DevBuf solve_part;          // partial products of the sliced wide node products
    int solve_path = 0;              // 0: node products on the CUDA cores; 1: tensor cores where they apply
    fio::DevBuf mv_ws;               // per-level vectors of the matvec
    fio::DevBuf fio_ws;              // K~^* u and refinement vectors of fio_solve
    int64_t samples = 0;
    int m(int l) const { return l == Lh ? leaf : 2 * ranks[l + 1]; }
    int64_t rows(int l) const { return (int64_t(1) << l) * m(l); }   // sum of m over level l
    int64_t rrows(int l) const { return (int64_t(1) << l) * ranks[l]; }
};

namespace fio {
// hss_solve with the precision of the tensor-core node products (0: FP16 parts, 1: BF16 parts).
fio_status hss_solve_prec(const fio_hss* h, const void* B, void* X, int64_t ld, int k, int prec, cudaStream_t st);
// Whether a bounded wait of a tensor-core ULV kernel ran out since the last call (cleared); -1 on error.
int ulv_tc_timeouts();
// Large nodes (dense64.cu): levels with at most 16 nodes of size m >= the
// threshold (default 384, fio_set_large_node) run level-3 formulations in mixed
// precision: FP32 bulk products of the node pass, postprocessing and ULV when the
// HSS tolerance is >= 1e-4 (FP64 node pass below it); FP64 Gram matrix and pivoted
// Cholesky of the rank-revealing step, root, eliminated-block Cholesky and merge.
struct BigScratch;
BigScratch* big_scratch_new();
void big_scratch_free(BigScratch* b);
void set_large_node_min(int m);
bool large_level(int nodes, int m);
fio_status big_level_nodes(BigScratch& w, int nn, int m, int s, int rhat, const float2* Om, const float2* Y, int64_t ld,
                           double tol, std::vector<int>& hk, std::vector<int>& hs, cudaStream_t st);
fio_status big_level_finish(BigScratch& w, int nn, int m, int rl, float2* Uout, float2* Dchk, cudaStream_t st);
fio_status big_root(BigScratch& w, int m0, int s0, const float2* Om, const float2* Y, double2* D0, cudaStream_t st);
fio_status big_post(BigScratch& w, int nn, int rc, int mc, double2* Dcur, const float2* Uc, const float2* Dchk,
                    float2* Bout, double2* Dnext, cudaStream_t st);
fio_status big_ulv_nodes(BigScratch& b, int nn, int m, int r, const double2* D, const double2* U, float2* Wout,
                         double2* Dh22, double2* Uh2, int* d_status, cudaStream_t st);
template <class C>
fio_status ulv_merge_gemm(BigScratch& b, int np, int r, const C* Dh22, const C* Uh2, const float2* B, const float2* Up,
                          int rp, C* Dplus, C* Uplus, cudaStream_t st);
fio_status big_ulv_root(BigScratch& b, int m0, const double2* Dp, float2* Rinv, int* d_status, cudaStream_t st);

// Block products over the nodes of level l (column-major vectors, ld = rows):
//   expand:   out[t*m + i] (+)= sum_c U_t[i][c] in[t*r + c]
//   compress: out[t*r + c]  = sum_i conj(U_t[i][c]) in[t*m + i]
void launch_expand(const float2* U, int nodes, int m, int r, const float2* in, int64_t ldin, float2* out,
                   int64_t ldout, int k, bool accumulate, cudaStream_t st);
void launch_compress(const float2* U, int nodes, int m, int r, const float2* in, int64_t ldin, float2* out,
                     int64_t ldout, int k, cudaStream_t st);

// The ULV solve as data: per level one node-product descriptor for the up
// pass and one for the down pass, and the root product.
struct UlvGemmDesc {
    const float2* W;
    const float2* inA;
    const float2* inB;
    float2* outC;
    float2* outD;
    int64_t ldA, ldB, ldC, ldD;
    int m, nA, nC, k, nodes;
};
// One item of the persistent batched solve: type (kP*), payload (a, b, c, d), for ULV node
// products a second block (a, b2, c2, d2) of the same stage run by the other half of the CTA
// (b2 < 0: none), the counter it waits on (dep, -1 for none) until it reaches `target`, and the
// counter it increments.
enum { kPLeft = 0, kPRight = 1, kPUp = 2, kPRoot = 3, kPDown = 4 };
struct PItem {
    int type, a, b, c, d;
    int b2, c2, d2;
    int dep, target, done, pad;
};
struct UlvRootDesc {
    const float2* A;   // m x m
    const float2* x;   // m x k (ld m)
    float2* y;
    int m, k;
};
struct UlvSolvePlan {
    int Lh = 0;
    std::vector<UlvGemmDesc> up, down;   // index = level l (1..Lh)
    UlvRootDesc root{};
};
int64_t ulv_solve_ws_elems(const fio_hss* h, int k);
fio_status ulv_solve_plan(fio_hss* h, const float2* B, float2* X, int64_t ld, int k, float2* ws, UlvSolvePlan& plan);
void ulv_gemm_items(const UlvGemmDesc& d, int di, std::vector<int4>& items);
fio_status ulv_group_launch(const UlvGemmDesc* dd, const int4* ditems, int nitems, bool down, cudaStream_t st);
fio_status ulv_root_group_launch(const UlvRootDesc* dd, int n, cudaStream_t st);
// The persistent batched solve (bf_fused.cu): one launch over the work list `items`;
// head_and_counters: 1 + ncounters ints (zeroed here), mode: transfer-level mode of the BF items.
fio_status batch_persistent_launch(const void* dleft_args, const void* dright_args, const UlvGemmDesc* udesc,
                                   const UlvRootDesc* rdesc, const PItem* items, int nitems, int* head_and_counters,
                                   int ncounters, int mode, int spin_limit, cudaStream_t st);
}
