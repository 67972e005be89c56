// Butterfly factorization handle (Section 2.2, Eq. 2.1), device-resident.
//
// The factors are stored in a phase-folded factored form that is
// mathematically identical to Eq. 2.1.  Every transfer block of Eq. 2.4-2.6
// is  diag(phase) * P * diag(phase)  with P a real Lagrange matrix shared by
// all boxes of a level (dyadic boxes are scaled copies of each other).  The
// two diagonal phases of consecutive factors are merged into one table per
// level, so that the coefficient state between stages is expressed in
// "demodulated" bases:
//   c^(s)(tau,sigma,j)  stored as  e^{+2 pi i Phi(y_tau, gamma_sigma_j)} c   (right side)
//   d^(s)(tau,sigma,i)  stored as  e^{-2 pi i Phi(z_tau_i, eta_sigma)} d     (left side)
// Tables (complex64):
//   VP[a][j]        e^{2 pi i Phi(y_a, xi_j)}            a: space box of level sV
//   F_s[q][c][b][t] e^{2 pi i (Phi(y_tau', gamma_bt) - Phi(y_tau, gamma_bt))}   C level s
//                   (quads ordered by the frequency box of level L-h that holds them)
//   M[p][i][j]      e^{2 pi i (Phi(z_i, gamma_j) - Phi(z_i, eta) - Phi(y, gamma_j))}
//   E_s[q][c][b][i] e^{2 pi i (Phi(z_tau_i, eta_beta) - Phi(z_tau_i, eta_sigma))} B level s
//   UP[x][b]        e^{2 pi i Phi(x, eta_b)}              b: frequency box of level L-sU
// and real tables PV[q][j], PU[q][i] (Lagrange basis at the leaf points) and
// Pc[c][i][t] = l_t((c - 1/2) + t_i / 2) (parent basis at the child nodes).
// A "quad" q = (space box at level s, frequency box b' at level L-s-1)
// couples the two input pairs (tau, 2b'+e) with the two output pairs
// (2 tau + o, b').
#pragma once
#include "common.cuh"

// Amplitude of the middle factor, by value in kernel parameters.
struct AmpDev {
    int kind = FIO_AMP_ONE;
    int m = 0;
    double sigma2 = 1.0;
    double N = 1.0;                          // vector length (bumps scale xi by 1/N)
    double c[2 * FIO_AMP_MAX_BUMPS] = {};    // (x_k, xi_k)
};

struct fio_bf {
    fio_phase phase;
    AmpDev amp;
    int n = 0, d = 1, r = 0, L = 0, h = 0, sU = 0, sV = 0;   // n: vector length N (n^d)
    int nside = 0;                 // points per dimension; L = log2 nside
    int lsV = 0, lsU = 0;          // points per V frequency leaf / per U space leaf
    double tcheb[32];              // Chebyshev points on [-1, 1]
    fio::DevBuf VP, UP, M, P;      // P: PV | PU | Pc (float)
    std::vector<fio::DevBuf> C;    // index s - sV
    std::vector<fio::DevBuf> B;    // index s - h
    // C and B tables pre-arranged in the staged shared-memory layout of the fused passes, per
    // direction ([0] forward, [1] adjoint); empty where the staged fused kernels do not apply
    std::vector<fio::DevBuf> Cst[2], Bst[2];
    fio::DevBuf Mst;               // M in the staged layout of the forward right half
    fio::DevBuf ws;                // two coefficient states
    int64_t table_bytes = 0;
    bool force_unfused = false;    // use the per-level kernels even where the fused pass applies
    bool fused_v2 = false;         // fused pass without shared-memory table staging
    bool split = false;            // split-precision setting: transfer levels with BF16 hi + lo parts
    bool simt = false;             // FP32 setting on the CUDA cores instead of the tensor cores (staged fused path)
    int64_t N() const { return int64_t(n); }
    size_t pv_off() const { return 0; }
    size_t pu_off() const { return size_t(lsV) * r; }
    size_t pc_off() const { return size_t(lsV) * r + size_t(lsU) * r; }
};

namespace fio {
// Fused two-pass apply (r = 16, L >= 6): middle state `mid` of N*r*kc complex.
bool bf_fused_ok(const fio_bf* bf);
bool bf_v3_ok(const fio_bf* bf);   // staged fused kernels apply (64..512 pairs per CTA)
int bf_fused_kc(const fio_bf* bf);
// prec: -1 the handle's precision setting, 0 FP32, 1 split BF16.
fio_status bf_apply_fused(const fio_bf* bf, const float2* X, float2* Y, int64_t ld, int kc, int adjoint, float2* mid,
                          cudaStream_t st, int prec = -1);
// Pre-arrange the C and B tables in the staged layout of the fused kernels (bf_v3_ok handles).
fio_status bf_prestage(fio_bf* bf, cudaStream_t st);
// Transfer-level mode of the staged fused kernels (0 CUDA cores, 1 tensor cores FP16 parts,
// 2 tensor cores BF16 parts) for the given precision request.
int bf_fused_mode(const fio_bf* bf, int prec);
// Whether a bounded wait of a tensor-core kernel ran out since the last call (cleared); -1 on error.
int tc_wait_timeouts();
// bf_apply with an explicit precision (prec as above): the handle is not modified.
fio_status bf_apply_prec(const fio_bf* bf, const float2* X, float2* Y, int64_t ld, int k, int adjoint, int prec,
                         cudaStream_t st);
// Grouped fused apply over several operators (bf_v3_ok each): host tables, then
// launches that only read device copies of them.
struct BfGroupOp {
    const fio_bf* bf;
    const float2* X;
    float2* Y;
    float2* mid;   // N r k complex
    int k;
};
void bf_group_tables(const std::vector<BfGroupOp>& ops, int adjoint, std::vector<unsigned char>& left_args,
                     std::vector<int4>& left_items, std::vector<unsigned char>& right_args,
                     std::vector<int4>& right_items);
size_t bf_group_args_size();
fio_status bf_group_launch(const void* dleft_args, const int4* dleft_items, int nleft, const void* dright_args,
                           const int4* dright_items, int nright, int adjoint, int mode, cudaStream_t st);
// Host Lagrange polynomial l_k(u) on the nodes t[0..r).
double lagrange_host(const double* t, int r, int k, double u);
// 2D handles (d = 2, r = 25; bf2d.cu).  The same fio_bf fields hold the 2D
// tables: VP, UP, M, C (F_s), B (E_s) and P (Pc | Pc^T | QV | QU).
bool bf2d_ok_kind(int kind);
bool bf2d_ok_r1(int r1);
fio_status bf2d_build(fio_bf* bf, cudaStream_t st);
fio_status bf2d_apply_cols(const fio_bf* bf, const float2* X, float2* Y, int64_t ld, int kc, int adjoint, bool morton,
                           float2* s0, float2* s1, cudaStream_t st);
fio_status bf2d_unmorton(const fio_bf* bf, const float2* Xm, float2* X, int64_t ld, int k, cudaStream_t st);
// Sampled entries (rows[e], cols[e]) of a BF of the given rank, evaluated in FP64 from the factor
// definitions, and of K itself: out[2 e] = K~, out[2 e + 1] = K (device arrays).  1D: rank r;
// 2D: r1 x r1 grid, lexicographic indices.
fio_status bf1d_entries(const fio_phase& phase, const AmpDev& amp, int n, int r, const int64_t* rows,
                        const int64_t* cols, int S, double2* out, cudaStream_t st);
fio_status bf2d_entries(const fio_phase& phase, int amp_kind, int n, int r1, const int64_t* rows, const int64_t* cols,
                        int S, double2* out, cudaStream_t st);
// bf_apply with the frequency vectors of a 2D handle in quadtree (Morton)
// order when `morton` is set (the order of the HSS of K~^* K~); 1D: bf_apply.
fio_status bf_apply_ord(const fio_bf* bf, const float2* X, float2* Y, int64_t ld, int k, int adjoint, bool morton,
                        cudaStream_t st, int prec = -1);
// Y = K~ X or K~^* X for kc columns using states s0, s1 (each N*r*kc complex).
fio_status bf_apply_cols(const fio_bf* bf, const float2* X, float2* Y, int64_t ld, int kc, int adjoint,
                         float2* s0, float2* s1, cudaStream_t st);
}
