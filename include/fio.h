/*
 * fio.h -- C ABI of the B300 library for the two-stage approximate inverse of
 * discrete Fourier integral operators (Li & Liu, "Approximate Inversion of
 * Discrete Fourier Integral Operators via Hierarchically Semiseparable
 * Matrices").
 *
 * Problem (Eq. 1.1-1.2): K_ij = a(x_i, xi_j) exp(2 pi i Phi(x_i, xi_j)),
 * x_i = i/n, xi_j = j - n/2 (d = 1), N = n^d, amplitude a = 1.
 * Offline (Algorithm 1): butterfly factorization K~ of K (Section 2.2,
 * Eq. 2.1); randomized black-box HSS approximation G~ of G = K^* K sampled
 * through K~^* K~ (Section 3); ULV factorization of G~ (Section 2.4).
 * Online (Eq. 4.2): f = G~^{-1} K~^* u.
 *
 * Conventions shared by every call:
 *  - Vectors are complex64 (interleaved float re, im), column-major blocks of
 *    k columns with leading dimension ld >= N (in complex elements), in
 *    natural index order: entry j of a frequency-side vector is xi_j = j - n/2,
 *    entry i of a space-side vector is x_i = i/n.
 *  - Pointers named "device" must be CUDA device memory on the current
 *    device; the caller owns them and the library never frees them.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Calls are stream ordered and return before the GPU work finishes, except
 *    where a call says it synchronizes.  Asynchronous CUDA errors surface as
 *    FIO_ECUDA at a later call.
 *  - Handles (fio_bf, fio_hss) are owned by the library; free them with
 *    bf_free / hss_free.  A handle may be used by one stream at a time.
 *  - Every call returns a status; on failure fio_last_error() gives a
 *    message (thread local).  No call aborts the process.
 */
#ifndef FIO_H
#define FIO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FIO_OK = 0,
    FIO_EINVAL = 1,    /* bad argument (size, rank, pointer, layout) */
    FIO_ENOMEM = 2,    /* device allocation failed */
    FIO_ECUDA = 3,     /* CUDA runtime error (message in fio_last_error) */
    FIO_ENOTHPD = 4,   /* Cholesky pivot <= 0: G~ is not Hermitian positive definite */
    FIO_ERANK = 5,     /* HSS rank saturated the sample count */
    FIO_ETIMEOUT = 6,  /* a bounded device-side wait expired */
    FIO_EBUSY = 7      /* handle in use */
} fio_status;

typedef enum {
    FIO_PHASE_DFT = 0,        /* Phi = x . xi, d = 1 or 2  (then K^* K = N I exactly) */
    FIO_PHASE_1D_CABS = 1,    /* d = 1: Phi = x xi + c(x)|xi|, c(x) = (2 + s sin 2 pi x)/16 */
    FIO_PHASE_2D_ELLIPTIC = 2,/* d = 2: Phi = x . xi + sqrt(c1^2 xi1^2 + c2^2 xi2^2),
                                 c1 = (2 + sin 2 pi x1 sin 2 pi x2)/16,
                                 c2 = (2 + cos 2 pi x1 cos 2 pi x2)/16 (Section 5.2) */
    FIO_PHASE_1D_CABS8 = 3,   /* d = 1: Phi = x xi + c(x)|xi|, c(x) = (2 + s sin 2 pi x)/8
                                 (the operator of Section 5.1) */
    FIO_PHASE_2D_ISO = 4      /* d = 2: Phi = x . xi + c(x) ||xi||,
                                 c(x) = (3 + s sin 2 pi x1 sin 2 pi x2)/8 (Section 5.3) */
} fio_phase_kind;

typedef struct {
    int kind;     /* fio_phase_kind */
    double s;     /* modulation depth s of c(x); 1.0 for the standard operator */
} fio_phase;

/* Amplitude a(x, xi) of Eq. 1.2 (a = 1 unless given).  It enters only the
 * middle factor of the BF, M = a(z, gamma) e^{2 pi i Phi(z, gamma)} (Section
 * 2.2), so it must be smooth on the Chebyshev grids of the middle level. */
typedef enum {
    FIO_AMP_ONE = 0,     /* a = 1 */
    FIO_AMP_BUMPS = 1,   /* d = 1 (Section 5.1): a = sum_k exp(-((x - x_k)^2 + ((xi - xi_k)/N)^2) / sigma2) */
    FIO_AMP_HANKEL = 2   /* d = 2 with FIO_PHASE_2D_ISO (Section 5.3): a = H0^(1)(2 pi phi) e^{-2 pi i phi},
                            phi = Phi - x . xi = c(x) ||xi|| (infinite at xi = 0, which no Chebyshev
                            point of the middle level reaches) */
} fio_amp_kind;
#define FIO_AMP_MAX_BUMPS 32
typedef struct {
    int kind;               /* fio_amp_kind */
    int m;                  /* FIO_AMP_BUMPS: number of bumps, 1 .. FIO_AMP_MAX_BUMPS */
    double sigma2;          /* FIO_AMP_BUMPS: sigma^2 > 0 */
    const double* centers;  /* FIO_AMP_BUMPS: host array of m pairs (x_k, xi_k), read during the call */
} fio_amp;

typedef struct fio_bf fio_bf;
typedef struct fio_hss fio_hss;

/* Sampler for the black-box HSS construction (Section 3): the matrix H whose
 * products H X the construction may request. */
typedef enum {
    FIO_SAMPLER_NORMAL = 0,   /* H = K~^* K~ through `bf` (Section 4.1) */
    FIO_SAMPLER_DENSE = 1     /* H = dense device matrix (N x N complex64,
                                 column-major, leading dimension `ld`); for tests */
} fio_sampler_kind;

typedef struct {
    int kind;              /* fio_sampler_kind */
    const fio_bf* bf;      /* FIO_SAMPLER_NORMAL */
    const void* dense;     /* FIO_SAMPLER_DENSE: device pointer */
    int64_t ld;            /* FIO_SAMPLER_DENSE: leading dimension (>= N) */
} fio_sampler;

/* ------------------------------------------------------------------------
 * bf_build -- butterfly factorization K~ of K (Section 2.2, Eq. 2.1).
 *   n: points per dimension (power of two); d: dimension.
 *   d = 1: 16 <= n <= 2^24, r: Chebyshev interpolation rank (1..16), N = n.
 *   d = 2: 8 <= n <= 1024, r = r1^2 with 3 <= r1 <= 7 (r1 x r1 tensor
 *     Chebyshev grid; the 2D workloads use r = 25), N = n^2;
 *     quadtrees, vectors in lexicographic order (x_i = (i1, i2)/n with
 *     i = i1 n + i2, xi_j = (j1 - n/2, j2 - n/2) with j = j1 n + j2).
 *   Trees: space/frequency trees of depth L = log2 n; middle level
 *   h = floor(L/2); outermost factors at max(L-3, h) (practical top level,
 *   Section 5.2).
 *   Every factor entry is evaluated on the device from its definition
 *   (phase differences in FP64, reduced mod 1, stored complex64).
 *   Synchronizes `stream` before returning.  *out receives the handle.
 *   Errors: FIO_EINVAL (sizes), FIO_ENOMEM, FIO_ECUDA.
 * ---------------------------------------------------------------------- */
fio_status bf_build(const fio_phase* phase, int n, int d, int r, void* stream, fio_bf** out);

/* bf_build_amp -- bf_build with an amplitude (the paper's bf_build(phase, amp,
 *   n, d, r)); amp = NULL is a = 1.  Only the middle factor changes: its
 *   entries are multiplied by a(z_i, gamma_j), evaluated in FP64 on the device
 *   (the Bessel functions J0, Y0 of the Hankel amplitude by CUDA's j0, y0).
 *   Errors: FIO_EINVAL for an amplitude the dimension or phase does not admit
 *   (bumps: d = 1; Hankel: d = 2 with FIO_PHASE_2D_ISO), m out of range or
 *   sigma2 <= 0; otherwise as bf_build. */
fio_status bf_build_amp(const fio_phase* phase, const fio_amp* amp, int n, int d, int r, void* stream,
                        fio_bf** out);

/* bf_entries -- S sampled entries of K~ and of K (Section 2.2; the error
 *   measure of Section 5).  rows, cols: host arrays of S indices in [0, N)
 *   (lexicographic in 2D); 1 <= S <= 2^22.  Each K~ entry is evaluated in FP64
 *   from the factor definitions of Eq. 2.1 (not from the stored complex64
 *   tables): only one chain of pairs couples x_i with xi_j, so the entry is a
 *   product of one r x r block per level.  K(i, j) = a(x_i, xi_j)
 *   e^{2 pi i Phi(x_i, xi_j)} in FP64.  out: host array of 4 S doubles,
 *   sample e at out[4e .. 4e+3] = (Re K~, Im K~, Re K, Im K).  A Hankel sample
 *   at xi = 0 (amplitude infinite) is returned as zeros.  Synchronizes
 *   `stream`.  Errors: FIO_EINVAL (null pointer, S or index out of range),
 *   FIO_ENOMEM, FIO_ECUDA. */
fio_status bf_entries(const fio_bf* bf, const int64_t* rows, const int64_t* cols, int S, void* stream, double* out);

/* bf_entry_error -- e = sqrt(sum_e |K~_e - K_e|^2 / sum_e |K_e|^2) over the
 *   samples, for the BF of rank r of (phase, amp, n, d) (amp may be NULL),
 *   without building its tables; for a random sample this estimates the
 *   relative error ||K~ - K|| / ||K|| in the Frobenius norm, the expected
 *   value of the sampled-row error e_cBF of Section 5 for random vectors.
 *   Arguments as bf_build_amp and bf_entries.  Errors: FIO_EINVAL (as
 *   bf_build_amp; also when no sample has a finite nonzero K), FIO_ENOMEM,
 *   FIO_ECUDA. */
fio_status bf_entry_error(const fio_phase* phase, const fio_amp* amp, int n, int d, int r, const int64_t* rows,
                          const int64_t* cols, int S, void* stream, double* err);

/* bf_build_tol -- adaptive BF rank (the BF tolerance of Section 5): the
 *   smallest rank of the candidate list whose bf_entry_error on the given
 *   samples is <= tol, then bf_build_amp at that rank.  Candidates: d = 1:
 *   r = 4, 6, ..., 16; d = 2: r = r1^2, r1 = 3 .. 7.  If no candidate reaches
 *   tol the largest is built and *err_out (> tol) says so.  *r_out, *err_out
 *   (may be NULL): the rank built and its sampled error.  Errors: as
 *   bf_build_amp and bf_entry_error; FIO_EINVAL for tol <= 0. */
fio_status bf_build_tol(const fio_phase* phase, const fio_amp* amp, int n, int d, double tol, const int64_t* rows,
                        const int64_t* cols, int S, void* stream, fio_bf** out, int* r_out, double* err_out);

/* bf_apply -- Y = K~ X (adjoint = 0) or Y = K~^* X (adjoint = 1); the adjoint
 *   applies the conjugate-transposed factors in reverse order (Section 2.2).
 *   X, Y: device, N x k complex64, column-major, leading dimension ld >= N;
 *   X and Y must not overlap.  k >= 0 (k = 0 is a no-op).  Uses the handle's
 *   scratch state (allocated on first use, grown as needed).
 *   Errors: FIO_EINVAL, FIO_ENOMEM, FIO_ECUDA. */
fio_status bf_apply(fio_bf* bf, const void* X, void* Y, int64_t ld, int k, int adjoint, void* stream);

/* bf_apply_noalloc -- the same products as bf_apply for callers that must
 *   not allocate device memory (no counterpart in the paper: it serves
 *   callers whose host framework owns all device memory, or that cannot
 *   afford a cudaMalloc, which may synchronize the device).  The coefficient
 *   state lives in a fixed 32 MiB array compiled into the library (held on
 *   every GPU that loads it until exit) instead of the handle's scratch, so
 *   this call allocates and frees nothing.  Columns are processed in chunks
 *   that fit the array; FIO_EINVAL if one column's state (N r complex64, twice
 *   that on the per-level path) exceeds 2^22 elements.  The first call on a
 *   device looks up the array's device address (cudaGetSymbolAddress) with
 *   that device current: make it before any stream capture.  All calls share
 *   the array: calls whose GPU work overlaps race, so order them on one
 *   stream.  1D handles only (FIO_EINVAL for 2D).  Arguments and errors as
 *   bf_apply. */
fio_status bf_apply_noalloc(const fio_bf* bf, const void* X, void* Y, int64_t ld, int k, int adjoint, void* stream);

/* bf_set_path -- choose the kernels of bf_apply (no paper counterpart; the
 *   results agree to FP32 rounding):  0 = automatic (fused two-pass kernels
 *   where r = 16 and n >= 64, else per-level kernels), 1 = one kernel per
 *   factor (per-level), 2 = fused two-pass (tables staged through shared
 *   memory where each half has 64..512 pairs per CTA; the transfer levels on
 *   the tensor cores), 3 = fused two-pass without the staging, 4 = the staged
 *   fused kernels with the FP32 transfer levels on the CUDA cores instead of
 *   the tensor cores.  FIO_EINVAL where a fused path is unsupported (2D
 *   handles: per-level kernels only). */
fio_status bf_set_path(fio_bf* bf, int path);

/* bf_set_precision -- arithmetic of the transfer levels of bf_apply (the real
 *   Lagrange products of Eq. 2.4-2.6, shared by every box of a level):
 *   FIO_FP32 (0, default) FP32 accuracy: on the staged fused kernels these
 *   products run on the tensor cores (tcgen05, FP32 accumulation in tensor
 *   memory) with both operands split into FP16 parts v = hi + lo (three
 *   products hi*hi + hi*lo + lo*hi; every row scaled by an exact power of two
 *   into the FP16 range), elsewhere (and with path 4) FP32 FMA on the CUDA
 *   cores; FIO_SPLIT_BF16 (1) the same tensor-core products on BF16 parts
 *   (8 + 8 bits, relative error of an apply about 1e-5).  Phases and the
 *   middle factor are FP32 in both.  Split precision runs on the staged fused
 *   kernels (r = 16, 2^12 <= n <= 2^18; FIO_EINVAL otherwise) whatever
 *   bf_set_path chose. */
typedef enum { FIO_FP32 = 0, FIO_SPLIT_BF16 = 1 } fio_precision;
fio_status bf_set_precision(fio_bf* bf, int precision);

/* bf_info -- sizes of a handle: out[0..7] = N (vector length n^d), d, r, L,
 *   h, sU (space level of U), sV (space level of V), bytes of device factor
 *   tables. */
fio_status bf_info(const fio_bf* bf, int64_t* out8);

void bf_free(fio_bf* bf);

/* ------------------------------------------------------------------------
 * hss_build_from_samples -- randomized black-box HSS construction of the
 *   Hermitian H given by `sampler` (Section 3.1-3.3), over an index set of
 *   size N split into 2^Lh leaves of size `leaf` (N = leaf * 2^Lh, Lh >= 1,
 *   leaf <= 256).  Per level l an independent Gaussian test matrix with
 *   s_l = rhat_l + m_l + p columns (p = `oversample`) is drawn from
 *   Philox4x32-10 with key `seed` and counter (row, col, l, attempt), Box-Muller
 *   to complex N(0,1) + i N(0,1).  rhat_l starts at m_l/2 and is doubled (new
 *   attempt) while the truncated rank exceeds it.  Per node: orthonormal null
 *   basis Gamma of Omega_tau, column-pivoted QR of Y_tau Gamma truncated where
 *   |R_kk| <= tol * max_j ||Y_tau(:,j)||, one rank per level (the level
 *   maximum), residual block D-check (Section 3.1), root H^[0] = Y^[0] Omega^+;
 *   top-down postprocessing for B and leaf D (Section 3.3).
 *   FIO_SAMPLER_NORMAL with a 2D BF: the index set is the frequency grid in
 *   quadtree (Morton) order, so that leaves and nodes are quadtree boxes and
 *   their halves.
 *   Synchronizes `stream` (ranks are decided on the host).
 *   Errors: FIO_EINVAL, FIO_ENOMEM, FIO_ECUDA, FIO_ERANK.
 * ---------------------------------------------------------------------- */
fio_status hss_build_from_samples(const fio_sampler* sampler, int64_t N, int leaf, int oversample,
                                  double tol, uint64_t seed, void* stream, fio_hss** out);

/* hss_from_generators -- build a handle from host generators (tests, restart).
 *   ranks[0..Lh] (ranks[0] = 0); U: concatenation over l = 1..Lh, node-major,
 *   of column-major m_l x r_l blocks (m_Lh = leaf, m_l = 2 r_{l+1});
 *   B: concatenation over l = 0..Lh-1, node-major, of column-major
 *   r_{l+1} x r_{l+1} blocks (B_{alpha2,alpha1}); D: 2^Lh column-major
 *   leaf x leaf blocks.  Host pointers, complex64, copied.  Synchronizes. */
fio_status hss_from_generators(int64_t N, int leaf, const int* ranks, const void* U, const void* B,
                               const void* D, void* stream, fio_hss** out);

/* hss_info -- out[0] = N, out[1] = leaf, out[2] = Lh, out[3 + l] = r_l for
 *   l = 0..Lh (needs 3 + Lh + 1 entries; max_out bounds the writes), and the
 *   number of sample columns drawn is returned in *samples if non-NULL. */
fio_status hss_info(const fio_hss* hss, int64_t* out, int max_out, int64_t* samples);

/* hss_matvec -- Y = G~ X through the telescoping factorization (Eq. 2.8).
 *   X, Y: device, N x k complex64, ld >= N, no overlap. */
fio_status hss_matvec(const fio_hss* hss, const void* X, void* Y, int64_t ld, int k, void* stream);

/* hss_ulv_factor -- ULV factorization of G~ (Section 2.4, Eq. 2.9-2.12):
 *   per node a unitary Q with Q^* U = [0; U^_2] (QR of U with the R block
 *   moved to the bottom), Cholesky of D-check_11, D^_21, Schur complement,
 *   merge into the parent, Cholesky of the root.  Stored per node as the
 *   single matrix W = [[L11^{-1}, 0], [-D^_21 L11^{-1}, I]] Q^* (the up pass
 *   applies W, the down pass W^*).  Synchronizes.
 *   Errors: FIO_ENOTHPD (a pivot <= 0), FIO_ENOMEM, FIO_ECUDA. */
fio_status hss_ulv_factor(fio_hss* hss, void* stream);

/* hss_solve -- X = G~^{-1} B by the ULV bottom-up / root / top-down passes
 *   (Section 2.4).  B, X: device, N x k complex64, ld >= N; B may equal X.
 *   Per level the node products W_t y_t (up) and W_t^* c_t (down) run as:
 *   k <= 8: one row per thread streaming W (the small upper levels and the
 *   root in one launch); k > 8: register-tiled CUDA-core FP32 products, or
 *   with solve path 1 (hss_set_solve_path) and 32 <= m_l <= 512 on the tensor
 *   cores (tcgen05, FP16 hi/lo parts with power-of-two row and column scales,
 *   FP32 accumulation: FP32 accuracy; BF16 parts when fio_solve runs on a
 *   split-precision BF handle).  A bounded MMA wait that runs out is reported
 *   by fio_device_status.
 *   Errors: FIO_EINVAL (not factored, k < 0, ld < N), FIO_ENOMEM, FIO_ECUDA. */
fio_status hss_solve(const fio_hss* hss, const void* B, void* X, int64_t ld, int k, void* stream);

/* hss_set_solve_path -- 0 (default): node products on the CUDA cores in FP32;
 *   1: the tensor-core node products where they apply (see hss_solve; split
 *   precision of Section 5's mixed-precision setting for the HSS products).
 *   Errors: FIO_EINVAL (null handle, path not 0 or 1). */
fio_status hss_set_solve_path(fio_hss* hss, int path);

/* fio_solve -- online stage f = G~^{-1} K~^* u (Eq. 4.2), plus `refine_steps`
 *   steps of iterative refinement f += G~^{-1}(K~^* u - K~^* K~ f) whose
 *   residuals use the FP32 applies of K~ and K~^* (also for a handle set to
 *   split precision).
 *   U, F: device, N x k complex64, ld >= N, no overlap.  2D handles: the HSS
 *   (built by hss_build_from_samples from this BF) is over the frequency
 *   index in quadtree (Morton) order; the solve runs in that order and F is
 *   returned in lexicographic order. */
fio_status fio_solve(const fio_bf* bf, const fio_hss* hss, const void* U, void* F, int64_t ld, int k,
                     int refine_steps, void* stream);

/* fio_pcg -- the iterative use of Algorithm 1's output (Section 4.1): conjugate
 *   gradients on the approximate normal equation K~^* K~ f = K~^* u (Eq. 4.3),
 *   preconditioned by the ULV factorization F~ = G~^{-1} of the HSS.  Each
 *   column is its own CG run from f_0 = 0; a column stops when its recurrence
 *   residual satisfies ||r|| <= tol ||K~^* u|| (the paper's stopping rule with
 *   tol = 1e-12 in FP64; the complex64 applies here floor the attainable
 *   relative residual near 1e-6, so useful tolerances are >= 1e-6), or after
 *   maxit iterations.  Inner products and CG scalars are FP64 on the device.
 *   U, F: device, N x k complex64, ld >= N, no overlap (2D: lexicographic
 *   order, the iteration runs in the HSS's quadtree order).  iters (host, may
 *   be NULL): iterations taken by the slowest column; relres (host, k
 *   doubles, may be NULL): final relative residual per column.  The HSS must
 *   be factored (hss_ulv_factor).  Synchronizes `stream` once per iteration
 *   (convergence test on the host).  Errors: FIO_EINVAL, FIO_ENOMEM, FIO_ECUDA. */
fio_status fio_pcg(const fio_bf* bf, const fio_hss* hss, const void* U, void* F, int64_t ld, int k, double tol,
                   int maxit, int* iters, double* relres, void* stream);

/* fio_set_large_node -- node-size threshold of the large-node kernels (no
 *   paper counterpart; process-wide, default 384).  HSS levels with at most 16
 *   nodes of size m >= m_min (the top levels of 2D operators, whose ranks grow
 *   like sqrt(N)) run level-3 formulations of the node steps, batched over the
 *   level's nodes: Y Omega^+ through the Gram matrix Omega Omega^* and its
 *   Cholesky factor; a null basis Gamma of Omega_tau from a projected Gaussian
 *   block; the rank-revealing step as a pivoted Cholesky of (Y Gamma)^*(Y Gamma)
 *   (the pivots of the column-pivoted QR of Y Gamma) truncated at the same
 *   threshold; bases orthonormalized by CholQR2; the ULV elimination with
 *   Q = [Q1 Q2] (Q2 R = U by CholQR2, Q1 its orthonormal complement).  Products
 *   by cuBLAS GEMMs in FP32 (FP64 for the node pass when tol < 1e-4), with the
 *   Gram matrix of Y Gamma, its pivoted Cholesky, the root and the Cholesky
 *   factorizations of the eliminated blocks in FP64.  Mathematically these give
 *   the same HSS approximation and an exact ULV factorization; generators differ
 *   by unitary changes of basis, and ranks at the truncation boundary may differ
 *   by a few.
 *   Errors: FIO_EINVAL for m_min < 1. */
fio_status fio_set_large_node(int m_min);

/* fio_set_large_node_count -- the large-node kernels take levels with at most
 *   max_nodes nodes (process-wide, default 16); FIO_EINVAL for max_nodes < 1. */
fio_status fio_set_large_node_count(int max_nodes);

void hss_free(fio_hss* hss);

/* ------------------------------------------------------------------------
 * Batched online stage over several resident operators of uneven size (the
 * batched workload: many independent 1D operators, a block of RHS each; no
 * paper counterpart beyond applying Eq. 4.2 to each operator).
 * fio_batch_create -- group n_ops built pairs (bfs[i], hss[i]) of 1D
 *   operators (FIO_EINVAL for a 2D one); the HSS handles must be factored.  The batch keeps pointers to the handles (they
 *   must outlive it) and owns its workspaces.
 * fio_batch_set_mode -- 0: one fio_solve per operator; 1: grouped launches
 *   (each stage one launch over all operators: the two fused BF half passes,
 *   one ULV node-product launch per tree depth, one for the roots); 2: the
 *   grouped launches captured once into a CUDA graph and replayed (default);
 *   3: one persistent launch (one CTA per SM) that walks a device work list
 *   of (stage, operator, block) items -- BF left and right half passes, ULV
 *   up levels, roots, down levels -- each item waiting (bounded; a wait that
 *   runs out is reported by fio_device_status) until the previous stage of
 *   its own operator is complete, so operators advance independently.
 * fio_batch_solve -- F[i] = G~_i^{-1} K~_i^* U[i] for every i: U, F host
 *   arrays of n_ops device pointers to N_i x k[i] complex64 blocks with
 *   leading dimension N_i (U[i] and F[i] must not overlap).  The launch plan
 *   (device tables of arguments and work items; the graph) is built on the
 *   first call for a given (U, F, k) and reused while they stay the same;
 *   building it synchronizes the stream.
 * fio_batch_autotune -- times each candidate configuration (per-operator
 *   calls with the fused staged, fused unstaged or one-kernel-per-factor BF;
 *   grouped launches; grouped launches in a graph; the persistent launch; the
 *   grouped and persistent launches with the BF transfer levels on the CUDA
 *   cores instead of the tensor cores) over `reps` solves on
 *   the given buffers, keeps the fastest, and writes one line per candidate
 *   ("name ms") into report (len bytes, may be NULL).
 * ---------------------------------------------------------------------- */
typedef struct fio_batch fio_batch;
fio_status fio_batch_create(fio_bf* const* bfs, fio_hss* const* hss, int n_ops, fio_batch** out);
fio_status fio_batch_set_mode(fio_batch* batch, int mode);
fio_status fio_batch_solve(fio_batch* batch, const void* const* U, void* const* F, const int* k, void* stream);
fio_status fio_batch_autotune(fio_batch* batch, const void* const* U, void* const* F, const int* k, int reps,
                              void* stream, char* report, int64_t len);
void fio_batch_free(fio_batch* batch);

/* fio_device_status -- FIO_ETIMEOUT if a bounded wait inside a tensor-core
 *   kernel (an mbarrier wait for its MMAs: BF half passes or ULV node products)
 *   ran out since the last call, which
 *   marks that launch's results invalid; the flag is cleared.  Synchronizes
 *   with the device (reads a device flag).  No paper counterpart. */
fio_status fio_device_status(void);

/* fio_selftest_wait_timeout -- runs the persistent batched kernel on a one-item
 *   work list whose prerequisite never completes, so that the item's bounded
 *   wait runs out (failure detection without a GPU fault; no paper
 *   counterpart).  Returns FIO_ETIMEOUT (read back through fio_device_status,
 *   which clears the flag) when the bound works; synchronizes `stream`. */
fio_status fio_selftest_wait_timeout(void* stream);

/* fio_last_error -- message of the last failing call on this thread. */
const char* fio_last_error(void);

/* fio_profile_enable -- diagnostics, not part of the method: while enabled,
 *   every kernel launched by bf_apply, hss_solve and fio_solve is bracketed
 *   by a pair of CUDA events recorded on its stream (two event records per
 *   launch).  Process-wide, not thread safe. */
fio_status fio_profile_enable(int on);

/* fio_profile_report -- waits for the recorded events and writes one line
 *   "kernel_name launches total_ms" per kernel into buf (NUL terminated),
 *   then clears the record.  FIO_EINVAL if len is too small. */
fio_status fio_profile_report(char* buf, int64_t len);

#ifdef __cplusplus
}
#endif
#endif /* FIO_H */
