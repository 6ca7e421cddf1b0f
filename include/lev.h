/*
 * lev.h -- C ABI of the GB300 (sm_103a) rank-revealing leverage-score estimator.
 *
 * The library computes the estimator of Alg. 10 (LS-HRN-approx) of Sobczyk and
 * Gallopoulos, "Estimating leverage scores via rank revealing methods and
 * randomization": a CountGauss sketch A~ = G S A (Alg. 3), a column-pivoted QR
 * of the sketch that reveals the numerical rank r and the selected columns K
 * (Alg. 4), and the squared row norms theta~_i = ||A_{i,K} R_11^{-1} Omega||^2
 * (Alg. 8 steps 4-5; the squared row norms of A (Pi_1 A)^+ Pi_2, eq. (10)). The problem statement (Sec. 1; Alg. 10
 * Require/Ensure): a tall matrix A (n x d, n >> d, dense or sparse, any rank)
 * in; the estimated leverage scores theta~ (n) and the numerical rank r out.
 *
 * Conventions shared by every entry point:
 *  - Return value: LEV_OK (0) or one of the LEV_E* codes below; no C++
 *    exception crosses the ABI. lev_last_error() gives a message for the last
 *    failing call on the calling thread.
 *  - Ownership: every array is owned by the caller. Device pointers are plain
 *    CUDA device pointers. The handle owns its scratch memory (grown on demand
 *    with cudaMalloc), a cache of the Gaussian sketch matrix G per
 *    (seed, m, s, precision) and of the CountSketch bucket permutation per
 *    (seed, n, s).
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream). Work is enqueued on it; a call returns before the work finishes
 *    unless it writes a host-side result (rank), in which case it synchronises
 *    `stream` once at the end.
 *  - Layouts: dense matrices are row-major with a leading dimension (elements);
 *    CSR uses int64 row_ptr (n+1), int32 col (nnz, any order within a row,
 *    duplicates are summed) and FP32 values.
 *  - Limits: 1 <= d <= 4096, 1 <= n < 2^31, 1 <= s < 2^31, 1 <= m <= 2^20 (m < d is
 *    accepted: the rank is then at most m), 1 <= k <= 4096.
 *  - Thread safety: a handle may be used by one host thread at a time. Its scratch and caches are
 *    shared by all its calls, so calls of one handle on different streams must not overlap on
 *    the device (order them, e.g. with an event); work in flight on several streams takes one
 *    handle per stream.
 *
 * Random streams (both the library and its test oracle implement these from
 * the published definitions; no code is shared):
 *  - splitmix64(key, c): state = key + (c+1) * 0x9E3779B97F4A7C15 (mod 2^64),
 *    then the splitmix64 finaliser (Steele, Lea and Flood 2014);
 *  - key_t = seed XOR (t * 0xD1B54A32D192ED03), t = 1 hash, 2 G, 3 Omega;
 *  - CountSketch (Sec. 3.4.3): x = splitmix64(key_1, i), bucket h(i) =
 *    (hi32(x) * s) >> 32, sign = +1 if bit 0 of x is 0 else -1;
 *  - N(0,1) number c of stream t: Box-Muller, cosine branch, with
 *    u1 = ((splitmix64(key_t, 2c) >> 11) + 1) 2^-53, u2 = (splitmix64(key_t, 2c+1) >> 11) 2^-53;
 *  - G[j, b] = N_{j*s + b} / sqrt(m) (a Gaussian embedding, Sec. 3.4.1 scaling) for the draws N_c
 *    of stream 2; the tensor-core forms of the Gaussian stage take fl32(N_c) in their operand type
 *    (the BF16 hi + lo pair with LEV_BF16X3, about 2^-17 of N_c) and apply 1/sqrt(m) in FP32;
 *    Omega[p, q] = N_{p*k + q} / sqrt(k) (stream 3), p the pivot position (0 <= p < r), q < k.
 */
#ifndef LEV_H
#define LEV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define LEV_OK        0
#define LEV_EINVAL    1  /* bad shape, pointer, parameter, or CSR structure */
#define LEV_ENOMEM    2  /* cudaMalloc of handle scratch failed */
#define LEV_ECUDA     3  /* a CUDA runtime call or kernel launch failed */
#define LEV_ETIMEOUT  4  /* a bounded device-side wait gave up (the kernel returned early) */
#define LEV_ERANK0    5  /* numerical rank 0 (A = 0 or |R_00| = 0): theta~ is set to 0 */

/* Arithmetic of a stage (the sketch's Gaussian product, or the final pass). */
#define LEV_FP32    0   /* FP32 SIMT FMA */
#define LEV_TF32    1   /* tcgen05 kind::tf32, FP32 accumulate */
#define LEV_BF16    2   /* tcgen05 kind::f16 with BF16 operands, FP32 accumulate */
#define LEV_BF16X3  3   /* split hi+lo BF16 of FP32 operands, FP32 accumulate: hi*hi + lo*hi + hi*lo */

/* Flags (lev_params.flags). */
#define LEV_OMEGA_IDENTITY  1u  /* Omega = I_r, k = r (the Pi_2-free mode of Sec. 7.4) */
#define LEV_SKETCH_IDENTITY 2u  /* S = I, G = I, A~ = A (tests; needs n <= 65536) */
#define LEV_FORCE_PIVOTS    4u  /* take perm_in[0..rank_in) as the pivots, no rank test */
#define LEV_HOST_ASYNC      8u  /* lev_estimate_dense with host buffers and rank == NULL: enqueue only */
#define LEV_SKETCH_SRHT    16u  /* A~ = G F S A: an SRHT F (t = srht_t rows) after the CountSketch (Sec. 4.1) */
#define LEV_RANK_SVD       32u  /* rank = #{sigma_j(A~) > tau sigma_1(A~)} (Alg. 11 step 3, Sec. 7.2); columns
                                   from the pivoted QR run to the end; d <= 1024 */
#define LEV_SRRQR          64u  /* after the rank: strong-RRQR swaps at that rank until every
                                   rho_ij <= phi (Alg. 2); d <= 1024 */
#define LEV_CSR_UNCHECKED 128u  /* the caller vouches for the CSR structure: no validation pass */
#define LEV_OMEGA_REDUCED 256u  /* lev_omega_factor: the r-column factor R_11^{-1} L_r when r < k (below) */

typedef struct lev_handle lev_handle;

typedef struct lev_params {
    double   eps;          /* CountSketch OSE parameter (Alg. 3 step 1), used when s == 0 */
    double   delta;        /* CountSketch OSE failure probability, used when s == 0 */
    double   gamma;        /* oversampling, m = ceil(gamma d) when m == 0 (Alg. 3 step 2) */
    int64_t  s;            /* CountSketch buckets (the paper's r); 0 = from eps, delta */
    int64_t  m;            /* rows of G; 0 = ceil(gamma d) */
    int64_t  k;            /* columns of Omega; 0 = JL size 4 ln n / (eps^2/2 - eps^3/3) */
    double   tau;          /* rank rule |R_jj| > tau |R_00| (Sec. 7.2); <= 0 means 1e-5 */
    uint64_t seed;         /* seed of the three random streams */
    int32_t  sketch_prec;  /* LEV_FP32 | LEV_TF32 | LEV_BF16 | LEV_BF16X3 for A~ = G B */
    int32_t  final_prec;   /* same set for theta~ = ||A M_full||^2 */
    uint32_t flags;        /* LEV_* flags above */
    int32_t  srht_t;       /* rows t of the SRHT with LEV_SKETCH_SRHT (1 <= t <= s; s a power of two) */
    const int32_t* perm_in;  /* device, d entries; read with LEV_FORCE_PIVOTS */
    int64_t  rank_in;        /* number of forced pivots; read with LEV_FORCE_PIVOTS */
    int64_t  row0;           /* row shard: global index of local row 0 (hash and sign of row i use
                                row0 + i); read by lev_sketch_* and lev_resolve_sizes, 0 elsewhere */
    int64_t  n_total;        /* row shard: rows of the whole matrix (k = 0 is derived from it);
                                0 = the call's n; same entry points as row0 */
    double   phi;            /* strong-RRQR bound (LEV_SRRQR), >= 1; 0 means 2 */
} lev_params;

/* Create a handle on CUDA device `device` (the device is made current for every
 * call on the handle). *out receives the handle. Errors: LEV_EINVAL (NULL out or
 * bad device), LEV_ECUDA. */
int lev_create(lev_handle** out, int device);

/* Free the handle and all its scratch memory. NULL is accepted. Waits for
 * pending work on the handle's device. */
int lev_destroy(lev_handle* h);

/* Message of the last failing call on this thread ("" if none). Never NULL. */
const char* lev_last_error(void);

/* Device memory the handle holds now, in bytes: its scratch buffers (grown on demand by the calls
 * made on it, never shrunk) and its caches of G, Omega and the CountSketch bucket permutation.
 * Host only (no device work, no synchronisation). lev_destroy releases all of it.
 * Errors: LEV_EINVAL (NULL handle or bytes). */
int lev_workspace_bytes(lev_handle* h, int64_t* bytes);

/* Fill *p with the paper's practical defaults (Alg. 3: eps = 1/2, delta = 1/3,
 * gamma = 2), tau = 1e-5, seed 0, FP32 stages, sizes 0 (derived), no flags. */
int lev_params_init(lev_params* p);

/* Resolve the sizes a call with (p, n, d) would use: s = ceil((d^2+d) /
 * ((2 eps - eps^2)^2 delta)) (Alg. 3 step 1), m = ceil(gamma d) (Alg. 3 step 2),
 * k = ceil(4 ln n / (eps^2/2 - eps^3/3)) (Gaussian JLT lemma, Sec. 3.4.1),
 * each unless set explicitly in p. Any output pointer may be NULL. */
int lev_resolve_sizes(const lev_params* p, int64_t n, int64_t d,
                      int64_t* s, int64_t* m, int64_t* k);

/* Build the handle's caches of data-independent operands for a call with (n, d, p) on `stream`,
 * ahead of the first call that needs them: the CountSketch bucket permutation (Sec. 3.4.3, per
 * seed, n, s and row0), G in the operand form of p->sketch_prec (Alg. 3 step 3; m x t with
 * LEV_SKETCH_SRHT) and Omega with the Cholesky factor of its Gram matrix (d <= 1024, unless
 * LEV_OMEGA_IDENTITY; see lev_omega_factor). Later calls with the same
 * seed and sizes reuse them. Asynchronous; no arrays are read. Errors: LEV_EINVAL, LEV_ENOMEM,
 * LEV_ECUDA. */
int lev_prepare(lev_handle* h, int64_t n, int64_t d, const lev_params* p, void* stream);

/* Row shards. S A = sum_p S_{:,P_p} A_{P_p,:} for any partition of the rows into blocks P_p
 * (block matrix product), and G and the SRHT act linearly on S A, so the sketch of a matrix
 * whose rows are split across processes is the SUM of the sketches of its row blocks when each
 * block hashes its rows by their global index: call lev_sketch_* on each block with
 * p->row0 = the block's first global row and p->n_total = the rows of the whole matrix, sum the
 * m x d results (one all-reduce), then lev_rrqr and lev_omega_factor on the sum (the same on
 * every process) and lev_final_* on each block. Every other entry point sums over the rows of
 * its own A and rejects row0 != 0 or n_total != 0 with LEV_EINVAL. */

/* CountGauss sketch of dense A (Alg. 3): Atilde (m x d, row-major, ld = d,
 * FP32, device) = G (S A). A: device, n x d FP32, leading dimension lda >= d.
 * p->sketch_prec selects the arithmetic of the product G B. With LEV_SKETCH_SRHT
 * the CountSketch is followed by the SRHT F = sqrt(s/t) P H D of Sec. 3.4.2 (D:
 * signs of stream 4; H: Walsh-Hadamard / sqrt(s); P: t uniform row draws of
 * stream 5, multiply-shift of the high word), S~ = F S (Sec. 4.1), and G is
 * m x t: A~ = G (F (S A)). s must be a power of two, at most 2^24.
 * Errors: LEV_EINVAL, LEV_ENOMEM, LEV_ECUDA. */
int lev_sketch_dense(lev_handle* h, const float* A, int64_t n, int64_t d, int64_t lda,
                     const lev_params* p, float* Atilde, void* stream);

/* CountGauss sketch of CSR A (Alg. 3); arguments as lev_sketch_dense, with A
 * given by device arrays row_ptr (n+1, int64, row_ptr[0] = 0, non-decreasing,
 * row_ptr[n] = nnz), col (nnz, int32 in [0, d)) and val (nnz, FP32). Every CSR entry
 * point checks the structure of row_ptr first, in one device pass whose verdict it reads
 * (one synchronisation of `stream`), and returns LEV_EINVAL before any kernel reads col or
 * val if it is malformed; LEV_CSR_UNCHECKED in p->flags skips the check (the caller vouches
 * for row_ptr). Out-of-range columns are skipped by the kernels. */
int lev_sketch_csr(lev_handle* h, const int64_t* row_ptr, const int32_t* col, const float* val,
                   int64_t n, int64_t d, int64_t nnz, const lev_params* p,
                   float* Atilde, void* stream);

/* Column-pivoted QR of the sketch in FP64 (Alg. 4 step 2, with the xGEQP3-style
 * pivoting of Sec. 7): at step j the remaining column with the largest trailing
 * norm (recomputed exactly, ties to the lowest original index) becomes column j;
 * the factorisation stops at the first j with |R_jj| <= tau |R_00| and
 * *rank = j (Sec. 7.2 rank check); diag(R) >= 0. Two routes give the same pivots,
 * rank and R (identical in exact arithmetic):
 *  - d <= 1024 and tau >= 1e-6: the Gram matrix A~^T A~ (products of the FP32
 *    entries exact, sums compensated to about FP64 accuracy), then a pivoted
 *    Cholesky factorisation of it in FP64 (the squared trailing norms of the QR
 *    are the diagonal of its Schur complements); R then agrees with the
 *    Householder R to about u kappa(R_11)^2 relative, and ranks are resolved down
 *    to about 1e-7 of |R_00|, hence the tau condition;
 *  - otherwise a column-pivoted Householder QR in FP64 on one cooperative grid.
 * Atilde: device, m x d FP32 row-major (ld = d). perm: device, d int32; entries
 * 0..r-1 are the pivots in order, r..d-1 the other columns in increasing order.
 * R: device, d x d FP64 row-major; rows 0..r-1 hold [R_11 R_12] in pivoted
 * column order, rows r..d-1 are zero. rank: host, may be NULL (then the call
 * does not synchronise). Errors: LEV_EINVAL, LEV_ENOMEM, LEV_ECUDA,
 * LEV_ETIMEOUT, LEV_ERANK0 (rank 0; perm = identity, R = 0). */
int lev_rrqr(lev_handle* h, const float* Atilde, int64_t m, int64_t d, double tau,
             int32_t* perm, double* R, int64_t* rank, void* stream);

/* The pivoted QR of A~ (as lev_rrqr) with the rank rule of p->flags, tau = p->tau:
 *  - no flag: the diagonal test of lev_rrqr;
 *  - LEV_RANK_SVD: the QR runs to the end (column order only) and the rank is the number of
 *    singular values of A~ above tau sigma_1 (Alg. 11 step 3; Sec. 7.2 advises the singular
 *    values where the diagonal of R misses a small gap), from a one-sided Jacobi SVD of R;
 *  - LEV_SRRQR: then strong-RRQR swaps at that rank (Alg. 2, Gu and Eisenstat): while the
 *    largest rho_ij = sqrt((R11^{-1} R12)_ij^2 + (gamma_j(R22) ||e_i^T R11^{-1}||)^2) exceeds
 *    p->phi (0 means 2), selected column i and unselected column j trade places; each swap
 *    re-factors through the Gram matrix of A~ and synchronises `stream` once.
 * perm, R, rank: as lev_rrqr (R rows < rank for the final columns). sigma: device, d doubles or
 * NULL: the singular values of A~, descending (LEV_RANK_SVD only). swaps: host or NULL: the
 * number of swaps. d <= 1024 with either flag. Errors: LEV_EINVAL (shapes, phi < 1, no
 * settling within 64 d swaps), LEV_ECUDA, LEV_ETIMEOUT, LEV_ERANK0. */
int lev_rrqr_select(lev_handle* h, const float* Atilde, int64_t m, int64_t d, const lev_params* p,
                    int32_t* perm, double* R, int64_t* rank, double* sigma, int64_t* swaps,
                    void* stream);

/* Diagnostics of the last lev_rrqr_select / LEV_RANK_SVD / LEV_SRRQR call on h: the strong-RRQR
 * swaps and the Jacobi sweeps (41 when the last of 40 sweeps still rotated). Synchronises the
 * device. Either pointer may be NULL. */
int lev_rank_stats(lev_handle* h, int64_t* swaps, int32_t* jacobi_sweeps);

/* Alg. 11 (CountGaussPrecondition) on dense A (device, n x d FP32, lda >= d): the CountGauss
 * sketch A~ = G S A with p's sizes, seed and sketch_prec, its SVD (the LEV_RANK_SVD path of
 * lev_rrqr_select), k = #{sigma_j > p->tau sigma_1}, and N = V_k Sigma_k^{-1} written to N (device,
 * d x d FP64, row-major; columns >= k are zero). By Theorem 8 (GSA preconditioning, Sec. 6.2)
 * kappa(A N) <= xi eta with high probability, whatever kappa(A) is. rank: host, may be NULL.
 * sigma: device d doubles or NULL (the sketch's singular values, descending). d <= 1024.
 * Synchronises `stream`. Errors: LEV_EINVAL, LEV_ENOMEM, LEV_ECUDA, LEV_ETIMEOUT, LEV_ERANK0. */
int lev_precondition_dense(lev_handle* h, const float* A, int64_t n, int64_t d, int64_t lda,
                           const lev_params* p, double* N, int64_t* rank, double* sigma,
                           void* stream);

/* The same on CSR A (device arrays, the conventions of lev_sketch_csr). */
int lev_precondition_csr(lev_handle* h, const int64_t* row_ptr, const int32_t* col, const float* val,
                         int64_t n, int64_t d, int64_t nnz, const lev_params* p, double* N,
                         int64_t* rank, double* sigma, void* stream);

/* LSQR (Paige and Saunders) on min_y ||A N y - b|| with A dense (device, n x d FP32, lda >= d), N
 * (device, d x d FP64 row-major, first k columns used, e.g. from lev_precondition_dense) and b
 * (device, n FP32); x = N y (device, d FP64), the minimum-norm least-squares solution A^+ b when N
 * comes from Alg. 11. Each iteration is one pass over A (A (N v) and A^T u' together) plus FP64
 * steps on d-vectors; the passes compute in FP32 with FP64 partial sums, so atol and btol much
 * below 1e-6 are not reached. Stops when ||(AN)^T r|| <= atol ||AN||_F ||r||, ||r|| <= btol ||b||,
 * or after max_iter iterations (atol, btol <= 0 mean 1e-6). iters, rnorm (host, may be NULL):
 * iterations run and the residual norm estimate. d <= 1024. Synchronises `stream` every 16
 * iterations. Errors: LEV_EINVAL, LEV_ENOMEM, LEV_ECUDA. */
int lev_lsqr_dense(lev_handle* h, const float* A, int64_t n, int64_t d, int64_t lda, const double* N,
                   int64_t k, const float* b, double* x, int32_t max_iter, double atol, double btol,
                   int32_t* iters, double* rnorm, void* stream);

/* The same on CSR A (device arrays, the conventions of lev_sketch_csr; columns outside [0, d) count
 * as zero). Each pass takes the rows of at most 8 entries four to a warp and the others a warp
 * each. A repeated column within a row adds through a shared-memory atomic, so its rounding order
 * (and x's last bits) may vary between runs; otherwise the sums run in a fixed order. */
int lev_lsqr_csr(lev_handle* h, const int64_t* row_ptr, const int32_t* col, const float* val,
                 int64_t n, int64_t d, int64_t nnz, const double* N, int64_t k, const float* b,
                 double* x, int32_t max_iter, double atol, double btol, int32_t* iters,
                 double* rnorm, void* stream);

/* The small factor of the final pass (Alg. 8 step 4 with the QR
 * orthogonaliser): M = R_11^{-1} Omega (r x k) by back-substitution (d <= 1024: in
 * double-float arithmetic, FP32 pairs of about 48 bits, on the FP64 R and Omega; above: FP64), with
 * Omega drawn from stream 3 of `seed` (or I_r with LEV_OMEGA_IDENTITY, k = r),
 * scattered into Mfull (device, d x k FP32 row-major): row perm[p] holds M[p, :]
 * and the d - r rows outside K are 0. R, perm as produced by lev_rrqr; d_rank:
 * device int64 holding r (read on the device, no host round trip).
 * With LEV_OMEGA_REDUCED (d <= 1024) and r < k, row perm[p] holds row p of
 * W = R_11^{-1} L_r in columns 0..r-1 and zeros after, where L_r (r x r, lower
 * triangular) is the Cholesky factor of Omega_r Omega_r^T, Omega_r the first r
 * rows of Omega. Then W W^T = M M^T, so every final pass gives the same
 * theta~_i = ||a_K,i M||^2 = ||a_K,i W||^2 up to rounding, and the dense
 * tensor-core final pass multiplies r columns instead of k. L_r is the leading
 * block of one factor per (seed, d, k) (Cholesky factors of leading blocks
 * nest), computed with Omega and kept by the handle. The estimate entry points
 * always take this form.
 * Errors: LEV_EINVAL, LEV_ECUDA. */
int lev_omega_factor(lev_handle* h, const double* R, const int32_t* perm, const int64_t* d_rank,
                     int64_t d, int64_t k, uint64_t seed, uint32_t flags,
                     float* Mfull, void* stream);

/* Fused final pass over dense A (Alg. 8 step 5): theta[i] = sum_q (A[i,:] Mfull[:, q])^2
 * for i < n; the n x k product is never written to memory. A: device n x d
 * FP32 (lda >= d); Mfull: device d x k FP32 row-major; theta: device n FP32.
 * prec: LEV_FP32 (SIMT), LEV_TF32, LEV_BF16 or LEV_BF16X3 (tensor cores).
 * Errors: LEV_EINVAL, LEV_ENOMEM, LEV_ECUDA. */
int lev_final_dense(lev_handle* h, const float* A, int64_t n, int64_t d, int64_t lda,
                    const float* Mfull, int64_t k, int32_t prec, float* theta, void* stream);

/* Fused final pass over CSR A: theta[i] = sum_q (sum_t val_t Mfull[col_t, q])^2
 * (Lemma 1, product form). Arrays as lev_sketch_csr; Mfull as lev_final_dense;
 * prec must be LEV_FP32. Errors: LEV_EINVAL, LEV_ENOMEM, LEV_ECUDA. */
int lev_final_csr(lev_handle* h, const int64_t* row_ptr, const int32_t* col, const float* val,
                  int64_t n, int64_t d, int64_t nnz, const float* Mfull, int64_t k,
                  int32_t prec, float* theta, void* stream);

/* The whole estimator (Alg. 10) on dense A: sketch, rrqr, omega_factor and the
 * final pass on one stream. A and theta may be device pointers or host
 * pointers (pageable or pinned). A host A is copied by the handle's own copy
 * stream into one of two device stage buffers that alternate between calls;
 * `stream` waits for that copy, and the copy of the next call waits only for
 * the kernels of the call that last used its buffer, so with pinned buffers
 * the copy of call i+1 overlaps the kernels of call i. A host theta is
 * copied back on `stream`. rank: host, may be NULL. The call synchronises
 * `stream` before it returns when rank is non-NULL, or when a buffer is on the
 * host, unless p->flags has LEV_HOST_ASYNC and rank is NULL: then it only
 * enqueues the work, the host A must stay unchanged and theta is valid once
 * `stream` has been synchronised, and a device-side timeout is reported by
 * lev_device_status instead of the return code. perm: device d int32, may be
 * NULL. Errors: any of the above. */
int lev_estimate_dense(lev_handle* h, const float* A, int64_t n, int64_t d, int64_t lda,
                       const lev_params* p, float* theta, int64_t* rank, int32_t* perm,
                       void* stream);

/* Alg. 7 (LS-HRN-exact) on dense A: the columns K and the rank k come from the
 * pivoted QR of the CountGauss sketch (as in lev_estimate_dense, with p's sizes,
 * tau, seed and sketch_prec); then B = A_K^T A_K in FP64 (Lemma 8, Sec. 5.1: the Gram
 * matrix of A, products of the FP32 entries exact, sums in FP64, restricted to K
 * in pivot order), its Cholesky factor B = R^T R (step 5 asks for the SVD
 * B = V Sigma^2 V^T; both give theta_i = a_K B^{-1} a_K^T, B being positive
 * definite), and theta_i = ||A_{i,K} R^{-1}||^2 with the final pass of
 * p->final_prec (tensor-core forms need d <= 256); d <= 1024. If the Cholesky meets a
 * non-positive pivot before k steps, *rank is the number of steps taken.
 * A, theta: device. perm: device d int32 or NULL (the pivots of the sketch's QR).
 * rank: host, may be NULL; the call synchronises `stream` twice (after each
 * factorisation). Errors: as lev_estimate_dense; LEV_ERANK0 sets theta to 0. */
int lev_exact_dense(lev_handle* h, const float* A, int64_t n, int64_t d, int64_t lda,
                    const lev_params* p, float* theta, int64_t* rank, int32_t* perm,
                    void* stream);

/* Alg. 7 (LS-HRN-exact) on CSR A (row_ptr: n + 1 int64; col: nnz int32; val: nnz FP32; all
 * device; the CSR conventions of lev_sketch_csr): K and k from the pivoted QR of the CountSketch
 * + Gaussian sketch, then B = A_K^T A_K as the sum of the rows' outer products (Lemma 8, Sec. 5.1: products
 * of the FP32 entries exact; rows of at most max(32, d/5) entries summed by FP64 atomics, longer
 * rows densified and summed by the compensated dense Gram kernel, so the last bits of B and of
 * theta may differ between runs), its Cholesky factor B = R^T R with the pivots forced, and
 * theta_i = ||A_{i,K} R^{-1}||^2 by the CSR final pass (LEV_FP32 only); d <= 1024.
 * theta: device n. perm: device d int32 or NULL. rank: host, may be NULL; the call synchronises
 * `stream` three times. Errors: as lev_estimate_csr; LEV_ERANK0 sets theta to 0. */
int lev_exact_csr(lev_handle* h, const int64_t* row_ptr, const int32_t* col, const float* val,
                  int64_t n, int64_t d, int64_t nnz, const lev_params* p, float* theta,
                  int64_t* rank, int32_t* perm, void* stream);

/* Exact leverage scores of A itself (Sec. 1: theta_i = diag(A (A^T A)^+ A^T)_i, the squared row norms
 * of an orthonormal basis of range(A)), by the Gram route of Alg. 5 with the QR orthogonaliser: the
 * Gram matrix A^T A (products of the FP32 entries exact, sums compensated to about FP64 accuracy),
 * its pivoted Cholesky factorisation in FP64 (the pivots, rank and R of a column-pivoted QR of A in
 * exact arithmetic; rank rule |R_jj| > tau |R_00| of Sec. 7.2), and theta_i = ||A_{i,K} R_11^{-1}||^2
 * by the FP32 final pass. No sketch and no Omega: the reference the estimator approximates.
 * A: device, n x d FP32 (lda >= d); theta: device, n FP32. perm: device d int32 or NULL (the
 * columns K in pivot order first). rank: host, may be NULL; the call synchronises `stream` once.
 * d <= 1024; tau >= 1e-6 (the Gram route resolves |R_jj| / |R_00| down to about 1e-7; tau <= 0
 * means 1e-5). Errors: LEV_EINVAL, LEV_ENOMEM, LEV_ECUDA, LEV_ETIMEOUT, LEV_ERANK0 (theta = 0). */
int lev_exact_reference_dense(lev_handle* h, const float* A, int64_t n, int64_t d, int64_t lda, double tau,
                              float* theta, int64_t* rank, int32_t* perm, void* stream);

/* The same for CSR A (device arrays, the conventions of lev_sketch_csr): A^T A as the sum of the
 * rows' outer products (Lemma 8, Sec. 5.1; rows of more than max(32, d / 5) entries densified and
 * summed by the compensated dense kernel, the others by FP64 atomics, so the last bits of A^T A and
 * theta may differ between runs), then the pivoted Cholesky and the CSR final pass. The call
 * synchronises `stream` twice (the count of long rows, the rank). */
int lev_exact_reference_csr(lev_handle* h, const int64_t* row_ptr, const int32_t* col, const float* val,
                            int64_t n, int64_t d, int64_t nnz, double tau, float* theta, int64_t* rank,
                            int32_t* perm, void* stream);

/* The whole estimator on CSR A (arrays as lev_sketch_csr, device or host). */
int lev_estimate_csr(lev_handle* h, const int64_t* row_ptr, const int32_t* col, const float* val,
                     int64_t n, int64_t d, int64_t nnz, const lev_params* p,
                     float* theta, int64_t* rank, int32_t* perm, void* stream);

/* Gradient of g(A) = sum_i w_i theta~_i(A) with respect to dense A, with the
 * sketch S, G, Omega, the pivots and the rank held at the values of a forward
 * pass. The paper has no backward pass; this is the reverse-mode adjoint of
 * Alg. 10 (QR adjoint with a zero Q cotangent): with Y = A_K M, Z = 2 W Y,
 * C = A_K^T Z, Rbar = -R_11^{-T} C M^T, Xbar = Q_1 copyltu(R_11 Rbar^T) R_11^{-T}
 * and T = G^T Xbar, row i of the gradient on the columns of K is
 * Z_i M^T + sigma_i T[h(i), :]; the columns outside K are 0. With
 * LEV_SKETCH_SRHT in p->flags (the sketch G F S A), T = F^T G^T Xbar with
 * F^T = D H P^T / sqrt(t): the t drawn rows scattered back (repeated draws
 * added in draw order), the Walsh-Hadamard butterflies, the signs. The n x k
 * intermediate Y is recomputed in both passes, never stored.
 * The forward state is passed explicitly (all device pointers), as produced by
 * lev_sketch_dense / lev_rrqr / lev_omega_factor with the same p: Atilde
 * (m x d FP32), perm (d int32), d_rank (int64), R (d x d FP64), Mfull (d x k
 * FP32). A: n x d FP32 (lda); w: n FP32 (= dL/dtheta~); gradA: n x d FP32
 * (ld = d). Limits: d <= 256, k <= 256. Errors: LEV_EINVAL, LEV_ENOMEM, LEV_ECUDA. */
int lev_backward_dense(lev_handle* h, const float* A, int64_t n, int64_t d, int64_t lda,
                       const lev_params* p, const float* Atilde, const int32_t* perm,
                       const int64_t* d_rank, const double* R, const float* Mfull,
                       const float* w, float* gradA, void* stream);

/* Fault injection for tests of the error paths (host side only; nothing is injected on the
 * device): with the environment variable LEV_FAULT set to "alloc" every scratch allocation that a
 * call needs reports failure (LEV_ENOMEM), to "launch" the launch of the pivoted QR reports failure
 * (LEV_ECUDA), to "timeout" the status read after a synchronisation reports an expired device wait
 * (LEV_ETIMEOUT), and to "pivwait" the pivoted Cholesky of the Gram route never publishes the pivot
 * column of its second step: the other CTAs' bounded waits for it run out (about a second each), the
 * kernel records the timeout in the status word and returns, and the call reports LEV_ETIMEOUT. Unset,
 * it costs one getenv per such point. */

/* Device-side status word of the handle: nonzero after a bounded wait gave up. */
int lev_device_status(lev_handle* h, int32_t* status);

/* Diagnostics (no counterpart in the paper). With timing on (enable != 0) every pivoted QR of
 * the handle (lev_rrqr and the rrqr stage of lev_estimate_*) records CUDA events on its stream
 * before the factorisation, after the Gram product with its reduction (Gram route; nothing
 * runs before the factorisation kernel on the Householder route) and after the factorisation
 * kernel (the grid pivoted Cholesky, or the Householder kernel). lev_rrqr_timing waits for the
 * events of the last such call and returns the two durations in milliseconds; either output
 * pointer may be NULL. Errors: LEV_EINVAL (timing off, or no QR since it was enabled),
 * LEV_ECUDA. The tensor-core dense final pass (lev_final_dense with LEV_TF32, LEV_BF16 or
 * LEV_BF16X3, and the final stage of lev_estimate_dense) likewise records events around its
 * main kernel, after the packing of Mfull's operand image; lev_final_timing waits for those of
 * the last such call and returns the kernel's duration. */
int lev_set_timing(lev_handle* h, int enable);
int lev_rrqr_timing(lev_handle* h, float* gram_ms, float* factor_ms);
int lev_final_timing(lev_handle* h, float* kernel_ms);

/* lev_rrqr without any allocation. The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc -- code that lives inside
 * another allocator's fixed memory budget (for example a serving framework's
 * pool) and latency-critical paths that cannot afford the implicit device
 * synchronisation of cudaMalloc/cudaFree. It computes exactly what lev_rrqr
 * computes (same kernels, same arguments and results; no handle), on the
 * calling thread's current device, with its scratch in a fixed 8 MiB device
 * array that every GPU which loads the library holds until the process exits.
 * Limit: the QR working set must fit in 8 MiB: about 8 (m d + 3 d^2) bytes plus,
 * on the Gram route (lev_rrqr), the Gram matrix's partial sums (at most 4 MiB;
 * their count follows the device's SM count, so a shape near the limit may be
 * accepted on one GPU model and rejected on another). For example m = 1024,
 * d = 256 fits. Larger shapes return LEV_EINVAL.
 * The first call in a CUDA context (and the first after the current context
 * changed, e.g. after cudaDeviceReset) looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * Every call clears what must start at zero; all calls share the one array,
 * so calls that overlap on the GPU (different streams, or different host
 * threads) race and give wrong results. rank: host, may be NULL; with a rank
 * pointer the call reads the rank into host memory and synchronises `stream`,
 * without one it only enqueues the work. Errors: LEV_EINVAL, LEV_ECUDA,
 * LEV_ETIMEOUT, LEV_ERANK0. */
int lev_rrqr_noalloc(const float* Atilde, int64_t m, int64_t d, double tau,
                     int32_t* perm, double* R, int64_t* rank, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LEV_H */
