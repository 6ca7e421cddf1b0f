// Host-side launch functions of the CUDA kernels (one .cu file per stage).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace lev {

// ---- sketch.cu: hash, bucket permutation, CountSketch, G, Gaussian stage ----

// Bucket permutation of rows 0..n-1 (counting sort by h(i), rows ascending in
// each bucket). count: s+1 ints (scratch), off: s+1 ints (out), tmp and perm:
// n uint32 each (perm out). A perm entry is row | (sign < 0) << 31.
cudaError_t launch_bucket_perm(int64_t n, int64_t s, uint64_t seed, int64_t row0, int* count, int* off,
                               uint32_t* tmp, uint32_t* perm, cudaStream_t st);

// B (s x d, ld = d, FP32) = S A for dense A (n x d, lda).
cudaError_t launch_countsketch_dense(const float* A, int64_t lda, int64_t d, int64_t s,
                                     const int* off, const uint32_t* perm, float* B, cudaStream_t st);

// The same B = S A written as the K-major BF16 operand of the tensor-core Gaussian stage, blocked by
// 64 buckets (img[g][c][k] = B[64 g + k][c], g < ld / 64, buckets s..ld zero): hi = bf16(B) and,
// when lo is not null, lo = bf16(B - hi). cudaErrorNotSupported when A, lda or d do not allow
// 16-byte loads, d > 1024, or ld is not a multiple of 64 at least s (the caller then writes B).
cudaError_t launch_countsketch_dense_op(const float* A, int64_t lda, int64_t d, int64_t s, int64_t ld,
                                        const int* off, const uint32_t* perm, __nv_bfloat16* hi, __nv_bfloat16* lo,
                                        cudaStream_t st);

// B (s x d, ld = d, FP32) = S A for CSR A.
cudaError_t launch_countsketch_csr(const int64_t* row_ptr, const int32_t* col, const float* val,
                                   int64_t d, int64_t s, const int* off, const uint32_t* perm,
                                   float* B, cudaStream_t st);

// G[j, b] = N_{j s + b} / sqrt(m) (m x s, N the counter draws of stream 2) as an image with leading
// dimension ld >= s (columns s..ld zero). form 0: g32 = fl32(N / sqrt(m)); form 1: g32 = the TF32
// rounding of fl32(N), unscaled; form 2: ghi = bf16(fl32(N)) and ghi + m ld = bf16(fl32(N) - hi),
// unscaled.
cudaError_t launch_gen_gaussian(int64_t m, int64_t s, int64_t ld, uint64_t seed, float* g32, int form,
                                __nv_bfloat16* ghi, cudaStream_t st);

// Atilde (m x d) = G (m x s) B (s x d), FP32 SIMT, split-K with a fixed-order
// reduction. partial: splits * m * d floats of scratch; returns splits used.
int gaussian_stage_splits(int64_t m, int64_t d, int64_t s);
cudaError_t launch_gaussian_stage_fp32(const float* G, const float* B, int64_t m, int64_t s,
                                       int64_t d, float* partial, int splits, float* Atilde,
                                       cudaStream_t st);

// CSR structure check: *bad |= 1 (row_ptr[0] != 0), 2 (row_ptr decreases), 4 (row_ptr[n] != nnz).
cudaError_t launch_check_csr(const int64_t* row_ptr, int64_t n, int64_t nnz, int32_t* bad, cudaStream_t st);

// Identity sketch: Atilde = A (n x d) copied densely (ld = d).
cudaError_t launch_copy_dense(const float* A, int64_t lda, int64_t n, int64_t d, float* out,
                              cudaStream_t st);

// ---- qr.cu: pivoted QR (FP64), omega factor ----

struct QrScratch {
    double* W;        // m x d FP64, column-major (ld = m)
    double* norms;    // 2 x d FP64 (double-buffered trailing norms^2)
    double* Rorig;    // d x d FP64: row j, original column c
    int32_t* piv;     // d int32: pivot order (original column ids)
    int64_t* rank;    // 1 int64 (device)
    unsigned* barrier;  // 1 uint32 grid-barrier counter
    double* G;        // d x d FP64 Gram matrix (Gram route)
    double* Gp;       // split partials of the Gram matrix (Gram route)
    double* U;        // d x d FP64: unscaled pivot rows exchanged by the grid pivoted Cholesky (Gram route)
};

// C (t x d) = F B with the SRHT F = sqrt(s/t) P H D (srht.cu); B (s x d, s a power of two) is
// overwritten with H' D B, H' the unscaled Walsh-Hadamard matrix.
cudaError_t launch_srht(float* B, int64_t s, int64_t d, int64_t t, uint64_t seed, float* C, cudaStream_t st);
// X (s x d) = F^T Y for Y (t x d): D H' P^T Y / sqrt(t), the adjoint of launch_srht's F. The drawn rows of
// each row of s are added in increasing draw order (bit-reproducible). count, off: s + 1 int each;
// tmp, ord: t uint32 each.
cudaError_t launch_srht_adjoint(const float* Y, int64_t s, int64_t d, int64_t t, uint64_t seed, int* count, int* off,
                                uint32_t* tmp, uint32_t* ord, float* X, cudaStream_t st);
// The exclusive scan and the per-segment rank sort of the bucket permutation (sketch.cu).
cudaError_t launch_scan_offsets(const int* count, int* off, int64_t s, cudaStream_t st);
cudaError_t launch_segment_sort(const int* off, int64_t s, const uint32_t* in, uint32_t* out, cudaStream_t st);

// Gram route of the pivoted QR (gramqr.cu): G = A~^T A~ in FP64, then a
// pivoted Cholesky on one cooperative grid; fills Rorig, piv and rank.
int gram_splits(int64_t m, int64_t d);
size_t gram_partial_doubles(int64_t m, int64_t d);
// G (d x d FP64, both triangles) = A^T A for A (m x d FP32, leading dimension lda); Gp holds
// gram_partial_doubles(m, d) doubles of split partials.
cudaError_t launch_gram_fp64(const float* A, int64_t lda, int64_t m, int64_t d, double* Gp, double* G,
                             cudaStream_t st);
// G (d x d FP64, both triangles) = A^T A for CSR A (n rows) by the rows' outer products, FP64
// atomics (the order of the sums varies between runs).
cudaError_t launch_gram_csr_fp64(const int64_t* row_ptr, const int32_t* col, const float* val, int64_t n,
                                 int64_t d, double* G, cudaStream_t st);
// The same over the rows of at most max_len entries, plus Gheavy (d x d FP64 upper, may be null):
// the Gram of the longer rows formed densely. launch_heavy_rows lists the longer rows (count on
// the device); launch_densify_rows writes them as an nh x d FP32 matrix.
cudaError_t launch_gram_csr_light(const int64_t* row_ptr, const int32_t* col, const float* val, int64_t n, int64_t d,
                                  int64_t max_len, const double* Gheavy, double* G, cudaStream_t st);
cudaError_t launch_heavy_rows(const int64_t* row_ptr, int64_t n, int64_t max_len, unsigned long long* count,
                              int32_t* idx, cudaStream_t st);
cudaError_t launch_densify_rows(const int64_t* row_ptr, const int32_t* col, const float* val, const int32_t* idx,
                                const unsigned long long* count, int64_t nh, int64_t d, float* H, cudaStream_t st);
// LEV_FAULT=pivwait is set (api.cu): the pivoted Cholesky withholds the pivot column of step 1.
bool fault_pivot_wait();
// The grid pivoted Cholesky of q.G (rank test as lev_rrqr's with min(m, d) steps; forced pivots
// optional): fills q.Rorig, q.piv, q.rank.
cudaError_t launch_pivoted_cholesky(int64_t m, int64_t d, double tau, const int32_t* forced, int64_t forced_rank,
                                    const QrScratch& q, int32_t* status, cudaStream_t st);
// R (d x d FP64, pivoted order) and perm of a pivoted Cholesky of the Gram matrix already in q.G
// (forced pivots optional); the output conventions of launch_pivoted_qr.
cudaError_t launch_factor_gram(int64_t m, int64_t d, double tau, const int32_t* forced, int64_t forced_rank,
                               const QrScratch& q, int32_t* perm, double* R, int32_t* status, cudaStream_t st);
cudaError_t launch_gram_pivoted_cholesky(const float* Atilde, int64_t m, int64_t d, double tau,
                                         const int32_t* forced, int64_t forced_rank, const QrScratch& q,
                                         int32_t* status, cudaStream_t st, cudaEvent_t after_gram = nullptr);
size_t qr_scratch_bytes(int64_t m, int64_t d);

// Rank decisions (rank.cu). launch_svd_rank: sigma (d, descending) of the first *d_rows rows of R
// (d x d, d <= 1024) by one-sided Jacobi in double-float arithmetic on a split copy Yhl (2 d^2
// FP32), joined back into Y (d x d FP64); order[j] = the row of Y holding
// sigma_j (its normalised row is the right singular vector), *rank_out = #{sigma_j > tau sigma_1};
// work: 64 uint32 zeroed here. launch_srrqr_step: one strong-RRQR step at fixed k from R (k rows
// of the forced factor, pivot order), Rs (R11 scaled and transposed), G (the Gram matrix): out =
// {rho^2, i, j} of the largest rho, and perm[i] <-> perm[j] when rho > phi.
size_t rank_scratch_doubles(int64_t d);
cudaError_t launch_svd_rank(const double* R, const int64_t* d_rows, int64_t d, double tau, double* Y, float* Yhl,
                            unsigned* work, double* sigma, int32_t* order, int64_t* rank_out, int32_t* sweeps_out,
                            unsigned* version, int32_t* status, int num_sms, cudaStream_t st);
cudaError_t launch_srrqr_step(const double* R, const double* Rs, const double* G, int32_t* perm, int64_t d, int64_t k,
                              double phi, double* Z, double* wn, double* g2, double* part_v, long long* part_e,
                              double* out, cudaStream_t st);
cudaError_t launch_scaled_transpose(const double* R, const int64_t* d_rank, int64_t d, double* Rs, cudaStream_t st);

// Preconditioning and LSQR (lsqr.cu). launch_precond_n: N (d x d FP64, row-major; columns >= k
// zero) = V_k Sigma_k^{-1} from the Jacobi rows Y, order and sigma of launch_svd_rank and the
// pivots perm. launch_lsqr: LSQR on min ||A N y - b|| with u holding b on entry (overwritten), x =
// N y (d FP64); ws: lsqr_scratch_doubles(d, parts) doubles; host_state: pinned, lsqr_state_doubles().
size_t lsqr_scratch_doubles(int64_t d, int parts);
int lsqr_parts(int num_sms);
int lsqr_state_doubles();
cudaError_t launch_precond_n(const double* Y, const int32_t* order, const double* sigma, const int32_t* perm,
                             const int64_t* d_rank, int64_t d, double* N, cudaStream_t st);
// A dense (A, lda) or CSR (row_ptr, col, val; A == nullptr).
cudaError_t launch_lsqr(const float* A, int64_t lda, const int64_t* row_ptr, const int32_t* col, const float* val,
                        int64_t n, int64_t d, const double* N, int64_t k, float* u,
                        double* x, int max_iter, double atol, double btol, double* ws, int parts, double* host_state,
                        int* iters_out, double* rnorm_out, cudaStream_t st);
void qr_scratch_carve(void* base, int64_t m, int64_t d, QrScratch* q);

// Pivoted QR of Atilde (m x d FP32 row-major). forced_perm may be null. marks (optional, three
// events): recorded before the factorisation, after the Gram product (Gram route; at the start
// on the Householder route) and after the factorisation kernel.
// Writes perm (d), R (d x d row-major), d_rank. status: device status word.
cudaError_t launch_pivoted_qr(const float* Atilde, int64_t m, int64_t d, double tau,
                              const int32_t* forced_perm, int64_t forced_rank,
                              const QrScratch& q, int32_t* perm, double* R, int32_t* status,
                              int num_sms, cudaStream_t st,
                              const cudaEvent_t* marks = nullptr);

// Mfull (d x k FP32) = scatter of R_11^{-1} Omega by perm; reads r from d_rank. Omega: d x k FP64
// from launch_gen_omega (unused with omega_identity); Rs: d x d FP64 scratch. With d > 1024 or
// without Rs the one-warp-per-column kernel runs and draws Omega itself. Lc (optional): the
// factor of launch_omega_chol (kc x kc, its rank at d_kc); when r < k and r <= *d_kc, column q < r
// of Mfull is R_11^{-1} times column q of L_r instead (L_r L_r^T = Omega_r Omega_r^T, Omega_r the
// first r rows), the columns q >= r stay 0, and Mfull Mfull^T is unchanged.
cudaError_t launch_omega_factor(const double* R, const int32_t* perm, const int64_t* d_rank,
                                int64_t d, int64_t k, uint64_t seed, bool omega_identity,
                                const double* Omega, const double* Lc, int64_t kc, const int64_t* d_kc,
                                double* Rs, float* Mfull, cudaStream_t st);
// The Cholesky factor of Omega_kc Omega_kc^T (kc = min(d, k) leading rows of Omega): the Gram
// product in FP64 into q.G, then the grid pivoted Cholesky with the pivots forced to 0, 1, ...
// (iota: kc int32 scratch). Leaves the upper factor U (U^T U = Omega_kc Omega_kc^T) in q.Rorig
// (row j, column i >= j; ld = kc) and the number of steps taken in q.rank. q: scratch for (k, kc).
cudaError_t launch_omega_chol(const double* Omega, int64_t d, int64_t k, const QrScratch& q, int32_t* iota,
                              int32_t* status, cudaStream_t st);
// Omega (d x k FP64) of stream 3 of seed, every pivot position p < d.
cudaError_t launch_gen_omega(uint64_t seed, int64_t d, int64_t k, double* Omega, cudaStream_t st);

// ---- backward.cu: gradient of sum_i w_i theta~_i ----
// srht_t > 0: the sketch had the SRHT to srht_t rows after the CountSketch (G is m x srht_t and the
// G image's columns are srht_t); 0: plain CountGauss.

int backward_chunks(int64_t n, int64_t d, int64_t k);
size_t backward_scratch_bytes(int64_t n, int64_t d, int64_t k, int64_t s, int64_t m, int64_t srht_t, int chunks);
cudaError_t launch_backward_dense(const float* A, int64_t lda, int64_t n, int64_t d, int64_t s, int64_t m, int64_t k,
                                  uint64_t seed, const float* Atilde, const int32_t* perm, const int64_t* d_rank,
                                  const double* R, const float* Mfull, const float* w, const float* G32,
                                  const __nv_bfloat16* Ghi, int64_t ldg, float g_scale, bool identity,
                                  int64_t srht_t, void* scratch, int chunks, float* gradA, cudaStream_t st);

// ---- final.cu: fused final pass (SIMT) ----

cudaError_t launch_final_dense_fp32(const float* A, int64_t lda, int64_t n, int64_t d,
                                    const float* Mfull, int64_t k, float* theta, cudaStream_t st);
// CSR final pass in the second form of Lemma 1 for rows of at most 32 entries (theta~ = a P a^T,
// P = Mfull Mfull^T in FP64 built here from Mfull) and the first form for longer rows; scratch:
// csr_gram_scratch_bytes(d, k). csr_gram_pays: whether the second form is the cheaper one.
size_t csr_gram_scratch_bytes(int64_t d, int64_t k);
bool csr_gram_pays(int64_t n, int64_t d, int64_t nnz, int64_t k);
cudaError_t launch_final_csr_gram(const int64_t* row_ptr, const int32_t* col, const float* val, int64_t n, int64_t d,
                                  const float* Mfull, int64_t k, void* scratch, float* theta, cudaStream_t st);
cudaError_t launch_final_csr_fp32(const int64_t* row_ptr, const int32_t* col, const float* val,
                                  int64_t n, int64_t d, const float* Mfull, int64_t k,
                                  float* theta, cudaStream_t st);

}  // namespace lev
