// C ABI of the leverage-score library: handle, scratch, argument checks and
// the composition of the stages of Alg. 10 (see include/lev.h).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

#include "lev_common.cuh"
#include "lev_kernels.cuh"
#include "lev_tc.cuh"

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

#define LEV_CUDA(call)                                                                         \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(e_ == cudaErrorMemoryAllocation ? LEV_ENOMEM : LEV_ECUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                    \
    } while (0)

// Fault injection for the tests of the error paths, chosen on the host: LEV_FAULT=alloc makes the
// next scratch allocation report failure, LEV_FAULT=launch the launch of the pivoted QR,
// LEV_FAULT=timeout the read of the device status word after a synchronisation, and
// LEV_FAULT=pivwait has the pivoted Cholesky withhold one published pivot column, so that the
// bounded waits for it run out on the device (no trap, no fault: the kernels record the timeout in
// the status word and return).
bool fault_is(const char* kind) {
    const char* f = getenv("LEV_FAULT");
    return f && strcmp(f, kind) == 0;
}

#define LEV_TRY(expr)              \
    do {                           \
        int rc_ = (expr);          \
        if (rc_ != LEV_OK) return rc_; \
    } while (0)

struct Buf {
    void* ptr = nullptr;
    size_t bytes = 0;
};

struct GCache {
    void* ptr = nullptr;
    size_t bytes = 0;
    uint64_t seed = 0;
    int64_t m = -1, s = -1;
    int kind = -1;   // 0: FP32 Z/sqrt(m) (ld = s); 2: Z in BF16 (ld = s rounded up to 64); 3: Z in FP32 (ld)
};

}  // namespace

struct lev_handle {
    int device = 0;
    int num_sms = 0;
    int32_t* status = nullptr;      // device status word
    int64_t* host_rank = nullptr;   // pinned
    Buf count, off, tmp, perm_rows, B, partial, Atilde, qr, R, perm_d, Mfull, stageTheta,
        tc_ws, tc_ws2, csr_rp, csr_col, csr_val, bwd;
    GCache g;
    // the CountSketch bucket permutation (off, perm_rows) of the last (seed, n, s), and an event
    // recorded after it was built so that a call on another stream waits for it
    // diagnostics: events around the Gram product and the factorisation of the last rrqr
    bool timing = false, timed_once = false, final_timed = false;
    cudaEvent_t tmark[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t fmark[2] = {nullptr, nullptr};   // around the tensor-core final pass kernel
    uint64_t perm_seed = 0;
    int64_t perm_n = -1, perm_s = -1, perm_row0 = 0;
    cudaEvent_t ev_perm = nullptr;
    // Omega (d x k FP64) of the last (seed, d, k), with its event, and the R_11 scratch of the solve
    Buf omega, omega_rs;
    uint64_t omega_seed = 0;
    int64_t omega_d = -1, omega_k = -1;
    cudaEvent_t ev_omega = nullptr;
    // the Cholesky factor of Omega's Gram matrix (launch_omega_chol scratch and its forced pivots),
    // valid for the cached Omega when omega_chol_ok
    Buf omega_chol;
    bool omega_chol_ok = false;
    // host A of lev_estimate_dense: two stage buffers filled by a copy stream of the handle
    Buf stageA[2];
    Buf exact_gp;  // split partials of the Gram matrix of A (LS-HRN-exact)
    Buf srht_c;    // F (S A), t x d (LEV_SKETCH_SRHT)
    Buf rank_ws;   // Jacobi copy of R, strong-RRQR Z, norms and argmax partials (LEV_RANK_SVD, LEV_SRRQR)
    int64_t last_swaps = 0;
    int64_t rank_ws_d = 0;   // d of the last carve of rank_ws
    Buf csr_p;     // CSR final pass, second form of Lemma 1: P = Mfull Mfull^T (FP64), Gram partials, Mfull^T
    Buf csr_heavy; // Alg. 7 on CSR: count and indices of the long rows
    Buf csr_dense; // Alg. 7 on CSR: the long rows densified, their Gram partials and Gram matrix
    Buf lsqr_u;    // LSQR: the unnormalised left vector u (n FP32)
    Buf lsqr_ws;   // LSQR: state, short vectors, pass partials, N^T
    double* host_lsqr = nullptr;   // pinned LSQR state read back by the host
    Buf tc_pad;   // A copied with a 16-byte row stride when the caller's cannot feed TMA
    cudaStream_t copy_st = nullptr;
    cudaEvent_t ev_copied[2] = {nullptr, nullptr}, ev_used[2] = {nullptr, nullptr};
    bool used_once[2] = {false, false};
    int stage_next = 0;
};

namespace {

// Every scratch buffer of a handle: the one list that lev_destroy releases and lev_workspace_bytes
// counts.
template <class F>
void for_each_buf(lev_handle* h, F f) {
    Buf* all[] = {&h->count, &h->off, &h->tmp, &h->perm_rows, &h->B, &h->partial, &h->Atilde, &h->qr,
                  &h->R, &h->perm_d, &h->Mfull, &h->stageA[0], &h->stageA[1], &h->stageTheta, &h->tc_ws, &h->tc_ws2,
                  &h->bwd, &h->csr_rp, &h->csr_col, &h->csr_val, &h->omega, &h->omega_rs, &h->omega_chol, &h->tc_pad,
                  &h->exact_gp, &h->srht_c, &h->rank_ws, &h->lsqr_u, &h->lsqr_ws, &h->csr_p, &h->csr_heavy,
                  &h->csr_dense};
    for (Buf* b : all) f(*b);
}

int ensure(Buf& b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return LEV_OK;
    if (b.ptr) {
        cudaError_t e = cudaFree(b.ptr);
        b.ptr = nullptr;
        b.bytes = 0;
        if (e != cudaSuccess) return fail(LEV_ECUDA, "cudaFree: %s", cudaGetErrorString(e));
    }
    if (fault_is("alloc")) return fail(LEV_ENOMEM, "cudaMalloc(%zu bytes) failed (injected by LEV_FAULT=alloc)", bytes);
    cudaError_t e = cudaMalloc(&b.ptr, bytes);
    if (e != cudaSuccess) {
        b.ptr = nullptr;
        cudaGetLastError();
        return fail(LEV_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
    }
    b.bytes = bytes;
    return LEV_OK;
}

void release(Buf& b) {
    if (b.ptr) cudaFree(b.ptr);
    b.ptr = nullptr;
    b.bytes = 0;
}

int set_device(lev_handle* h) {
    if (!h) return fail(LEV_EINVAL, "handle is NULL");
    LEV_CUDA(cudaSetDevice(h->device));
    return LEV_OK;
}

bool is_host_pointer(const void* p) {
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

struct Sizes {
    int64_t s, m, k;
    int64_t row0;  // global index of local row 0 (hash and sign of a row shard)
};

// Sizes of a call with (p, n, d). Only the sketch entry points take a row shard (row0, n_total):
// every other entry point sums over all rows of A itself, so it rejects them.
int resolve(const lev_params* p, int64_t n, int64_t d, Sizes* z, bool shard_ok = false) {
    if (!p) return fail(LEV_EINVAL, "params is NULL");
    if (n < 1 || n >= (int64_t)1 << 31) return fail(LEV_EINVAL, "n = %lld out of range [1, 2^31)", (long long)n);
    if (d < 1 || d > 4096) return fail(LEV_EINVAL, "d = %lld out of range [1, 4096]", (long long)d);
    if ((p->row0 != 0 || p->n_total != 0) && !shard_ok)
        return fail(LEV_EINVAL, "row0 / n_total (a row shard) are read by lev_sketch_* and lev_resolve_sizes only");
    if (p->row0 < 0 || p->n_total < 0 || p->n_total >= (int64_t)1 << 62 ||
        (p->n_total != 0 && p->row0 > p->n_total - n))
        return fail(LEV_EINVAL, "row shard [%lld, %lld) outside n_total = %lld", (long long)p->row0,
                    (long long)(p->row0 + n), (long long)p->n_total);
    if ((p->flags & LEV_SKETCH_IDENTITY) && (p->row0 != 0 || p->n_total != 0))
        return fail(LEV_EINVAL, "LEV_SKETCH_IDENTITY takes no row shard");
    const int64_t n_all = p->n_total != 0 ? p->n_total : n;   // k from the rows of the whole matrix
    const double eps = p->eps, delta = p->delta;
    int64_t s = p->s, m = p->m, k = p->k;
    if (s == 0) {
        if (!(eps > 0 && eps < 1 && delta > 0 && delta < 1)) return fail(LEV_EINVAL, "eps, delta must be in (0,1)");
        const double t = 2 * eps - eps * eps;
        s = (int64_t)std::ceil(((double)d * d + d) / (t * t * delta));
    }
    if (m == 0) {
        if (!(p->gamma > 0)) return fail(LEV_EINVAL, "gamma must be > 0");
        m = (int64_t)std::ceil(p->gamma * (double)d);
    }
    if (k == 0) {
        if (!(eps > 0 && eps < 1)) return fail(LEV_EINVAL, "eps must be in (0,1)");
        k = (int64_t)std::ceil(4.0 * std::log((double)(n_all > 1 ? n_all : 2)) / (eps * eps / 2 - eps * eps * eps / 3));
    }
    if (p->flags & LEV_SKETCH_IDENTITY) {
        s = n;
        m = n;
        if (n > 65536) return fail(LEV_EINVAL, "LEV_SKETCH_IDENTITY needs n <= 65536");
    }
    if (p->flags & LEV_OMEGA_IDENTITY) k = d;
    if (s < 1 || s >= (int64_t)1 << 31) return fail(LEV_EINVAL, "s = %lld out of range [1, 2^31)", (long long)s);
    if (m < 1 || m > (int64_t)1 << 20) return fail(LEV_EINVAL, "m = %lld out of range [1, 2^20]", (long long)m);
    if (k < 1 || k > 4096) return fail(LEV_EINVAL, "k = %lld out of range [1, 4096]", (long long)k);
    if ((double)m * (double)s > 8.0e9) return fail(LEV_EINVAL, "m * s = %.3g too large", (double)m * s);
    z->s = s;
    z->m = m;
    z->k = k;
    z->row0 = p->row0;
    return LEV_OK;
}

int check_prec(int32_t prec, const char* what) {
    if (prec < LEV_FP32 || prec > LEV_BF16X3) return fail(LEV_EINVAL, "%s precision %d unknown", what, prec);
    return LEV_OK;
}

double tau_of(const lev_params* p) { return p->tau > 0 ? p->tau : 1e-5; }

// Make sure G (m x s) for (seed, kind) is in the cache; returns its pointers.
// G = N / sqrt(m) with N the FP64 counter draws. Kind 0: FP32 entries fl32(N / sqrt(m)), leading
// dimension s. Kind 2: the BF16 pair of fl32(N), hi then lo (two m x ld images, ld = s rounded up
// to 64: TMA rows of whole 128-byte lines); the tensor-core stage applies 1 / sqrt(m) in its
// reduction. Kind 3: the TF32 rounding of fl32(N) in FP32 words, same padded leading dimension,
// same deferred scale.
int ensure_g(lev_handle* h, int64_t m, int64_t s, uint64_t seed, int kind, cudaStream_t st,
             const float** g32, const __nv_bfloat16** ghi) {
    GCache& g = h->g;
    const int64_t ld = kind == 0 ? s : (s + 63) / 64 * 64;
    const size_t elems = (size_t)m * (size_t)ld;
    const size_t bytes = kind == 2 ? 2 * elems * sizeof(__nv_bfloat16) : elems * sizeof(float);
    if (!(g.ptr && g.seed == seed && g.m == m && g.s == s && g.kind == kind)) {
        if (g.bytes < bytes) {
            if (g.ptr) cudaFree(g.ptr);
            g.ptr = nullptr;
            g.bytes = 0;
            cudaError_t e = cudaMalloc(&g.ptr, bytes);
            if (e != cudaSuccess) {
                g.ptr = nullptr;
                cudaGetLastError();
                return fail(LEV_ENOMEM, "cudaMalloc(G, %zu bytes) failed", bytes);
            }
            g.bytes = bytes;
        }
        cudaError_t e;
        if (kind == 2)
            e = lev::launch_gen_gaussian(m, s, ld, seed, nullptr, 2, (__nv_bfloat16*)g.ptr, st);
        else
            e = lev::launch_gen_gaussian(m, s, ld, seed, (float*)g.ptr, kind == 3 ? 1 : 0, nullptr, st);
        if (e != cudaSuccess) return fail(LEV_ECUDA, "G generation: %s", cudaGetErrorString(e));
        g.seed = seed;
        g.m = m;
        g.s = s;
        g.kind = kind;
    }
    if (g32) *g32 = kind != 2 ? (const float*)g.ptr : nullptr;
    if (ghi) *ghi = kind == 2 ? (const __nv_bfloat16*)g.ptr : nullptr;
    return LEV_OK;
}

// Gaussian stage A~ = G B for the selected precision.
int gaussian_stage(lev_handle* h, const float* B, int64_t m, int64_t s, int64_t d, uint64_t seed,
                   int32_t prec, float* Atilde, cudaStream_t st) {
    if (prec == LEV_FP32) {
        const float* g32 = nullptr;
        LEV_TRY(ensure_g(h, m, s, seed, 0, st, &g32, nullptr));
        const int splits = lev::gaussian_stage_splits(m, d, s);
        LEV_TRY(ensure(h->partial, sizeof(float) * (size_t)splits * m * d));
        LEV_CUDA(lev::launch_gaussian_stage_fp32(g32, B, m, s, d, (float*)h->partial.ptr, splits, Atilde, st));
        return LEV_OK;
    }
    return lev::tc_gaussian_stage(h, B, m, s, d, seed, prec, Atilde, st);
}

// The rows of each bucket in increasing order (off: s+1 bucket offsets, perm_rows: n local rows,
// hashed by their global index row0 + i). It depends on (seed, n, s, row0) only, so the handle
// keeps the last one and rebuilds it only when one of those (or the buffers) changes.
int bucket_perm(lev_handle* h, int64_t n, int64_t s, uint64_t seed, int64_t row0, cudaStream_t st) {
    const void* off0 = h->off.ptr;
    const void* perm0 = h->perm_rows.ptr;
    LEV_TRY(ensure(h->count, sizeof(int) * (size_t)(s + 1)));
    LEV_TRY(ensure(h->off, sizeof(int) * (size_t)(s + 1)));
    LEV_TRY(ensure(h->tmp, sizeof(uint32_t) * (size_t)n));
    LEV_TRY(ensure(h->perm_rows, sizeof(uint32_t) * (size_t)n));
    if (!h->ev_perm) LEV_CUDA(cudaEventCreateWithFlags(&h->ev_perm, cudaEventDisableTiming));
    if (h->perm_n == n && h->perm_s == s && h->perm_seed == seed && h->perm_row0 == row0 && h->off.ptr == off0 &&
        h->perm_rows.ptr == perm0) {
        LEV_CUDA(cudaStreamWaitEvent(st, h->ev_perm, 0));
        return LEV_OK;
    }
    h->perm_n = -1;
    LEV_CUDA(lev::launch_bucket_perm(n, s, seed, row0, (int*)h->count.ptr, (int*)h->off.ptr, (uint32_t*)h->tmp.ptr,
                                     (uint32_t*)h->perm_rows.ptr, st));
    LEV_CUDA(cudaEventRecord(h->ev_perm, st));
    h->perm_seed = seed;
    h->perm_row0 = row0;
    h->perm_n = n;
    h->perm_s = s;
    return LEV_OK;
}

// Omega (d x k FP64, d <= 1024) of (seed, d, k), drawn once and kept by the handle; with `chol`
// also the Cholesky factor of Omega_kc Omega_kc^T (kc = min(d, k)), kept with it. `st` waits for
// an Omega (and factor) that an earlier call made, possibly on another stream.
int ensure_omega(lev_handle* h, uint64_t seed, int64_t d, int64_t k, bool chol, cudaStream_t st,
                 const double** Om, lev::QrScratch* qc) {
    const int64_t kc = d < k ? d : k;
    const size_t qbytes = (lev::qr_scratch_bytes(k, kc) + 255) & ~size_t(255);
    const void* p0 = h->omega.ptr;
    const void* c0 = h->omega_chol.ptr;
    LEV_TRY(ensure(h->omega, sizeof(double) * (size_t)d * k));
    if (chol) LEV_TRY(ensure(h->omega_chol, qbytes + sizeof(int32_t) * (size_t)kc));
    if (!h->ev_omega) LEV_CUDA(cudaEventCreateWithFlags(&h->ev_omega, cudaEventDisableTiming));
    const bool have = h->omega_seed == seed && h->omega_d == d && h->omega_k == k && h->omega.ptr == p0;
    const bool have_chol = have && h->omega_chol_ok && h->omega_chol.ptr == c0;
    if (have && (!chol || have_chol)) {
        LEV_CUDA(cudaStreamWaitEvent(st, h->ev_omega, 0));
    } else {
        if (!have) {
            h->omega_d = -1;
            h->omega_chol_ok = false;
            LEV_CUDA(lev::launch_gen_omega(seed, d, k, (double*)h->omega.ptr, st));
        } else {
            LEV_CUDA(cudaStreamWaitEvent(st, h->ev_omega, 0));
        }
        if (chol) {
            lev::QrScratch q;
            lev::qr_scratch_carve(h->omega_chol.ptr, k, kc, &q);
            int32_t* iota = (int32_t*)((char*)h->omega_chol.ptr + qbytes);
            LEV_CUDA(lev::launch_omega_chol((const double*)h->omega.ptr, d, k, q, iota, h->status, st));
            h->omega_chol_ok = true;
        }
        LEV_CUDA(cudaEventRecord(h->ev_omega, st));
        h->omega_seed = seed;
        h->omega_d = d;
        h->omega_k = k;
    }
    if (Om) *Om = (const double*)h->omega.ptr;
    if (qc && chol) lev::qr_scratch_carve(h->omega_chol.ptr, k, kc, qc);
    return LEV_OK;
}

// M = R_11^{-1} Omega into Mfull through the handle's Omega cache (drawn once per (seed, d, k)).
// `reduced`: when r < k, R_11^{-1} L_r (r columns) instead, L_r L_r^T = Omega_r Omega_r^T.
int omega_factor(lev_handle* h, const double* R, const int32_t* perm, const int64_t* d_rank, int64_t d, int64_t k,
                 uint64_t seed, bool identity, bool reduced, float* Mfull, cudaStream_t st) {
    const double* Om = nullptr;
    const double* Lc = nullptr;
    const int64_t* d_kc = nullptr;
    const int64_t kc = d < k ? d : k;
    if (!identity && d <= 1024) {
        const bool chol = reduced;
        lev::QrScratch qc;
        LEV_TRY(ensure_omega(h, seed, d, k, chol, st, &Om, &qc));
        if (chol) {
            Lc = qc.Rorig;
            d_kc = qc.rank;
        }
    }
    double* Rs = nullptr;
    if (d <= 1024) {
        LEV_TRY(ensure(h->omega_rs, sizeof(double) * (size_t)d * d));
        Rs = (double*)h->omega_rs.ptr;
    }
    LEV_CUDA(lev::launch_omega_factor(R, perm, d_rank, d, k, seed, identity, Om, Lc, kc, d_kc, Rs, Mfull, st));
    return LEV_OK;
}

// The stages after B = S A (in h->B): A~ = G B, or with LEV_SKETCH_SRHT A~ = G (F B), F the
// SRHT to t = p->srht_t rows (B is transformed in place) and G m x t.
int gaussian_after_countsketch(lev_handle* h, const lev_params* p, const Sizes& z, int64_t d, float* Atilde,
                               cudaStream_t st) {
    if (!(p->flags & LEV_SKETCH_SRHT))
        return gaussian_stage(h, (const float*)h->B.ptr, z.m, z.s, d, p->seed, p->sketch_prec, Atilde, st);
    const int64_t t = p->srht_t;
    if ((z.s & (z.s - 1)) != 0 || z.s > (int64_t(1) << 24))
        return fail(LEV_EINVAL, "LEV_SKETCH_SRHT needs s a power of two <= 2^24 (s = %lld)", (long long)z.s);
    if (t < 1 || t > z.s) return fail(LEV_EINVAL, "LEV_SKETCH_SRHT needs 1 <= srht_t <= s");
    LEV_TRY(ensure(h->srht_c, sizeof(float) * (size_t)t * d));
    LEV_CUDA(lev::launch_srht((float*)h->B.ptr, z.s, d, t, p->seed, (float*)h->srht_c.ptr, st));
    return gaussian_stage(h, (const float*)h->srht_c.ptr, z.m, t, d, p->seed, p->sketch_prec, Atilde, st);
}

int sketch_common_dense(lev_handle* h, const float* A, int64_t n, int64_t d, int64_t lda,
                        const lev_params* p, const Sizes& z, float* Atilde, cudaStream_t st) {
    if (p->flags & LEV_SKETCH_IDENTITY) {
        LEV_CUDA(lev::launch_copy_dense(A, lda, n, d, Atilde, st));
        return LEV_OK;
    }
    LEV_TRY(bucket_perm(h, n, z.s, p->seed, z.row0, st));
    // BF16 forms without the SRHT: the CountSketch writes the Gaussian stage's BF16 operand itself
    // (no FP32 B, no transpose); the operand's values are those the transpose would produce
    if (!(p->flags & LEV_SKETCH_SRHT) && (p->sketch_prec == LEV_BF16 || p->sketch_prec == LEV_BF16X3)) {
        __nv_bfloat16 *hi = nullptr, *lo = nullptr;
        int64_t ld = 0;
        LEV_TRY(lev::tc_gaussian_operand(h, z.s, d, p->sketch_prec, &hi, &lo, &ld));
        const cudaError_t e = lev::launch_countsketch_dense_op(A, lda, d, z.s, ld, (const int*)h->off.ptr,
                                                               (const uint32_t*)h->perm_rows.ptr, hi, lo, st);
        if (e == cudaSuccess) return lev::tc_gaussian_stage_blocked(h, z.m, z.s, d, p->seed, p->sketch_prec, Atilde, st);
        if (e != cudaErrorNotSupported) return fail(LEV_ECUDA, "CountSketch: %s", cudaGetErrorString(e));
    }
    LEV_TRY(ensure(h->B, sizeof(float) * (size_t)z.s * d));
    LEV_CUDA(lev::launch_countsketch_dense(A, lda, d, z.s, (const int*)h->off.ptr,
                                           (const uint32_t*)h->perm_rows.ptr, (float*)h->B.ptr, st));
    return gaussian_after_countsketch(h, p, z, d, Atilde, st);
}

int sketch_common_csr(lev_handle* h, const int64_t* row_ptr, const int32_t* col, const float* val,
                      int64_t n, int64_t d, const lev_params* p, const Sizes& z, float* Atilde,
                      cudaStream_t st) {
    if (p->flags & LEV_SKETCH_IDENTITY) return fail(LEV_EINVAL, "LEV_SKETCH_IDENTITY is for dense A only");
    LEV_TRY(bucket_perm(h, n, z.s, p->seed, z.row0, st));
    LEV_TRY(ensure(h->B, sizeof(float) * (size_t)z.s * d));
    LEV_CUDA(lev::launch_countsketch_csr(row_ptr, col, val, d, z.s, (const int*)h->off.ptr,
                                         (const uint32_t*)h->perm_rows.ptr, (float*)h->B.ptr, st));
    return gaussian_after_countsketch(h, p, z, d, Atilde, st);
}

int rrqr_common(lev_handle* h, const float* Atilde, int64_t m, int64_t d, double tau,
                const int32_t* forced, int64_t forced_rank, int32_t* perm, double* R,
                lev::QrScratch* qs, cudaStream_t st) {
    LEV_TRY(ensure(h->qr, lev::qr_scratch_bytes(m, d)));
    lev::qr_scratch_carve(h->qr.ptr, m, d, qs);
    if (fault_is("launch")) return fail(LEV_ECUDA, "pivoted QR launch failed (injected by LEV_FAULT=launch)");
    LEV_CUDA(lev::launch_pivoted_qr(Atilde, m, d, tau, forced, forced_rank, *qs, perm, R, h->status,
                                    h->num_sms, st, h->timing ? h->tmark : nullptr));
    if (h->timing) h->timed_once = true;
    return LEV_OK;
}

// Synchronise, read the rank and the device status word.

int finish(lev_handle* h, const lev::QrScratch& qs, int64_t* rank, cudaStream_t st) {
    LEV_CUDA(cudaMemcpyAsync(h->host_rank, qs.rank, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    int32_t status = 0;
    LEV_CUDA(cudaMemcpyAsync(h->host_rank + 1, h->status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    LEV_CUDA(cudaStreamSynchronize(st));
    memcpy(&status, h->host_rank + 1, sizeof(int32_t));
    if (fault_is("timeout") && status == 0)
        return fail(LEV_ETIMEOUT, "a bounded device wait gave up (injected by LEV_FAULT=timeout)");
    if (status != 0) {
        cudaMemsetAsync(h->status, 0, sizeof(int32_t), st);
        return fail(LEV_ETIMEOUT, "a bounded device wait gave up (status %d)", status);
    }
    if (rank) *rank = h->host_rank[0];
    if (h->host_rank[0] == 0) return fail(LEV_ERANK0, "numerical rank is 0");
    return LEV_OK;
}

// Pieces of the handle's rank workspace: Y or Z (d x d), sigma, wn, g2 (d each), out (16),
// argmax partials (1024 values, 1024 indices), 64 uint32 of barrier and rotation counts, order (d
// int32), the sweep count.
struct RankWs {
    double *Y, *sig, *wn, *g2, *out, *part_v;
    long long* part_e;
    unsigned* work;
    int32_t *order, *sweeps;
    unsigned* version;
    float* Yhl;        // 2 d x d FP32: the double-float rows of the Jacobi
};
int rank_ws(lev_handle* h, int64_t d, RankWs* w) {
    LEV_TRY(ensure(h->rank_ws, sizeof(double) * lev::rank_scratch_doubles(d)));
    h->rank_ws_d = d;
    double* ws = (double*)h->rank_ws.ptr;
    w->Y = ws;
    w->sig = ws + d * d;
    w->wn = w->sig + d;
    w->g2 = w->wn + d;
    w->out = w->g2 + d;
    w->part_v = w->out + 16;
    w->part_e = reinterpret_cast<long long*>(w->part_v + 1024);
    w->work = reinterpret_cast<unsigned*>(w->part_e + 1024);
    w->order = reinterpret_cast<int32_t*>(w->work + 64);
    w->sweeps = w->order + d;
    w->version = reinterpret_cast<unsigned*>(w->sweeps + 2);
    w->Yhl = reinterpret_cast<float*>(ws + (((reinterpret_cast<char*>(w->version + d) - reinterpret_cast<char*>(ws)) + 63) / 64) * 8);
    return LEV_OK;
}

// The pivoted QR of A~ with the rank rule of p: the diagonal test of rrqr_common by default;
// with LEV_RANK_SVD the QR runs to the end and the rank is the count of singular values of A~
// above tau sigma_1 (sigma: optional device output, d doubles, descending); with LEV_SRRQR
// strong-RRQR swaps at that rank follow, each step a forced-pivot Cholesky of the Gram matrix of
// A~ for the current columns, then the largest rho, until rho <= phi. Leaves perm, R (rows < rank,
// pivot order) and qs->rank like rrqr_common; h->last_swaps counts the swaps. Synchronises `st`
// once per strong-RRQR step.
int select_common(lev_handle* h, const float* Atilde, int64_t m, int64_t d, const lev_params* p, int32_t* perm,
                  double* R, lev::QrScratch* qs, double* sigma_out, cudaStream_t st) {
    const bool svd = (p->flags & LEV_RANK_SVD) != 0, sr = (p->flags & LEV_SRRQR) != 0;
    h->last_swaps = 0;
    if (!svd && !sr) {
        if (sigma_out) return fail(LEV_EINVAL, "sigma is computed with LEV_RANK_SVD only");
        return rrqr_common(h, Atilde, m, d, tau_of(p), nullptr, 0, perm, R, qs, st);
    }
    if (d > 1024) return fail(LEV_EINVAL, "LEV_RANK_SVD and LEV_SRRQR need d <= 1024");
    if (p->flags & LEV_FORCE_PIVOTS) return fail(LEV_EINVAL, "forced pivots take no rank rule");
    const double phi = p->phi == 0 ? 2.0 : p->phi;
    if (sr && !(phi >= 1.0)) return fail(LEV_EINVAL, "phi must be >= 1 (got %g)", phi);
    RankWs rw;
    LEV_TRY(rank_ws(h, d, &rw));
    double *Y = rw.Y, *sig = rw.sig, *wn = rw.wn, *g2 = rw.g2, *out = rw.out, *part_v = rw.part_v;
    long long* part_e = rw.part_e;
    unsigned* work = rw.work;
    int32_t *order = rw.order, *sweeps = rw.sweeps;
    if (svd) {
        LEV_TRY(rrqr_common(h, Atilde, m, d, 0.0, nullptr, 0, perm, R, qs, st));      // every step
        LEV_CUDA(lev::launch_svd_rank(R, qs->rank, d, tau_of(p), Y, rw.Yhl, work, sigma_out ? sigma_out : sig, order,
                                      qs->rank, sweeps, rw.version, h->status, h->num_sms, st));
    } else {
        LEV_TRY(rrqr_common(h, Atilde, m, d, tau_of(p), nullptr, 0, perm, R, qs, st));
    }
    if (!sr) return LEV_OK;
    int64_t k = 0;
    LEV_TRY(finish(h, *qs, &k, st));
    if (k >= d) return LEV_OK;
    LEV_TRY(ensure(h->omega_rs, sizeof(double) * (size_t)d * d));
    double* Rs = (double*)h->omega_rs.ptr;
    LEV_CUDA(lev::launch_gram_fp64(Atilde, d, m, d, qs->Gp, qs->G, st));
    const int64_t max_swaps = 64 * d;
    double* host_out = reinterpret_cast<double*>(h->host_rank + 2);
    for (int64_t it = 0;; ++it) {
        LEV_CUDA(lev::launch_factor_gram(m, d, tau_of(p), perm, k, *qs, perm, R, h->status, st));
        LEV_CUDA(lev::launch_scaled_transpose(R, qs->rank, d, Rs, st));
        LEV_CUDA(lev::launch_srrqr_step(R, Rs, qs->G, perm, d, k, phi, Y, wn, g2, part_v, part_e, out, st));
        LEV_CUDA(cudaMemcpyAsync(host_out, out, sizeof(double), cudaMemcpyDeviceToHost, st));
        int64_t k2 = 0;
        LEV_TRY(finish(h, *qs, &k2, st));
        if (k2 != k) return fail(LEV_EINVAL, "strong RRQR: the forced factor stopped at %lld of %lld columns",
                                 (long long)k2, (long long)k);
        if (!(*host_out > phi * phi)) break;
        h->last_swaps = it + 1;
        if (it + 1 >= max_swaps) return fail(LEV_EINVAL, "strong RRQR did not settle in %lld swaps", (long long)max_swaps);
    }
    return LEV_OK;
}

// The CSR structure of the input contract (row_ptr[0] = 0, non-decreasing, row_ptr[n] = nnz), checked
// by one device pass over row_ptr whose verdict the host reads (one synchronisation) before any kernel
// reads col or val. Skipped with LEV_CSR_UNCHECKED.
int check_csr(lev_handle* h, const int64_t* row_ptr, int64_t n, int64_t nnz, uint32_t flags, cudaStream_t st) {
    if (flags & LEV_CSR_UNCHECKED) return LEV_OK;
    int32_t* bad = h->status + 1;
    LEV_CUDA(cudaMemsetAsync(bad, 0, sizeof(int32_t), st));
    LEV_CUDA(lev::launch_check_csr(row_ptr, n, nnz, bad, st));
    int32_t* hb = reinterpret_cast<int32_t*>(h->host_rank + 4);
    LEV_CUDA(cudaMemcpyAsync(hb, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    LEV_CUDA(cudaStreamSynchronize(st));
    const int32_t v = *hb;
    if (v == 0) return LEV_OK;
    return fail(LEV_EINVAL, "malformed CSR row_ptr:%s%s%s", (v & 1) ? " row_ptr[0] != 0;" : "",
                (v & 2) ? " row_ptr decreases;" : "", (v & 4) ? " row_ptr[n] != nnz;" : "");
}

// B = A^T A of CSR A (d x d FP64) as the sum of the rows' outer products (Lemma 8, Sec. 5.1): rows of
// more than max(32, d / 5) entries are densified and their Gram formed by the compensated dense
// kernel (about 30x the rate of the FP64 atomics per product, so it pays beyond about d / 5
// entries); the others add their pairs by FP64 atomics. Synchronises `st` once (the count of long
// rows sizes the dense part).
int csr_gram(lev_handle* h, const int64_t* row_ptr, const int32_t* col, const float* val, int64_t n, int64_t d,
             double* G, cudaStream_t st) {
    const int64_t max_len = std::max<int64_t>(32, d / 5);
    LEV_TRY(ensure(h->csr_heavy, sizeof(int32_t) * (size_t)n + 256));
    auto* hcount = reinterpret_cast<unsigned long long*>(h->csr_heavy.ptr);
    auto* hidx = reinterpret_cast<int32_t*>(static_cast<char*>(h->csr_heavy.ptr) + 256);
    LEV_CUDA(lev::launch_heavy_rows(row_ptr, n, max_len, hcount, hidx, st));
    LEV_CUDA(cudaMemcpyAsync(h->host_rank + 3, hcount, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    LEV_CUDA(cudaStreamSynchronize(st));
    const int64_t nh = h->host_rank[3];
    const double* Gheavy = nullptr;
    if (nh > 0) {
        const size_t gp = lev::gram_partial_doubles(nh, d);
        LEV_TRY(ensure(h->csr_dense, sizeof(double) * (gp + (size_t)d * d) + sizeof(float) * (size_t)nh * d));
        double* Gh = static_cast<double*>(h->csr_dense.ptr);
        double* Gp2 = Gh + (size_t)d * d;
        float* H = reinterpret_cast<float*>(Gp2 + gp);
        LEV_CUDA(lev::launch_densify_rows(row_ptr, col, val, hidx, hcount, nh, d, H, st));
        LEV_CUDA(lev::launch_gram_fp64(H, d, nh, d, Gp2, Gh, st));
        Gheavy = Gh;
    }
    LEV_CUDA(lev::launch_gram_csr_light(row_ptr, col, val, n, d, max_len, Gheavy, G, st));
    return LEV_OK;
}

// theta~ of CSR A: the second form of Lemma 1 (a P a^T with P = Mfull Mfull^T) when the rows are
// short against k, else the first (||a Mfull||^2).
int final_csr(lev_handle* h, const int64_t* rp, const int32_t* cl, const float* vl, int64_t n, int64_t d, int64_t nnz,
              const float* Mfull, int64_t k, float* theta, cudaStream_t st) {
    if (lev::csr_gram_pays(n, d, nnz, k)) {
        LEV_TRY(ensure(h->csr_p, lev::csr_gram_scratch_bytes(d, k)));
        LEV_CUDA(lev::launch_final_csr_gram(rp, cl, vl, n, d, Mfull, k, h->csr_p.ptr, theta, st));
        return LEV_OK;
    }
    LEV_CUDA(lev::launch_final_csr_fp32(rp, cl, vl, n, d, Mfull, k, theta, st));
    return LEV_OK;
}

int final_dense(lev_handle* h, const float* A, int64_t n, int64_t d, int64_t lda, const float* Mfull,
                int64_t k, int32_t prec, float* theta, cudaStream_t st) {
    if (prec == LEV_FP32) {
        LEV_CUDA(lev::launch_final_dense_fp32(A, lda, n, d, Mfull, k, theta, st));
        return LEV_OK;
    }
    return lev::tc_final_dense(h, A, n, d, lda, Mfull, k, prec, theta, st);
}

}  // namespace

// ---------------------------------------------------------------------------
// scratch access for the tensor-core module
// ---------------------------------------------------------------------------
namespace lev {
int handle_scratch(lev_handle* h, int which, size_t bytes, void** out) {
    Buf* b = which == 0 ? &h->tc_ws : (which == 1 ? &h->partial : (which == 2 ? &h->tc_ws2 : &h->tc_pad));
    LEV_TRY(ensure(*b, bytes));
    *out = b->ptr;
    return LEV_OK;
}
int handle_num_sms(lev_handle* h) { return h->num_sms; }
bool fault_pivot_wait() { return fault_is("pivwait"); }
const cudaEvent_t* handle_final_marks(lev_handle* h) {
    if (!h->timing) return nullptr;
    h->final_timed = true;
    return h->fmark;
}
int32_t* handle_status(lev_handle* h) { return h->status; }
int handle_gaussian(lev_handle* h, int64_t m, int64_t s, uint64_t seed, int kind, cudaStream_t st,
                    const float** g32, const __nv_bfloat16** ghi) {
    return ensure_g(h, m, s, seed, kind, st, g32, ghi);
}
int handle_fail(int code, const char* msg) { return fail(code, "%s", msg); }
}  // namespace lev

extern "C" {

const char* lev_last_error(void) { return g_last_error.c_str(); }

int lev_params_init(lev_params* p) {
    if (!p) return fail(LEV_EINVAL, "params is NULL");
    memset(p, 0, sizeof(*p));
    p->eps = 0.5;
    p->delta = 1.0 / 3.0;
    p->gamma = 2.0;
    p->tau = 1e-5;
    p->sketch_prec = LEV_FP32;
    p->final_prec = LEV_FP32;
    return LEV_OK;
}

int lev_resolve_sizes(const lev_params* p, int64_t n, int64_t d, int64_t* s, int64_t* m, int64_t* k) {
    Sizes z;
    LEV_TRY(resolve(p, n, d, &z, true));
    if (s) *s = z.s;
    if (m) *m = z.m;
    if (k) *k = z.k;
    return LEV_OK;
}

int lev_create(lev_handle** out, int device) {
    if (!out) return fail(LEV_EINVAL, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    LEV_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(LEV_EINVAL, "device %d out of range (%d devices)", device, ndev);
    LEV_CUDA(cudaSetDevice(device));
    int sms = 0;
    LEV_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    if (sms < 1) return fail(LEV_ECUDA, "device %d reports %d SMs", device, sms);
    lev_handle* h = new lev_handle();
    h->device = device;
    h->num_sms = sms;
    if (cudaMalloc(&h->status, 64) != cudaSuccess || cudaMemset(h->status, 0, 64) != cudaSuccess ||
        cudaMallocHost(&h->host_rank, 64) != cudaSuccess) {
        cudaGetLastError();
        lev_destroy(h);
        return fail(LEV_ENOMEM, "handle allocation failed");
    }
    *out = h;
    return LEV_OK;
}

int lev_destroy(lev_handle* h) {
    if (!h) return LEV_OK;
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    for_each_buf(h, [](Buf& b) { release(b); });
    for (int i = 0; i < 2; ++i) {
        if (h->ev_copied[i]) cudaEventDestroy(h->ev_copied[i]);
        if (h->ev_used[i]) cudaEventDestroy(h->ev_used[i]);
    }
    if (h->copy_st) cudaStreamDestroy(h->copy_st);
    if (h->ev_perm) cudaEventDestroy(h->ev_perm);
    for (int i = 0; i < 3; ++i)
        if (h->tmark[i]) cudaEventDestroy(h->tmark[i]);
    for (int i = 0; i < 2; ++i)
        if (h->fmark[i]) cudaEventDestroy(h->fmark[i]);
    if (h->ev_omega) cudaEventDestroy(h->ev_omega);
    if (h->g.ptr) cudaFree(h->g.ptr);
    if (h->status) cudaFree(h->status);
    if (h->host_rank) cudaFreeHost(h->host_rank);
    if (h->host_lsqr) cudaFreeHost(h->host_lsqr);
    delete h;
    return LEV_OK;
}

int lev_workspace_bytes(lev_handle* h, int64_t* bytes) {
    if (!h || !bytes) return fail(LEV_EINVAL, "handle or bytes is NULL");
    size_t total = h->g.bytes + (h->status ? 64 : 0);
    for_each_buf(h, [&total](Buf& b) { total += b.bytes; });
    *bytes = (int64_t)total;
    return LEV_OK;
}

int lev_set_timing(lev_handle* h, int enable) {
    LEV_TRY(set_device(h));
    if (enable && !h->tmark[0])
        for (int i = 0; i < 3; ++i) LEV_CUDA(cudaEventCreate(&h->tmark[i]));
    if (enable && !h->fmark[0])
        for (int i = 0; i < 2; ++i) LEV_CUDA(cudaEventCreate(&h->fmark[i]));
    h->timing = enable != 0;
    h->timed_once = false;
    h->final_timed = false;
    return LEV_OK;
}

int lev_final_timing(lev_handle* h, float* kernel_ms) {
    LEV_TRY(set_device(h));
    if (!h->timing || !h->final_timed)
        return fail(LEV_EINVAL, "timing is off or no tensor-core final pass ran since it was enabled");
    LEV_CUDA(cudaEventSynchronize(h->fmark[1]));
    float a = 0.f;
    LEV_CUDA(cudaEventElapsedTime(&a, h->fmark[0], h->fmark[1]));
    if (kernel_ms) *kernel_ms = a;
    return LEV_OK;
}

int lev_rrqr_timing(lev_handle* h, float* gram_ms, float* factor_ms) {
    LEV_TRY(set_device(h));
    if (!h->timing || !h->timed_once) return fail(LEV_EINVAL, "timing is off or no rrqr ran since it was enabled");
    LEV_CUDA(cudaEventSynchronize(h->tmark[2]));
    float a = 0.f, b = 0.f;
    LEV_CUDA(cudaEventElapsedTime(&a, h->tmark[0], h->tmark[1]));
    LEV_CUDA(cudaEventElapsedTime(&b, h->tmark[1], h->tmark[2]));
    if (gram_ms) *gram_ms = a;
    if (factor_ms) *factor_ms = b;
    return LEV_OK;
}

int lev_device_status(lev_handle* h, int32_t* status) {
    LEV_TRY(set_device(h));
    if (!status) return fail(LEV_EINVAL, "status is NULL");
    LEV_CUDA(cudaMemcpy(status, h->status, sizeof(int32_t), cudaMemcpyDeviceToHost));
    return LEV_OK;
}

int lev_prepare(lev_handle* h, int64_t n, int64_t d, const lev_params* p, void* stream) {
    LEV_TRY(set_device(h));
    Sizes z;
    LEV_TRY(resolve(p, n, d, &z, true));
    LEV_TRY(check_prec(p->sketch_prec, "sketch"));
    cudaStream_t st = (cudaStream_t)stream;
    if (p->flags & LEV_SKETCH_IDENTITY) return LEV_OK;
    LEV_TRY(bucket_perm(h, n, z.s, p->seed, z.row0, st));
    // G in the image the Gaussian stage of sketch_prec reads (m x t after an SRHT)
    const int64_t cols = (p->flags & LEV_SKETCH_SRHT) ? (int64_t)p->srht_t : z.s;
    if (cols < 1 || cols > z.s) return fail(LEV_EINVAL, "LEV_SKETCH_SRHT needs 1 <= srht_t <= s");
    const int kind = p->sketch_prec == LEV_FP32 ? 0 : (p->sketch_prec == LEV_TF32 ? 3 : 2);
    LEV_TRY(ensure_g(h, z.m, cols, p->seed, kind, st, nullptr, nullptr));
    if (!(p->flags & LEV_OMEGA_IDENTITY) && d <= 1024)
        LEV_TRY(ensure_omega(h, p->seed, d, z.k, true, st, nullptr, nullptr));
    return LEV_OK;
}

int lev_sketch_dense(lev_handle* h, const float* A, int64_t n, int64_t d, int64_t lda,
                     const lev_params* p, float* Atilde, void* stream) {
    LEV_TRY(set_device(h));
    Sizes z;
    LEV_TRY(resolve(p, n, d, &z, true));
    if (!A || !Atilde) return fail(LEV_EINVAL, "NULL array");
    if (lda < d) return fail(LEV_EINVAL, "lda < d");
    LEV_TRY(check_prec(p->sketch_prec, "sketch"));
    return sketch_common_dense(h, A, n, d, lda, p, z, Atilde, (cudaStream_t)stream);
}

int lev_sketch_csr(lev_handle* h, const int64_t* row_ptr, const int32_t* col, const float* val,
                   int64_t n, int64_t d, int64_t nnz, const lev_params* p, float* Atilde, void* stream) {
    LEV_TRY(set_device(h));
    Sizes z;
    LEV_TRY(resolve(p, n, d, &z, true));
    if (!row_ptr || (nnz > 0 && (!col || !val)) || !Atilde) return fail(LEV_EINVAL, "NULL array");
    if (nnz < 0) return fail(LEV_EINVAL, "nnz < 0");
    LEV_TRY(check_prec(p->sketch_prec, "sketch"));
    LEV_TRY(check_csr(h, row_ptr, n, nnz, p->flags, (cudaStream_t)stream));
    return sketch_common_csr(h, row_ptr, col, val, n, d, p, z, Atilde, (cudaStream_t)stream);
}

int lev_rrqr(lev_handle* h, const float* Atilde, int64_t m, int64_t d, double tau, int32_t* perm,
             double* R, int64_t* rank, void* stream) {
    LEV_TRY(set_device(h));
    if (!Atilde || !perm || !R) return fail(LEV_EINVAL, "NULL array");
    if (m < 1 || d < 1 || d > 4096 || m > (1 << 20)) return fail(LEV_EINVAL, "bad shape m=%lld d=%lld", (long long)m, (long long)d);
    if (tau <= 0) tau = 1e-5;
    cudaStream_t st = (cudaStream_t)stream;
    lev::QrScratch qs;
    LEV_TRY(rrqr_common(h, Atilde, m, d, tau, nullptr, 0, perm, R, &qs, st));
    if (!rank) return LEV_OK;
    return finish(h, qs, rank, st);
}

int lev_rrqr_select(lev_handle* h, const float* Atilde, int64_t m, int64_t d, const lev_params* p, int32_t* perm,
                    double* R, int64_t* rank, double* sigma, int64_t* swaps, void* stream) {
    LEV_TRY(set_device(h));
    if (!Atilde || !perm || !R || !p) return fail(LEV_EINVAL, "NULL array");
    if (m < 1 || d < 1 || d > 4096 || m > (1 << 20)) return fail(LEV_EINVAL, "bad shape m=%lld d=%lld", (long long)m, (long long)d);
    if (p->flags & LEV_FORCE_PIVOTS) return fail(LEV_EINVAL, "lev_rrqr_select takes no forced pivots");
    cudaStream_t st = (cudaStream_t)stream;
    lev::QrScratch qs;
    LEV_TRY(select_common(h, Atilde, m, d, p, perm, R, &qs, sigma, st));
    if (swaps) *swaps = h->last_swaps;
    if (!rank) return LEV_OK;
    return finish(h, qs, rank, st);
}

// Alg. 11 after the sketch in h->Atilde: the SVD rank rule, then N = V_k Sigma_k^{-1}.
static int precondition_tail(lev_handle* h, const Sizes& z, int64_t d, const lev_params* p, double* N,
                             int64_t* rank, double* sigma, cudaStream_t st) {
    if (d > 1024) return fail(LEV_EINVAL, "lev_precondition_* needs d <= 1024");
    lev_params q = *p;
    q.flags = (p->flags & ~(uint32_t)(LEV_SRRQR | LEV_FORCE_PIVOTS)) | LEV_RANK_SVD;
    LEV_TRY(ensure(h->R, sizeof(double) * (size_t)d * d));
    LEV_TRY(ensure(h->perm_d, sizeof(int32_t) * (size_t)d));
    lev::QrScratch qs;
    LEV_TRY(select_common(h, (const float*)h->Atilde.ptr, z.m, d, &q, (int32_t*)h->perm_d.ptr, (double*)h->R.ptr,
                          &qs, sigma, st));
    RankWs rw;
    LEV_TRY(rank_ws(h, d, &rw));
    LEV_CUDA(lev::launch_precond_n(rw.Y, rw.order, sigma ? sigma : rw.sig, (const int32_t*)h->perm_d.ptr, qs.rank, d,
                                   N, st));
    return finish(h, qs, rank, st);
}

int lev_precondition_dense(lev_handle* h, const float* A, int64_t n, int64_t d, int64_t lda, const lev_params* p,
                           double* N, int64_t* rank, double* sigma, void* stream) {
    LEV_TRY(set_device(h));
    Sizes z;
    LEV_TRY(resolve(p, n, d, &z));
    if (!A || !N) return fail(LEV_EINVAL, "NULL array");
    if (lda < d) return fail(LEV_EINVAL, "lda < d");
    if (is_host_pointer(A) || is_host_pointer(N)) return fail(LEV_EINVAL, "lev_precondition_dense takes device arrays");
    LEV_TRY(check_prec(p->sketch_prec, "sketch"));
    cudaStream_t st = (cudaStream_t)stream;
    LEV_TRY(ensure(h->Atilde, sizeof(float) * (size_t)z.m * d));
    LEV_TRY(sketch_common_dense(h, A, n, d, lda, p, z, (float*)h->Atilde.ptr, st));
    return precondition_tail(h, z, d, p, N, rank, sigma, st);
}

int lev_precondition_csr(lev_handle* h, const int64_t* row_ptr, const int32_t* col, const float* val, int64_t n,
                         int64_t d, int64_t nnz, const lev_params* p, double* N, int64_t* rank, double* sigma,
                         void* stream) {
    LEV_TRY(set_device(h));
    Sizes z;
    LEV_TRY(resolve(p, n, d, &z));
    if (!row_ptr || (nnz > 0 && (!col || !val)) || !N) return fail(LEV_EINVAL, "NULL array");
    if (nnz < 0) return fail(LEV_EINVAL, "nnz < 0");
    if (is_host_pointer(row_ptr) || is_host_pointer(N)) return fail(LEV_EINVAL, "lev_precondition_csr takes device arrays");
    LEV_TRY(check_prec(p->sketch_prec, "sketch"));
    cudaStream_t st = (cudaStream_t)stream;
    LEV_TRY(check_csr(h, row_ptr, n, nnz, p->flags, st));
    LEV_TRY(ensure(h->Atilde, sizeof(float) * (size_t)z.m * d));
    LEV_TRY(sketch_common_csr(h, row_ptr, col, val, n, d, p, z, (float*)h->Atilde.ptr, st));
    return precondition_tail(h, z, d, p, N, rank, sigma, st);
}

int lev_lsqr_dense(lev_handle* h, const float* A, int64_t n, int64_t d, int64_t lda, const double* N, int64_t k,
                   const float* b, double* x, int32_t max_iter, double atol, double btol, int32_t* iters,
                   double* rnorm, void* stream) {
    LEV_TRY(set_device(h));
    if (!A || !N || !b || !x) return fail(LEV_EINVAL, "NULL array");
    if (n < 1 || n >= (int64_t)1 << 31 || d < 1 || d > 1024 || lda < d)
        return fail(LEV_EINVAL, "bad shape n=%lld d=%lld lda=%lld", (long long)n, (long long)d, (long long)lda);
    if (k < 1 || k > d) return fail(LEV_EINVAL, "k = %lld outside [1, d]", (long long)k);
    if (max_iter < 0) return fail(LEV_EINVAL, "max_iter < 0");
    if (is_host_pointer(A) || is_host_pointer(N) || is_host_pointer(b) || is_host_pointer(x))
        return fail(LEV_EINVAL, "lev_lsqr_dense takes device arrays");
    cudaStream_t st = (cudaStream_t)stream;
    const int parts = lev::lsqr_parts(h->num_sms);
    LEV_TRY(ensure(h->lsqr_u, sizeof(float) * (size_t)n));
    LEV_TRY(ensure(h->lsqr_ws, sizeof(double) * lev::lsqr_scratch_doubles(d, parts)));
    if (!h->host_lsqr && cudaMallocHost(&h->host_lsqr, 256) != cudaSuccess)
        return fail(LEV_ENOMEM, "pinned host buffer");
    LEV_CUDA(cudaMemcpyAsync(h->lsqr_u.ptr, b, sizeof(float) * (size_t)n, cudaMemcpyDeviceToDevice, st));
    int it = 0;
    double rn = 0.0;
    LEV_CUDA(lev::launch_lsqr(A, lda, nullptr, nullptr, nullptr, n, d, N, k, (float*)h->lsqr_u.ptr, x, max_iter,
                              atol > 0 ? atol : 1e-6,
                              btol > 0 ? btol : 1e-6, (double*)h->lsqr_ws.ptr, parts, h->host_lsqr, &it, &rn, st));
    if (iters) *iters = it;
    if (rnorm) *rnorm = rn;
    return LEV_OK;
}

int lev_rank_stats(lev_handle* h, int64_t* swaps, int32_t* jacobi_sweeps) {
    LEV_TRY(set_device(h));
    if (swaps) *swaps = h->last_swaps;
    if (jacobi_sweeps) {
        *jacobi_sweeps = 0;
        if (h->rank_ws.ptr) {
            RankWs rw;
            LEV_TRY(rank_ws(h, h->rank_ws_d, &rw));
            LEV_CUDA(cudaDeviceSynchronize());
            LEV_CUDA(cudaMemcpy(jacobi_sweeps, rw.sweeps, sizeof(int32_t), cudaMemcpyDeviceToHost));
        }
    }
    return LEV_OK;
}

int lev_lsqr_csr(lev_handle* h, const int64_t* row_ptr, const int32_t* col, const float* val, int64_t n, int64_t d,
                 int64_t nnz, const double* N, int64_t k, const float* b, double* x, int32_t max_iter, double atol,
                 double btol, int32_t* iters, double* rnorm, void* stream) {
    LEV_TRY(set_device(h));
    if (!row_ptr || (nnz > 0 && (!col || !val)) || !N || !b || !x) return fail(LEV_EINVAL, "NULL array");
    if (n < 1 || n >= (int64_t)1 << 31 || d < 1 || d > 1024 || nnz < 0)
        return fail(LEV_EINVAL, "bad shape n=%lld d=%lld", (long long)n, (long long)d);
    if (k < 1 || k > d) return fail(LEV_EINVAL, "k = %lld outside [1, d]", (long long)k);
    if (max_iter < 0) return fail(LEV_EINVAL, "max_iter < 0");
    if (is_host_pointer(row_ptr) || is_host_pointer(N) || is_host_pointer(b) || is_host_pointer(x))
        return fail(LEV_EINVAL, "lev_lsqr_csr takes device arrays");
    cudaStream_t st = (cudaStream_t)stream;
    LEV_TRY(check_csr(h, row_ptr, n, nnz, 0u, st));
    const int parts = lev::lsqr_parts(h->num_sms);
    LEV_TRY(ensure(h->lsqr_u, sizeof(float) * (size_t)n));
    LEV_TRY(ensure(h->lsqr_ws, sizeof(double) * lev::lsqr_scratch_doubles(d, parts)));
    if (!h->host_lsqr && cudaMallocHost(&h->host_lsqr, 256) != cudaSuccess)
        return fail(LEV_ENOMEM, "pinned host buffer");
    LEV_CUDA(cudaMemcpyAsync(h->lsqr_u.ptr, b, sizeof(float) * (size_t)n, cudaMemcpyDeviceToDevice, st));
    int it = 0;
    double rn = 0.0;
    LEV_CUDA(lev::launch_lsqr(nullptr, 0, row_ptr, col, val, n, d, N, k, (float*)h->lsqr_u.ptr, x, max_iter,
                              atol > 0 ? atol : 1e-6, btol > 0 ? btol : 1e-6, (double*)h->lsqr_ws.ptr, parts,
                              h->host_lsqr, &it, &rn, st));
    if (iters) *iters = it;
    if (rnorm) *rnorm = rn;
    return LEV_OK;
}

int lev_omega_factor(lev_handle* h, const double* R, const int32_t* perm, const int64_t* d_rank,
                     int64_t d, int64_t k, uint64_t seed, uint32_t flags, float* Mfull, void* stream) {
    LEV_TRY(set_device(h));
    if (!R || !perm || !d_rank || !Mfull) return fail(LEV_EINVAL, "NULL array");
    if (d < 1 || d > 4096 || k < 1 || k > 4096) return fail(LEV_EINVAL, "bad shape d=%lld k=%lld", (long long)d, (long long)k);
    return omega_factor(h, R, perm, d_rank, d, k, seed, (flags & LEV_OMEGA_IDENTITY) != 0,
                        (flags & LEV_OMEGA_REDUCED) != 0, Mfull, (cudaStream_t)stream);
}

int lev_final_dense(lev_handle* h, const float* A, int64_t n, int64_t d, int64_t lda, const float* Mfull,
                    int64_t k, int32_t prec, float* theta, void* stream) {
    LEV_TRY(set_device(h));
    if (!A || !Mfull || !theta) return fail(LEV_EINVAL, "NULL array");
    if (n < 1 || n >= (int64_t)1 << 31 || d < 1 || d > 4096 || k < 1 || k > 4096 || lda < d)
        return fail(LEV_EINVAL, "bad shape");
    LEV_TRY(check_prec(prec, "final"));
    return final_dense(h, A, n, d, lda, Mfull, k, prec, theta, (cudaStream_t)stream);
}

int lev_final_csr(lev_handle* h, const int64_t* row_ptr, const int32_t* col, const float* val, int64_t n,
                  int64_t d, int64_t nnz, const float* Mfull, int64_t k, int32_t prec, float* theta,
                  void* stream) {
    LEV_TRY(set_device(h));
    if (!row_ptr || (nnz > 0 && (!col || !val)) || !Mfull || !theta) return fail(LEV_EINVAL, "NULL array");
    if (n < 1 || n >= (int64_t)1 << 31 || d < 1 || d > 4096 || k < 1 || k > 4096 || nnz < 0)
        return fail(LEV_EINVAL, "bad shape");
    if (prec != LEV_FP32) return fail(LEV_EINVAL, "the CSR final pass supports LEV_FP32 only");
    LEV_TRY(check_csr(h, row_ptr, n, nnz, 0u, (cudaStream_t)stream));
    LEV_TRY(final_csr(h, row_ptr, col, val, n, d, nnz, Mfull, k, theta, (cudaStream_t)stream));
    return LEV_OK;
}

static int estimate_tail(lev_handle* h, const Sizes& z, int64_t d, const lev_params* p, int32_t* perm_out,
                         lev::QrScratch* qs, cudaStream_t st) {
    LEV_TRY(ensure(h->R, sizeof(double) * (size_t)d * d));
    LEV_TRY(ensure(h->perm_d, sizeof(int32_t) * (size_t)d));
    int32_t* perm = perm_out ? perm_out : (int32_t*)h->perm_d.ptr;
    const bool forced = (p->flags & LEV_FORCE_PIVOTS) != 0;
    if (forced && (!p->perm_in || p->rank_in < 0 || p->rank_in > d))
        return fail(LEV_EINVAL, "LEV_FORCE_PIVOTS needs perm_in and 0 <= rank_in <= d");
    if (forced)
        LEV_TRY(rrqr_common(h, (const float*)h->Atilde.ptr, z.m, d, tau_of(p), p->perm_in, p->rank_in, perm,
                            (double*)h->R.ptr, qs, st));
    else
        LEV_TRY(select_common(h, (const float*)h->Atilde.ptr, z.m, d, p, perm, (double*)h->R.ptr, qs, nullptr, st));
    if (perm != (int32_t*)h->perm_d.ptr)
        LEV_CUDA(cudaMemcpyAsync(h->perm_d.ptr, perm, sizeof(int32_t) * (size_t)d, cudaMemcpyDeviceToDevice, st));
    LEV_TRY(ensure(h->Mfull, sizeof(float) * (size_t)d * z.k));
    LEV_TRY(omega_factor(h, (const double*)h->R.ptr, perm, qs->rank, d, z.k, p->seed,
                         (p->flags & LEV_OMEGA_IDENTITY) != 0, true, (float*)h->Mfull.ptr, st));
    return LEV_OK;
}

// Copy host A (n x d, lda) into the next of the handle's two stage buffers on the handle's copy
// stream. The copy waits for the kernels of the call that last read that buffer (event ev_used),
// and `st` waits for the copy; the caller records ev_used[*slot] on `st` after its last read.
int stage_host_dense(lev_handle* h, const float* A, int64_t n, int64_t d, int64_t lda, cudaStream_t st, int* slot,
                     const float** dA) {
    if (!h->copy_st) {
        LEV_CUDA(cudaStreamCreateWithFlags(&h->copy_st, cudaStreamNonBlocking));
        for (int i = 0; i < 2; ++i) {
            LEV_CUDA(cudaEventCreateWithFlags(&h->ev_copied[i], cudaEventDisableTiming));
            LEV_CUDA(cudaEventCreateWithFlags(&h->ev_used[i], cudaEventDisableTiming));
        }
    }
    const int k = h->stage_next;
    LEV_TRY(ensure(h->stageA[k], sizeof(float) * (size_t)n * d));
    if (h->used_once[k]) LEV_CUDA(cudaStreamWaitEvent(h->copy_st, h->ev_used[k], 0));
    if (lda == d)
        LEV_CUDA(cudaMemcpyAsync(h->stageA[k].ptr, A, sizeof(float) * (size_t)n * d, cudaMemcpyHostToDevice,
                                 h->copy_st));
    else
        LEV_CUDA(cudaMemcpy2DAsync(h->stageA[k].ptr, sizeof(float) * d, A, sizeof(float) * lda, sizeof(float) * d, n,
                                   cudaMemcpyHostToDevice, h->copy_st));
    LEV_CUDA(cudaEventRecord(h->ev_copied[k], h->copy_st));
    LEV_CUDA(cudaStreamWaitEvent(st, h->ev_copied[k], 0));
    h->stage_next ^= 1;
    *slot = k;
    *dA = (const float*)h->stageA[k].ptr;
    return LEV_OK;
}

int lev_exact_dense(lev_handle* h, const float* A, int64_t n, int64_t d, int64_t lda, const lev_params* p,
                    float* theta, int64_t* rank, int32_t* perm_out, void* stream) {
    LEV_TRY(set_device(h));
    Sizes z;
    LEV_TRY(resolve(p, n, d, &z));
    if (!A || !theta) return fail(LEV_EINVAL, "NULL array");
    if (lda < d) return fail(LEV_EINVAL, "lda < d");
    if (is_host_pointer(A) || is_host_pointer(theta)) return fail(LEV_EINVAL, "lev_exact_dense takes device arrays");
    if (p->flags & (LEV_FORCE_PIVOTS | LEV_OMEGA_IDENTITY))
        return fail(LEV_EINVAL, "lev_exact_dense takes neither forced pivots nor LEV_OMEGA_IDENTITY");
    if (d > 1024) return fail(LEV_EINVAL, "lev_exact_dense needs d <= 1024 (the Gram route of the QR)");
    if (p->final_prec != LEV_FP32 && d > 256)
        return fail(LEV_EINVAL, "tensor-core final pass of lev_exact_dense needs d <= 256");
    LEV_TRY(check_prec(p->sketch_prec, "sketch"));
    LEV_TRY(check_prec(p->final_prec, "final"));
    cudaStream_t st = (cudaStream_t)stream;
    // steps 1-3 (Alg. 7): the columns K and the rank k from the pivoted QR of the CountGauss sketch
    LEV_TRY(ensure(h->Atilde, sizeof(float) * (size_t)z.m * d));
    LEV_TRY(sketch_common_dense(h, A, n, d, lda, p, z, (float*)h->Atilde.ptr, st));
    LEV_TRY(ensure(h->R, sizeof(double) * (size_t)d * d));
    LEV_TRY(ensure(h->perm_d, sizeof(int32_t) * (size_t)d));
    int32_t* perm = perm_out ? perm_out : (int32_t*)h->perm_d.ptr;
    lev::QrScratch qs;
    LEV_TRY(select_common(h, (const float*)h->Atilde.ptr, z.m, d, p, perm, (double*)h->R.ptr, &qs, nullptr, st));
    int64_t k = 0;
    int rc = finish(h, qs, &k, st);
    if (rc == LEV_ERANK0) {
        LEV_CUDA(cudaMemsetAsync(theta, 0, sizeof(float) * (size_t)n, st));
        if (rank) *rank = 0;
        return rc;
    }
    LEV_TRY(rc);
    // step 4: B = A_K^T A_K, the Gram matrix of A in FP64 restricted to K in pivot order; step 5
    // by its Cholesky factor B = R^T R (the pivoted Cholesky with the pivots of step 2 forced)
    LEV_TRY(ensure(h->exact_gp, sizeof(double) * lev::gram_partial_doubles(n, d)));
    lev::QrScratch q2 = qs;
    q2.Gp = (double*)h->exact_gp.ptr;
    LEV_CUDA(lev::launch_gram_fp64(A, lda, n, d, q2.Gp, q2.G, st));
    LEV_CUDA(lev::launch_factor_gram(n, d, tau_of(p), perm, k, q2, perm, (double*)h->R.ptr, h->status, st));
    int64_t k2 = 0;
    rc = finish(h, q2, &k2, st);
    if (rc == LEV_ERANK0) {
        LEV_CUDA(cudaMemsetAsync(theta, 0, sizeof(float) * (size_t)n, st));
        if (rank) *rank = 0;
        return rc;
    }
    LEV_TRY(rc);
    // step 6: theta_i = ||A_{i,K} R^{-1}||^2: M = R^{-1} (Omega = I) scattered into Mfull (d x d)
    LEV_TRY(ensure(h->Mfull, sizeof(float) * (size_t)d * d));
    LEV_TRY(omega_factor(h, (const double*)h->R.ptr, perm, q2.rank, d, d, p->seed, true, false, (float*)h->Mfull.ptr,
                         st));
    if (perm != (int32_t*)h->perm_d.ptr)
        LEV_CUDA(cudaMemcpyAsync(h->perm_d.ptr, perm, sizeof(int32_t) * (size_t)d, cudaMemcpyDeviceToDevice, st));
    LEV_TRY(final_dense(h, A, n, d, lda, (const float*)h->Mfull.ptr, d, p->final_prec, theta, st));
    if (rank) *rank = k2;
    return LEV_OK;
}

int lev_exact_csr(lev_handle* h, const int64_t* row_ptr, const int32_t* col, const float* val, int64_t n, int64_t d,
                  int64_t nnz, const lev_params* p, float* theta, int64_t* rank, int32_t* perm_out, void* stream) {
    LEV_TRY(set_device(h));
    Sizes z;
    LEV_TRY(resolve(p, n, d, &z));
    if (!row_ptr || (nnz > 0 && (!col || !val)) || !theta) return fail(LEV_EINVAL, "NULL array");
    if (nnz < 0) return fail(LEV_EINVAL, "nnz < 0");
    if (is_host_pointer(row_ptr) || (nnz > 0 && (is_host_pointer(col) || is_host_pointer(val))) ||
        is_host_pointer(theta))
        return fail(LEV_EINVAL, "lev_exact_csr takes device arrays");
    if (p->flags & (LEV_FORCE_PIVOTS | LEV_OMEGA_IDENTITY))
        return fail(LEV_EINVAL, "lev_exact_csr takes neither forced pivots nor LEV_OMEGA_IDENTITY");
    if (d > 1024) return fail(LEV_EINVAL, "lev_exact_csr needs d <= 1024 (the Gram route of the QR)");
    if (p->final_prec != LEV_FP32) return fail(LEV_EINVAL, "the CSR final pass supports LEV_FP32 only");
    LEV_TRY(check_prec(p->sketch_prec, "sketch"));
    cudaStream_t st = (cudaStream_t)stream;
    LEV_TRY(check_csr(h, row_ptr, n, nnz, p->flags, st));
    // steps 1-3 (Alg. 7): K and the rank k from the pivoted QR of the CountGauss sketch
    LEV_TRY(ensure(h->Atilde, sizeof(float) * (size_t)z.m * d));
    LEV_TRY(sketch_common_csr(h, row_ptr, col, val, n, d, p, z, (float*)h->Atilde.ptr, st));
    LEV_TRY(ensure(h->R, sizeof(double) * (size_t)d * d));
    LEV_TRY(ensure(h->perm_d, sizeof(int32_t) * (size_t)d));
    int32_t* perm = perm_out ? perm_out : (int32_t*)h->perm_d.ptr;
    lev::QrScratch qs;
    LEV_TRY(select_common(h, (const float*)h->Atilde.ptr, z.m, d, p, perm, (double*)h->R.ptr, &qs, nullptr, st));
    int64_t k = 0;
    int rc = finish(h, qs, &k, st);
    if (rc == LEV_ERANK0) {
        LEV_CUDA(cudaMemsetAsync(theta, 0, sizeof(float) * (size_t)n, st));
        if (rank) *rank = 0;
        return rc;
    }
    LEV_TRY(rc);
    // step 4: B = A_K^T A_K (all of A^T A, read at K in pivot order), the sum of the rows' outer
    // products (csr_gram); step 5 by the Cholesky factor B = R^T R with the pivots of step 2 forced
    LEV_TRY(csr_gram(h, row_ptr, col, val, n, d, qs.G, st));
    LEV_CUDA(lev::launch_factor_gram(n, d, tau_of(p), perm, k, qs, perm, (double*)h->R.ptr, h->status, st));
    int64_t k2 = 0;
    rc = finish(h, qs, &k2, st);
    if (rc == LEV_ERANK0) {
        LEV_CUDA(cudaMemsetAsync(theta, 0, sizeof(float) * (size_t)n, st));
        if (rank) *rank = 0;
        return rc;
    }
    LEV_TRY(rc);
    // step 6: theta_i = ||A_{i,K} R^{-1}||^2 with M = R^{-1} (Omega = I) scattered into Mfull
    LEV_TRY(ensure(h->Mfull, sizeof(float) * (size_t)d * d));
    LEV_TRY(omega_factor(h, (const double*)h->R.ptr, perm, qs.rank, d, d, p->seed, true, false, (float*)h->Mfull.ptr,
                         st));
    if (perm != (int32_t*)h->perm_d.ptr)
        LEV_CUDA(cudaMemcpyAsync(h->perm_d.ptr, perm, sizeof(int32_t) * (size_t)d, cudaMemcpyDeviceToDevice, st));
    LEV_TRY(final_csr(h, row_ptr, col, val, n, d, nnz, (const float*)h->Mfull.ptr, d, theta, st));
    if (rank) *rank = k2;
    return LEV_OK;
}

// Exact leverage of A itself by the Gram route (Alg. 5 with the QR orthogonaliser): the Gram matrix
// already in q->G, its pivoted Cholesky with the rank rule |R_jj| > tau |R_00| (the same pivots and
// R as a column-pivoted QR of A in exact arithmetic), M = R_11^{-1} (Omega = I) scattered into Mfull,
// then theta_i = ||A_{i,K} R_11^{-1}||^2 by the FP32 final pass (dense or CSR).
static int exact_reference_tail(lev_handle* h, lev::QrScratch& q, int64_t n, int64_t d, double tau, const float* A,
                                int64_t lda, const int64_t* rp, const int32_t* cl, const float* vl, int64_t nnz,
                                float* theta, int64_t* rank, int32_t* perm_out, cudaStream_t st) {
    LEV_TRY(ensure(h->R, sizeof(double) * (size_t)d * d));
    LEV_TRY(ensure(h->perm_d, sizeof(int32_t) * (size_t)d));
    int32_t* perm = perm_out ? perm_out : (int32_t*)h->perm_d.ptr;
    LEV_CUDA(lev::launch_factor_gram(n, d, tau, nullptr, 0, q, perm, (double*)h->R.ptr, h->status, st));
    int64_t k = 0;
    int rc = finish(h, q, &k, st);
    if (rc == LEV_ERANK0) {
        LEV_CUDA(cudaMemsetAsync(theta, 0, sizeof(float) * (size_t)n, st));
        if (rank) *rank = 0;
        return rc;
    }
    LEV_TRY(rc);
    LEV_TRY(ensure(h->Mfull, sizeof(float) * (size_t)d * d));
    LEV_TRY(omega_factor(h, (const double*)h->R.ptr, perm, q.rank, d, d, 0, true, false, (float*)h->Mfull.ptr, st));
    if (A)
        LEV_CUDA(lev::launch_final_dense_fp32(A, lda, n, d, (const float*)h->Mfull.ptr, d, theta, st));
    else
        LEV_TRY(final_csr(h, rp, cl, vl, n, d, nnz, (const float*)h->Mfull.ptr, d, theta, st));
    if (rank) *rank = k;
    return LEV_OK;
}

int lev_exact_reference_dense(lev_handle* h, const float* A, int64_t n, int64_t d, int64_t lda, double tau,
                              float* theta, int64_t* rank, int32_t* perm, void* stream) {
    LEV_TRY(set_device(h));
    if (!A || !theta) return fail(LEV_EINVAL, "NULL array");
    if (n < 1 || n >= (int64_t)1 << 31 || d < 1 || d > 1024 || lda < d)
        return fail(LEV_EINVAL, "bad shape n=%lld d=%lld lda=%lld (d <= 1024)", (long long)n, (long long)d,
                    (long long)lda);
    if (tau <= 0) tau = 1e-5;
    if (tau < 1e-6) return fail(LEV_EINVAL, "tau = %g below the Gram route's resolution (1e-6)", tau);
    if (is_host_pointer(A) || is_host_pointer(theta))
        return fail(LEV_EINVAL, "lev_exact_reference_dense takes device arrays");
    cudaStream_t st = (cudaStream_t)stream;
    LEV_TRY(ensure(h->qr, lev::qr_scratch_bytes(1, d)));
    lev::QrScratch q;
    lev::qr_scratch_carve(h->qr.ptr, 1, d, &q);
    LEV_TRY(ensure(h->exact_gp, sizeof(double) * lev::gram_partial_doubles(n, d)));
    q.Gp = (double*)h->exact_gp.ptr;
    LEV_CUDA(lev::launch_gram_fp64(A, lda, n, d, q.Gp, q.G, st));
    return exact_reference_tail(h, q, n, d, tau, A, lda, nullptr, nullptr, nullptr, 0, theta, rank, perm, st);
}

int lev_exact_reference_csr(lev_handle* h, const int64_t* row_ptr, const int32_t* col, const float* val, int64_t n,
                            int64_t d, int64_t nnz, double tau, float* theta, int64_t* rank, int32_t* perm,
                            void* stream) {
    LEV_TRY(set_device(h));
    if (!row_ptr || (nnz > 0 && (!col || !val)) || !theta) return fail(LEV_EINVAL, "NULL array");
    if (n < 1 || n >= (int64_t)1 << 31 || d < 1 || d > 1024 || nnz < 0)
        return fail(LEV_EINVAL, "bad shape n=%lld d=%lld (d <= 1024)", (long long)n, (long long)d);
    if (tau <= 0) tau = 1e-5;
    if (tau < 1e-6) return fail(LEV_EINVAL, "tau = %g below the Gram route's resolution (1e-6)", tau);
    if (is_host_pointer(row_ptr) || (nnz > 0 && (is_host_pointer(col) || is_host_pointer(val))) ||
        is_host_pointer(theta))
        return fail(LEV_EINVAL, "lev_exact_reference_csr takes device arrays");
    cudaStream_t st = (cudaStream_t)stream;
    LEV_TRY(check_csr(h, row_ptr, n, nnz, 0u, st));
    LEV_TRY(ensure(h->qr, lev::qr_scratch_bytes(1, d)));
    lev::QrScratch q;
    lev::qr_scratch_carve(h->qr.ptr, 1, d, &q);
    LEV_TRY(csr_gram(h, row_ptr, col, val, n, d, q.G, st));
    return exact_reference_tail(h, q, n, d, tau, nullptr, 0, row_ptr, col, val, nnz, theta, rank, perm, st);
}

int lev_estimate_dense(lev_handle* h, const float* A, int64_t n, int64_t d, int64_t lda, const lev_params* p,
                       float* theta, int64_t* rank, int32_t* perm, void* stream) {
    LEV_TRY(set_device(h));
    Sizes z;
    LEV_TRY(resolve(p, n, d, &z));
    if (!A || !theta) return fail(LEV_EINVAL, "NULL array");
    if (lda < d) return fail(LEV_EINVAL, "lda < d");
    LEV_TRY(check_prec(p->sketch_prec, "sketch"));
    LEV_TRY(check_prec(p->final_prec, "final"));
    cudaStream_t st = (cudaStream_t)stream;
    const bool hostA = is_host_pointer(A), hostT = is_host_pointer(theta);
    float* dT = theta;
    if (hostT) {
        LEV_TRY(ensure(h->stageTheta, sizeof(float) * (size_t)n));
        dT = (float*)h->stageTheta.ptr;
    }
    LEV_TRY(ensure(h->Atilde, sizeof(float) * (size_t)z.m * d));
    const float* dA = A;
    int64_t ldA = lda;
    int slot = -1;
    if (hostA) {
        LEV_TRY(stage_host_dense(h, A, n, d, lda, st, &slot, &dA));
        ldA = d;
    }
    lev::QrScratch qs;
    auto kernels = [&]() -> int {
        LEV_TRY(sketch_common_dense(h, dA, n, d, ldA, p, z, (float*)h->Atilde.ptr, st));
        LEV_TRY(estimate_tail(h, z, d, p, perm, &qs, st));
        return final_dense(h, dA, n, d, ldA, (const float*)h->Mfull.ptr, z.k, p->final_prec, dT, st);
    };
    const int rc = kernels();
    if (slot >= 0) {
        // the stage buffer is free for a later copy once everything enqueued so far on `st` has run
        LEV_CUDA(cudaEventRecord(h->ev_used[slot], st));
        h->used_once[slot] = true;
    }
    LEV_TRY(rc);
    if (hostT) LEV_CUDA(cudaMemcpyAsync(theta, dT, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost, st));
    if (!rank && !hostA && !hostT) return LEV_OK;
    if (!rank && (p->flags & LEV_HOST_ASYNC)) return LEV_OK;
    return finish(h, qs, rank, st);
}

int lev_estimate_csr(lev_handle* h, const int64_t* row_ptr, const int32_t* col, const float* val, int64_t n,
                     int64_t d, int64_t nnz, const lev_params* p, float* theta, int64_t* rank, int32_t* perm,
                     void* stream) {
    LEV_TRY(set_device(h));
    Sizes z;
    LEV_TRY(resolve(p, n, d, &z));
    if (!row_ptr || (nnz > 0 && (!col || !val)) || !theta) return fail(LEV_EINVAL, "NULL array");
    if (nnz < 0) return fail(LEV_EINVAL, "nnz < 0");
    LEV_TRY(check_prec(p->sketch_prec, "sketch"));
    if (p->final_prec != LEV_FP32) return fail(LEV_EINVAL, "the CSR final pass supports LEV_FP32 only");
    cudaStream_t st = (cudaStream_t)stream;
    const bool hostA = is_host_pointer(row_ptr), hostT = is_host_pointer(theta);
    const int64_t* rp = row_ptr;
    const int32_t* cl = col;
    const float* vl = val;
    if (hostA) {
        LEV_TRY(ensure(h->csr_rp, sizeof(int64_t) * (size_t)(n + 1)));
        LEV_TRY(ensure(h->csr_col, sizeof(int32_t) * (size_t)nnz));
        LEV_TRY(ensure(h->csr_val, sizeof(float) * (size_t)nnz));
        LEV_CUDA(cudaMemcpyAsync(h->csr_rp.ptr, row_ptr, sizeof(int64_t) * (size_t)(n + 1), cudaMemcpyHostToDevice, st));
        if (nnz > 0) {
            LEV_CUDA(cudaMemcpyAsync(h->csr_col.ptr, col, sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice, st));
            LEV_CUDA(cudaMemcpyAsync(h->csr_val.ptr, val, sizeof(float) * (size_t)nnz, cudaMemcpyHostToDevice, st));
        }
        rp = (const int64_t*)h->csr_rp.ptr;
        cl = (const int32_t*)h->csr_col.ptr;
        vl = (const float*)h->csr_val.ptr;
    }
    float* dT = theta;
    if (hostT) {
        LEV_TRY(ensure(h->stageTheta, sizeof(float) * (size_t)n));
        dT = (float*)h->stageTheta.ptr;
    }
    LEV_TRY(check_csr(h, rp, n, nnz, p->flags, st));
    LEV_TRY(ensure(h->Atilde, sizeof(float) * (size_t)z.m * d));
    LEV_TRY(sketch_common_csr(h, rp, cl, vl, n, d, p, z, (float*)h->Atilde.ptr, st));
    lev::QrScratch qs;
    LEV_TRY(estimate_tail(h, z, d, p, perm, &qs, st));
    LEV_TRY(final_csr(h, rp, cl, vl, n, d, nnz, (const float*)h->Mfull.ptr, z.k, dT, st));
    if (hostT) LEV_CUDA(cudaMemcpyAsync(theta, dT, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost, st));
    if (!rank && !hostA && !hostT) return LEV_OK;
    return finish(h, qs, rank, st);
}

int lev_backward_dense(lev_handle* h, const float* A, int64_t n, int64_t d, int64_t lda, const lev_params* p,
                       const float* Atilde, const int32_t* perm, const int64_t* d_rank, const double* R,
                       const float* Mfull, const float* w, float* gradA, void* stream) {
    LEV_TRY(set_device(h));
    Sizes z;
    LEV_TRY(resolve(p, n, d, &z));
    if (!A || !Atilde || !perm || !d_rank || !R || !Mfull || !w || !gradA) return fail(LEV_EINVAL, "NULL array");
    if (lda < d) return fail(LEV_EINVAL, "lda < d");
    if (d > 256 || z.k > 256) return fail(LEV_EINVAL, "lev_backward_dense needs d <= 256 and k <= 256");
    LEV_TRY(check_prec(p->sketch_prec, "sketch"));
    cudaStream_t st = (cudaStream_t)stream;
    const bool identity = (p->flags & LEV_SKETCH_IDENTITY) != 0;
    // with the SRHT after the CountSketch the forward's G is m x t
    int64_t srht_t = 0;
    if (!identity && (p->flags & LEV_SKETCH_SRHT)) {
        srht_t = p->srht_t;
        if ((z.s & (z.s - 1)) != 0 || z.s > (int64_t(1) << 24))
            return fail(LEV_EINVAL, "LEV_SKETCH_SRHT needs s a power of two <= 2^24 (s = %lld)", (long long)z.s);
        if (srht_t < 1 || srht_t > z.s) return fail(LEV_EINVAL, "LEV_SKETCH_SRHT needs 1 <= srht_t <= s");
    }
    const int64_t gcols = srht_t > 0 ? srht_t : z.s;
    const float* g32 = nullptr;
    const __nv_bfloat16* ghi = nullptr;
    int64_t ldg = gcols;
    if (!identity) {
        // the G image the forward's sketch used (cached in the handle)
        const int kind = p->sketch_prec == LEV_FP32 ? 0 : (p->sketch_prec == LEV_TF32 ? 3 : 2);
        LEV_TRY(ensure_g(h, z.m, gcols, p->seed, kind, st, &g32, &ghi));
        if (kind != 0) ldg = (gcols + 63) / 64 * 64;
    }
    // the BF16 pair (kind 2) and the TF32 image (kind 3) hold the unscaled draws; the FP32 image is
    // N / sqrt(m)
    const float g_scale = (identity || p->sketch_prec == LEV_FP32) ? 1.f : (float)(1.0 / std::sqrt((double)z.m));
    const int chunks = lev::backward_chunks(n, d, z.k);
    LEV_TRY(ensure(h->bwd, lev::backward_scratch_bytes(n, d, z.k, z.s, z.m, srht_t, chunks)));
    LEV_CUDA(lev::launch_backward_dense(A, lda, n, d, z.s, z.m, z.k, p->seed, Atilde, perm, d_rank, R, Mfull, w, g32,
                                        ghi, ldg, g_scale, identity, srht_t, h->bwd.ptr, chunks, gradA, st));
    return LEV_OK;
}

}  // extern "C"
