// Rank-revealing QR of the sketch (FP64) and the small factor M = R_11^{-1} Omega (FP64 inputs and
// factor, a double-float triangular solve for d <= 1,024, FP64 above).
//
// Pivoted QR (Alg. 4 step 2 with the xGEQP3-style pivoting the paper's
// implementation uses, Sec. 7): one cooperatively launched persistent kernel.
// The FP64 working copy W (m x d, column-major) stays in global memory (it is
// L2 resident: 32 MB at 4096 x 1024). Every CTA owns a fixed set of columns.
// Step j, in every CTA after a grid barrier:
//   1. the pivot p_j is the active column with the largest trailing norm
//      ||W[j:, c]||^2 (recomputed exactly in step j-1, double-buffered by
//      parity; ties to the lowest column id) -- every CTA computes the same
//      argmax from the same data;
//   2. rank test |R_jj| = ||W[j:, p]|| <= tau |R_00| ends the factorisation;
//   3. the Householder vector of column p is read straight from W (v_j =
//      x_j - alpha, v_i = x_i) and applied to the CTA's own active columns,
//      which also write their new trailing norms and row j of R.
// A second small kernel orders the columns (pivots first, then the rest in
// increasing id) and writes R in pivoted order with diag(R) >= 0.
#include <cuda.h>

#include <mutex>

#include "df.cuh"
#include "lev_common.cuh"
#include "lev_kernels.cuh"
#include "lev_tc.cuh"

namespace lev {

namespace {

constexpr int QR_THREADS = 128;
constexpr int QR_WARPS = QR_THREADS / 32;

__device__ __forceinline__ double block_sum(double v, double* red) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int i = 0; i < QR_WARPS; ++i) t += red[i];
    return t;
}

struct QrArgs {
    const float* At;
    int m, d;
    double tau;
    const int32_t* forced;
    int forced_rank;
    QrScratch q;
    int32_t* status;
};

__global__ void __launch_bounds__(QR_THREADS) k_pivoted_qr(QrArgs a) {
    __shared__ double red[QR_WARPS];
    __shared__ double redv[QR_WARPS];
    __shared__ int redi[QR_WARPS];
    const int m = a.m, d = a.d;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    double* W = a.q.W;
    double* norms = a.q.norms;
    unsigned epoch = 0;

    // Phase 0: FP64 copy of the owned columns and their full norms.
    for (int c = blockIdx.x; c < d; c += gridDim.x) {
        double acc = 0.0;
        for (int i = tid; i < m; i += QR_THREADS) {
            const double x = (double)a.At[(int64_t)i * d + c];
            W[(int64_t)c * m + i] = x;
            acc += x * x;
        }
        acc = block_sum(acc, red);
        if (tid == 0) norms[c] = acc;
    }
    if (!grid_barrier(a.q.barrier, epoch, a.status)) return;

    const int steps = a.forced ? min(a.forced_rank, min(m, d)) : min(m, d);
    double r00 = 0.0;
    int j = 0;
    for (; j < steps; ++j) {
        const double* cur = norms + (j & 1) * d;
        double* nxt = norms + ((j + 1) & 1) * d;
        // 1. pivot
        int p;
        if (a.forced) {
            p = a.forced[j];
            if (p < 0 || p >= d || cur[p] < 0.0) break;       // invalid or repeated pivot
        } else {
            double bv = -2.0;
            int bi = d;
            for (int c = tid; c < d; c += QR_THREADS) {
                const double v = cur[c];
                if (v > bv) { bv = v; bi = c; }                   // c ascending: first max kept
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
            }
            __syncthreads();
            if (lane == 0) { redv[wid] = bv; redi[wid] = bi; }
            __syncthreads();
            bv = redv[0]; bi = redi[0];
            for (int i = 1; i < QR_WARPS; ++i)
                if (redv[i] > bv || (redv[i] == bv && redi[i] < bi)) { bv = redv[i]; bi = redi[i]; }
            p = bi;
        }
        const double nrm2 = cur[p];
        const double nrm = sqrt(fmax(nrm2, 0.0));
        // 2. rank test
        if (j == 0) r00 = nrm;
        if (!(nrm2 > 0.0)) break;
        if (!a.forced && nrm <= a.tau * r00) break;
        // 3. reflector from column p: H x = alpha e_j
        const double* x = W + (int64_t)p * m;
        const double x0 = x[j];
        const double alpha = (x0 >= 0.0) ? -nrm : nrm;
        const double v0 = x0 - alpha;
        const double beta = 1.0 / (nrm * (nrm + fabs(x0)));   // 2 / (v^T v)
        for (int c = blockIdx.x; c < d; c += gridDim.x) {
            if (c == p) continue;
            if (cur[c] < 0.0) {                                 // pivoted earlier: stays inactive
                if (tid == 0) nxt[c] = -1.0;
                continue;
            }
            double* w = W + (int64_t)c * m;
            double dot = 0.0;
            for (int i = j + 1 + tid; i < m; i += QR_THREADS) dot += x[i] * w[i];
            dot = block_sum(dot, red) + v0 * w[j];
            const double f = beta * dot;
            double acc = 0.0;
            for (int i = j + 1 + tid; i < m; i += QR_THREADS) {
                const double nv = w[i] - f * x[i];
                w[i] = nv;
                acc += nv * nv;
            }
            acc = block_sum(acc, red);
            if (tid == 0) {
                const double wj = w[j] - f * v0;
                w[j] = wj;
                a.q.Rorig[(int64_t)j * d + c] = wj;
                nxt[c] = acc;
            }
        }
        if (blockIdx.x == 0 && tid == 0) {
            a.q.Rorig[(int64_t)j * d + p] = alpha;
            a.q.piv[j] = p;
        }
        // the pivot column's owner retires it
        if ((p % gridDim.x) == (int)blockIdx.x && tid == 0) nxt[p] = -1.0;
        if (!grid_barrier(a.q.barrier, epoch, a.status)) return;
    }
    if (blockIdx.x == 0 && tid == 0) *a.q.rank = j;
}

// perm: pivots first, then the other columns ascending; R row-major in pivoted
// column order with diag(R) >= 0; rows >= rank are zero. k_assemble_perm runs
// in one CTA (a block-wide scan places the unpivoted columns), k_assemble_r on
// a grid over the rows of R.
__global__ void __launch_bounds__(1024) k_assemble_perm(QrScratch q, int d, int32_t* perm) {
    extern __shared__ int mark[];
    __shared__ int warp_tot[32];
    __shared__ int carry;
    const int r = (int)*q.rank;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    for (int c = t; c < d; c += blockDim.x) mark[c] = 0;
    if (t == 0) carry = r;
    __syncthreads();
    for (int j = t; j < r; j += blockDim.x) {
        mark[q.piv[j]] = 1;
        perm[j] = q.piv[j];
    }
    __syncthreads();
    for (int base = 0; base < d; base += blockDim.x) {
        const int c = base + t;
        const int un = (c < d && !mark[c]) ? 1 : 0;
        int incl = un;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) warp_tot[w] = incl;
        __syncthreads();
        if (w == 0) {
            const int wt = warp_tot[lane];
            int wi = wt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += y;
            }
            warp_tot[lane] = wi - wt;
        }
        __syncthreads();
        const int pos = carry + warp_tot[w] + incl - un;
        if (un) perm[pos] = c;
        __syncthreads();
        if (t == blockDim.x - 1) carry = pos + un;
        __syncthreads();
    }
}

__global__ void k_assemble_r(QrScratch q, int d, const int32_t* __restrict__ perm, double* __restrict__ R) {
    const int r = (int)*q.rank;
    const int j = blockIdx.x;                        // one CTA per row of R
    if (j >= d) return;
    double sgn = 1.0;
    if (j < r) sgn = (q.Rorig[(int64_t)j * d + q.piv[j]] < 0.0) ? -1.0 : 1.0;
    for (int t = threadIdx.x; t < d; t += blockDim.x) {
        double v = 0.0;
        if (j < r && t >= j) {
            v = q.Rorig[(int64_t)j * d + perm[t]];
            // entries the Gram route never wrote (columns retired before step j) hold its
            // "unwritten" pattern, a signalling NaN that arithmetic never produces
            if (__double_as_longlong(v) == (long long)0xFFF40000DEADBEEFull) v = 0.0;
            v *= sgn;
        }
        R[(int64_t)j * d + t] = v;
    }
}

// M = R_11^{-1} Omega by back-substitution in blocks of 32 rows, one warp per
// column q of Omega (the column lives in shared memory: Omega first, then M).
// For the block of rows p0..p0+31 lane l owns row i = p0 + l: it first sums
// the contributions of the rows below the block (already solved) on its own,
// then the 32 x 32 triangle is solved bottom-up, each solved entry broadcast
// with one shuffle and applied by the lanes above it.
__global__ void k_omega_factor(const double* __restrict__ R, const int32_t* __restrict__ perm,
                               const int64_t* __restrict__ d_rank, int d, int k, uint64_t key,
                               double inv_sqrt_k, int identity, float* __restrict__ Mfull) {
    extern __shared__ double colbuf[];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = blockIdx.x * (blockDim.x >> 5) + wib;
    if (q >= k) return;
    int r = (int)*d_rank;
    r = r < 0 ? 0 : (r > d ? d : r);
    double* Ms = colbuf + (int64_t)wib * d;
    for (int p = lane; p < r; p += 32)
        Ms[p] = identity ? (p == q ? 1.0 : 0.0) : box_muller(key, (uint64_t)p * k + q) * inv_sqrt_k;
    __syncwarp();
    for (int p0 = ((r - 1) / 32) * 32; r > 0 && p0 >= 0; p0 -= 32) {
        const int i = p0 + lane;
        const bool valid = i < r;
        const double* Ri = R + (int64_t)(valid ? i : 0) * d;
        double rhs = valid ? Ms[i] : 0.0;
        double acc0 = 0.0, acc1 = 0.0;
        if (valid) {
            int t = p0 + 32;
            for (; t + 1 < r; t += 2) {
                acc0 = fma(Ri[t], Ms[t], acc0);
                acc1 = fma(Ri[t + 1], Ms[t + 1], acc1);
            }
            if (t < r) acc0 = fma(Ri[t], Ms[t], acc0);
        }
        rhs -= acc0 + acc1;
        double rb[32];
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) rb[jj] = (valid && p0 + jj < r) ? Ri[p0 + jj] : 0.0;
        const double inv = valid ? 1.0 / Ri[i] : 0.0;
        double x = 0.0;
#pragma unroll
        for (int jj = 31; jj >= 0; --jj) {
            if (lane == jj) x = rhs * inv;
            const double xj = __shfl_sync(0xffffffffu, x, jj);
            if (lane < jj) rhs = fma(-rb[jj], xj, rhs);
        }
        if (valid) Ms[i] = x;
        __syncwarp();
    }
    for (int p = lane; p < r; p += 32) Mfull[(int64_t)perm[p] * k + q] = (float)Ms[p];
}

// G (kc x kc FP64, full) = Omega_kc Omega_kc^T, one thread an entry, the k products summed in order.
__global__ void k_omega_gram(const double* __restrict__ Om, int kc, int k, double* __restrict__ G) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)kc * kc;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / kc), j = (int)(e % kc);
        const int a = min(i, j), b = max(i, j);                  // the same sum for (i, j) and (j, i)
        const double* x = Om + (int64_t)a * k;
        const double* y = Om + (int64_t)b * k;
        double s = 0.0;
        for (int q = 0; q < k; ++q) s = fma(x[q], y[q], s);
        G[e] = s;
    }
}

__global__ void k_iota(int32_t* v, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v[i] = i;
}

// Omega (d x k FP64): entry (p, q) = N(0,1)/sqrt(k) from stream 3 at counter p k + q, for every pivot
// position p < d (a call with rank r uses rows 0..r-1). Grid-wide; the handle caches the result.
__global__ void k_gen_omega(uint64_t key, int d, int k, double inv_sqrt_k, double* __restrict__ Om) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)d * k;
         e += (int64_t)gridDim.x * blockDim.x)
        Om[e] = box_muller(key, (uint64_t)e) * inv_sqrt_k;
}

// Rs (d x d FP64): Rs[j][i] = R[i][j] / R[i][i] for i < j < r, the strictly upper part of R_11
// scaled to a unit diagonal and transposed, so that step j of the substitution reads row j.
__global__ void k_scaled_transpose(const double* __restrict__ R, const int64_t* __restrict__ d_rank, int d,
                                   double* __restrict__ Rs) {
    const int r = (int)min(max(*d_rank, (int64_t)0), (int64_t)d);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)r * r;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / r), i = (int)(e % r);
        if (i < j) Rs[(int64_t)j * d + i] = R[(int64_t)i * d + j] / R[(int64_t)i * d + i];
    }
}

// The same coefficients as double-float pairs (the solve below runs in FP32 arithmetic only).
__global__ void k_scaled_transpose_df(const double* __restrict__ R, const int64_t* __restrict__ d_rank, int d,
                                      float2* __restrict__ Rs) {
    const int r = (int)min(max(*d_rank, (int64_t)0), (int64_t)d);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)r * r;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / r), i = (int)(e % r);
        if (i < j) Rs[(int64_t)j * d + i] = df_from_double(R[(int64_t)i * d + j] / R[(int64_t)i * d + i]);
    }
}

// M = R_11^{-1} Omega column by column, one CTA per column q and one thread per row i (r <= 1024),
// in double-float arithmetic (FP32 pairs, about 48 bits; FP64 runs at 1/64 of the FP32 rate on
// GB300 and bound this solve at d = 1,024): with the unit-diagonal form
// x_i = w_i / R_ii - sum_{j > i} (R_ij / R_ii) x_j, step j (from the bottom) publishes x_j through
// shared memory (double-buffered by step parity, one barrier per step) and every thread i < j
// subtracts Rs[j][i] x_j, so each row sees its updates in the order j = r-1, ..., i+1. The
// coefficients of the next eight steps are loaded ahead. Row i of M goes to row perm[i] of Mfull,
// rounded to FP32.
// With the factor Lc of Omega's Gram matrix (upper U, row q holding column q of L = U^T) and
// r < k, r <= *d_kc, the right-hand side is column q of L_r instead and the CTAs q >= r leave
// their column 0.
constexpr int OMEGA_PF = 8;
__global__ void __launch_bounds__(1024) k_omega_solve(const double* __restrict__ R, const float2* __restrict__ Rs,
                                                      const double* __restrict__ Om, const double* __restrict__ Lc,
                                                      int kc, const int64_t* __restrict__ d_kc,
                                                      const int32_t* __restrict__ perm,
                                                      const int64_t* __restrict__ d_rank, int d, int k, int identity,
                                                      float* __restrict__ Mfull) {
    __shared__ float2 xs[2];
    const int q = blockIdx.x, i = threadIdx.x;
    const int r = (int)min(max(*d_rank, (int64_t)0), (int64_t)d);
    const bool reduced = Lc != nullptr && !identity && r < k && r <= kc && (int64_t)r <= *d_kc;
    if (reduced && q >= r) return;                               // the whole CTA: Mfull column q stays 0
    float2 x = make_float2(0.f, 0.f);
    if (i < r) {
        const double w = identity ? (i == q ? 1.0 : 0.0)
                                  : (reduced ? Lc[(int64_t)q * kc + i] : Om[(int64_t)i * k + q]);
        x = df_from_double(w / R[(int64_t)i * d + i]);
    }
    // ring of coefficients: c[t] holds Rs[j - t][i] for the current step j
    float2 c[OMEGA_PF];
#pragma unroll
    for (int t = 0; t < OMEGA_PF; ++t) {
        const int j = r - 1 - t;
        c[t] = (j > i) ? Rs[(int64_t)j * d + i] : make_float2(0.f, 0.f);
    }
    for (int j = r - 1; j >= 0; --j) {
        const float2 cj = c[0];
#pragma unroll
        for (int t = 0; t + 1 < OMEGA_PF; ++t) c[t] = c[t + 1];
        const int jn = j - OMEGA_PF;
        c[OMEGA_PF - 1] = (jn > i) ? Rs[(int64_t)jn * d + i] : make_float2(0.f, 0.f);
        if (i == j) xs[j & 1] = x;
        __syncthreads();
        if (i < j) x = df_sub_mul(x, cj, xs[j & 1]);
    }
    if (i < r) Mfull[(int64_t)perm[i] * k + q] = (float)df_to_double(x);
}

}  // namespace

// The Gram route (one cooperative grid over the SMs) serves d <= kGramMaxD and
// thresholds tau >= kGramMinTau (above its noise floor of about sqrt(m u)).
constexpr int64_t kGramMaxD = 1024;
constexpr double kGramMinTau = 1e-6;

// One layout for both the size and the carve: every piece starts on a 256-byte boundary.
static size_t qr_layout(int64_t m, int64_t d, char* base, QrScratch* q) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char* r = base ? base + off : nullptr;
        off += (bytes + 255) / 256 * 256;
        return r;
    };
    char* W = take(sizeof(double) * (size_t)(m * d));
    char* norms = take(sizeof(double) * (size_t)(2 * d));
    char* Rorig = take(sizeof(double) * (size_t)(d * d));
    char* piv = take(sizeof(int32_t) * (size_t)d);
    char* rank = take(sizeof(int64_t));
    char* barrier = take(sizeof(unsigned));
    const bool gram = d <= kGramMaxD;
    char* G = gram ? take(sizeof(double) * (size_t)(d * d)) : nullptr;
    char* Gp = gram ? take(sizeof(double) * gram_partial_doubles(m, d)) : nullptr;
    char* U = gram ? take(sizeof(double) * (size_t)(d * d)) : nullptr;
    if (q) {
        q->W = reinterpret_cast<double*>(W);
        q->norms = reinterpret_cast<double*>(norms);
        q->Rorig = reinterpret_cast<double*>(Rorig);
        q->piv = reinterpret_cast<int32_t*>(piv);
        q->rank = reinterpret_cast<int64_t*>(rank);
        q->barrier = reinterpret_cast<unsigned*>(barrier);
        q->G = reinterpret_cast<double*>(G);
        q->Gp = reinterpret_cast<double*>(Gp);
        q->U = reinterpret_cast<double*>(U);
    }
    return off;
}

size_t qr_scratch_bytes(int64_t m, int64_t d) { return qr_layout(m, d, nullptr, nullptr); }

void qr_scratch_carve(void* base, int64_t m, int64_t d, QrScratch* q) {
    qr_layout(m, d, static_cast<char*>(base), q);
}

cudaError_t launch_pivoted_qr(const float* Atilde, int64_t m, int64_t d, double tau,
                              const int32_t* forced_perm, int64_t forced_rank,
                              const QrScratch& q, int32_t* perm, double* R, int32_t* status,
                              int num_sms, cudaStream_t st, const cudaEvent_t* marks) {
    cudaError_t e;
    if (marks && (e = cudaEventRecord(marks[0], st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(q.barrier, 0, sizeof(unsigned), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(q.Rorig, 0, sizeof(double) * (size_t)(d * d), st)) != cudaSuccess) return e;
    if (d <= kGramMaxD && (forced_perm || tau >= kGramMinTau)) {
        e = launch_gram_pivoted_cholesky(Atilde, m, d, tau, forced_perm, forced_rank, q, status, st,
                                         marks ? marks[1] : nullptr);
        if (e != cudaSuccess) return e;
    } else {
        if (marks && (e = cudaEventRecord(marks[1], st)) != cudaSuccess) return e;
        int occ = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pivoted_qr, QR_THREADS, 0)) != cudaSuccess)
            return e;
        int64_t grid = (int64_t)num_sms * (occ < 1 ? 1 : (occ > 2 ? 2 : occ));
        if (grid > d) grid = d;
        if (grid < 1) grid = 1;
        QrArgs args{Atilde, (int)m, (int)d, tau, forced_perm, (int)forced_rank, q, status};
        void* kargs[] = {&args};
        e = cudaLaunchCooperativeKernel((const void*)k_pivoted_qr, dim3((unsigned)grid), dim3(QR_THREADS),
                                        kargs, 0, st);
        if (e != cudaSuccess) return e;
    }
    if (marks && (e = cudaEventRecord(marks[2], st)) != cudaSuccess) return e;
    k_assemble_perm<<<1, 1024, sizeof(int) * (size_t)d, st>>>(q, (int)d, perm);
    k_assemble_r<<<(unsigned)d, 256, 0, st>>>(q, (int)d, perm, R);
    return cudaGetLastError();
}

cudaError_t launch_scaled_transpose(const double* R, const int64_t* d_rank, int64_t d, double* Rs, cudaStream_t st) {
    int grid = (int)((d * d + 255) / 256);
    if (grid > 152 * 8) grid = 152 * 8;
    k_scaled_transpose<<<grid, 256, 0, st>>>(R, d_rank, (int)d, Rs);
    return cudaGetLastError();
}

cudaError_t launch_gen_omega(uint64_t seed, int64_t d, int64_t k, double* Omega, cudaStream_t st) {
    const int64_t total = d * k;
    int grid = (int)((total + 255) / 256);
    if (grid > 152 * 8) grid = 152 * 8;
    if (grid < 1) grid = 1;
    k_gen_omega<<<grid, 256, 0, st>>>(stream_key(seed, kStreamOmega), (int)d, (int)k, 1.0 / sqrt((double)k), Omega);
    return cudaGetLastError();
}

cudaError_t launch_factor_gram(int64_t m, int64_t d, double tau, const int32_t* forced, int64_t forced_rank,
                               const QrScratch& q, int32_t* perm, double* R, int32_t* status, cudaStream_t st) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(q.Rorig, 0, sizeof(double) * (size_t)(d * d), st)) != cudaSuccess) return e;
    if ((e = launch_pivoted_cholesky(m, d, tau, forced, forced_rank, q, status, st)) != cudaSuccess) return e;
    k_assemble_perm<<<1, 1024, sizeof(int) * (size_t)d, st>>>(q, (int)d, perm);
    k_assemble_r<<<(unsigned)d, 256, 0, st>>>(q, (int)d, perm, R);
    return cudaGetLastError();
}

cudaError_t launch_omega_chol(const double* Omega, int64_t d, int64_t k, const QrScratch& q, int32_t* iota,
                              int32_t* status, cudaStream_t st) {
    const int64_t kc = d < k ? d : k;
    if (kc < 1 || kc > kGramMaxD) return cudaErrorInvalidValue;
    int grid = (int)((kc * kc + 255) / 256);
    if (grid > 152 * 4) grid = 152 * 4;
    k_omega_gram<<<grid, 256, 0, st>>>(Omega, (int)kc, (int)k, q.G);
    k_iota<<<(unsigned)((kc + 255) / 256), 256, 0, st>>>(iota, (int)kc);
    cudaError_t e = cudaMemsetAsync(q.Rorig, 0, sizeof(double) * (size_t)(kc * kc), st);
    if (e != cudaSuccess) return e;
    return launch_pivoted_cholesky(k, kc, 0.0, iota, kc, q, status, st);
}

cudaError_t launch_omega_factor(const double* R, const int32_t* perm, const int64_t* d_rank,
                                int64_t d, int64_t k, uint64_t seed, bool omega_identity,
                                const double* Omega, const double* Lc, int64_t kc, const int64_t* d_kc,
                                double* Rs, float* Mfull, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(Mfull, 0, sizeof(float) * (size_t)(d * k), st);
    if (e != cudaSuccess) return e;
    if (d <= 1024 && Rs && (Omega || omega_identity)) {
        int grid = (int)((d * d + 255) / 256);
        if (grid > 152 * 8) grid = 152 * 8;
        float2* Rs2 = reinterpret_cast<float2*>(Rs);                // the same d x d bytes
        k_scaled_transpose_df<<<grid, 256, 0, st>>>(R, d_rank, (int)d, Rs2);
        const int threads = (int)((d + 31) / 32 * 32);
        k_omega_solve<<<(unsigned)k, threads, 0, st>>>(R, Rs2, Omega, Lc && d_kc ? Lc : nullptr, (int)kc, d_kc,
                                                       perm, d_rank, (int)d, (int)k, omega_identity ? 1 : 0, Mfull);
        return cudaGetLastError();
    }
    const int warps = 1;                              // spread the FP64 work over the SMs
    const size_t smem = sizeof(double) * (size_t)d * warps;
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(k_omega_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int grid = (int)((k + warps - 1) / warps);
    k_omega_factor<<<grid, 32 * warps, smem, st>>>(R, perm, d_rank, (int)d, (int)k, stream_key(seed, kStreamOmega),
                                                   1.0 / sqrt((double)k), omega_identity ? 1 : 0, Mfull);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// lev_rrqr_noalloc: the same pivoted QR with its scratch in a fixed device array.
//
// For callers that must not call cudaMalloc: code that runs inside another
// allocator's fixed memory budget (a serving framework's pool), and
// latency-critical paths where the implicit device synchronisation of
// cudaMalloc/cudaFree is not acceptable. The scratch is a file-scope
// __device__ array of kRrqrNoAllocBytes that every GPU which loads the library
// holds until the process exits. Host code must not pass the array's name to a
// kernel (in host code it is only a stand-in for the device symbol); its device
// address is looked up with cudaGetSymbolAddress on the first call made in a
// CUDA context (a device's primary context, or a context made current by the
// caller) and looked up again whenever the current context differs from the one
// the cached address belongs to (after a cudaDeviceReset, for example). That
// first call should come before any stream capture. All calls share the array:
// the pieces that must start at zero (barrier counter, status word, R scratch)
// are cleared by every call on its stream, and calls that overlap on the GPU
// race with one another.
// ---------------------------------------------------------------------------
namespace {
constexpr size_t kRrqrNoAllocBytes = size_t(8) << 20;   // 8 MiB
__device__ __align__(256) unsigned char g_rrqr_noalloc_scratch[kRrqrNoAllocBytes];
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
struct NoAllocAddr {
    unsigned long long ctx_id = 0;   // CUDA context the address belongs to
    void* addr = nullptr;
};
NoAllocAddr g_noalloc_addr[kMaxDevices];

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// Unique id of the calling thread's current CUDA context (0 if none is current or the driver
// entry points are unavailable). Called with g_noalloc_mu held.
unsigned long long current_ctx_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool resolved = false;
    if (!resolved) {
        resolved = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(p);
        cudaGetLastError();
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}
}  // namespace

}  // namespace lev

extern "C" int lev_rrqr_noalloc(const float* Atilde, int64_t m, int64_t d, double tau, int32_t* perm,
                                double* R, int64_t* rank, void* stream) {
    using namespace lev;
    if (!Atilde || !perm || !R) return handle_fail(LEV_EINVAL, "lev_rrqr_noalloc: NULL array");
    if (m < 1 || d < 1 || d > 4096 || m > (1 << 20))
        return handle_fail(LEV_EINVAL, "lev_rrqr_noalloc: bad shape");
    const size_t need = qr_layout(m, d, nullptr, nullptr) + 256;    // + status word
    if (need > kRrqrNoAllocBytes)
        return handle_fail(LEV_EINVAL,
                           "lev_rrqr_noalloc: m x d too large for the fixed 8 MiB scratch "
                           "(the QR working set is about 8 (m d + 3 d^2) bytes plus the Gram split partials)");
    if (tau <= 0) tau = 1e-5;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return handle_fail(LEV_ECUDA, "lev_rrqr_noalloc: no current CUDA device");
    }
    char* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        NoAllocAddr& slot = g_noalloc_addr[dev];
        const unsigned long long ctx = current_ctx_id();
        if (!slot.addr || ctx == 0 || ctx != slot.ctx_id) {
            void* addr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&addr, g_rrqr_noalloc_scratch);
            if (e != cudaSuccess || !addr) {
                cudaGetLastError();
                slot.addr = nullptr;
                return handle_fail(LEV_ECUDA, "lev_rrqr_noalloc: cudaGetSymbolAddress failed");
            }
            slot.addr = addr;
            slot.ctx_id = current_ctx_id();   // the lookup made the runtime's context current
        }
        base = static_cast<char*>(slot.addr);
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    QrScratch q;
    const size_t status_off = qr_layout(m, d, base, &q);
    int32_t* status = reinterpret_cast<int32_t*>(base + status_off);
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess && sms < 1) e = cudaErrorInvalidValue;
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int32_t), st);
    if (e == cudaSuccess) e = launch_pivoted_qr(Atilde, m, d, tau, nullptr, 0, q, perm, R, status, sms, st);
    if (e != cudaSuccess) return handle_fail(LEV_ECUDA, cudaGetErrorString(e));
    if (!rank) return LEV_OK;
    int64_t r = 0;
    int32_t flag = 0;
    e = cudaMemcpyAsync(&r, q.rank, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, status, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return handle_fail(LEV_ECUDA, cudaGetErrorString(e));
    if (flag != 0) return handle_fail(LEV_ETIMEOUT, "lev_rrqr_noalloc: a bounded device wait gave up");
    *rank = r;
    if (r == 0) return handle_fail(LEV_ERANK0, "numerical rank is 0");
    return LEV_OK;
}

