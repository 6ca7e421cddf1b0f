// Fused final pass theta~_i = ||A_i Mfull||^2 (Alg. 8 step 5), FP32 SIMT forms.
//
// Mfull (d x k) holds R_11^{-1} Omega on the rows of the selected columns K and
// zeros elsewhere, so A Mfull = A_K R_11^{-1} Omega. The n x k product never
// leaves registers: each CTA squares and sums its tile rows in the epilogue
// (warp shuffles) and writes only theta~ (n floats).
//
// Dense: 64-row x 256-column register tile, 8 x 8 per thread, A and Mfull
// staged through shared memory in 16-wide k slices (two stages).
// CSR: one warp per row (product form of Lemma 1): the warp broadcasts each
// (col, val) of the row and every lane accumulates 8 columns of
// val * Mfull[col, :] with 128-bit loads; then squares and warp-sums.
#include "lev_common.cuh"
#include "lev_kernels.cuh"

namespace lev {

namespace {

constexpr int FD_BM = 64, FD_BN = 256, FD_BK = 16;

template <bool VEC>
__global__ void __launch_bounds__(256) k_final_dense_fp32(
        const float* __restrict__ A, int64_t lda, int64_t n, int d,
        const float* __restrict__ M, int k, float* __restrict__ theta) {
    __shared__ __align__(16) float As[2][FD_BK][FD_BM];
    __shared__ __align__(16) float Ms[2][FD_BK][FD_BN];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int64_t row0 = (int64_t)blockIdx.x * FD_BM;
    // loader coordinates: A tile 64 x 16 (one float4 per thread), M tile 16 x 256 (4 float4)
    const int a_r = t >> 2, a_c = (t & 3) * 4;
    const int m_r = t >> 4, m_c = (t & 15) * 4;
    float th[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) th[i] = 0.f;

    for (int q0 = 0; q0 < k; q0 += FD_BN) {
        float acc[8][8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
        float ra[4], rm[4][4];
        auto load = [&](int k0) {
            const int64_t gr = row0 + a_r;
            if (VEC) {
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (gr < n && k0 + a_c < d) v = __ldg(reinterpret_cast<const float4*>(A + gr * lda + k0 + a_c));
                ra[0] = v.x; ra[1] = v.y; ra[2] = v.z; ra[3] = v.w;
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int c = k0 + a_c + i;
                    ra[i] = (gr < n && c < d) ? __ldg(A + gr * lda + c) : 0.f;
                }
            }
            const int mr = k0 + m_r;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int c = q0 + m_c + 64 * u;
                if (VEC) {
                    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (mr < d && c < k) v = __ldg(reinterpret_cast<const float4*>(M + (int64_t)mr * k + c));
                    rm[u][0] = v.x; rm[u][1] = v.y; rm[u][2] = v.z; rm[u][3] = v.w;
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        rm[u][i] = (mr < d && c + i < k) ? __ldg(M + (int64_t)mr * k + c + i) : 0.f;
                }
            }
        };
        auto store = [&](int st) {
#pragma unroll
            for (int i = 0; i < 4; ++i) As[st][a_c + i][a_r] = ra[i];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                *reinterpret_cast<float4*>(&Ms[st][m_r][m_c + 64 * u]) =
                    make_float4(rm[u][0], rm[u][1], rm[u][2], rm[u][3]);
        };
        int st = 0;
        load(0);
        __syncthreads();                 // previous chunk's readers are done
        store(0);
        __syncthreads();
        for (int k0 = 0; k0 < d; k0 += FD_BK) {
            const bool more = (k0 + FD_BK) < d;
            if (more) load(k0 + FD_BK);
#pragma unroll
            for (int kk = 0; kk < FD_BK; ++kk) {
                const float4 a0 = *reinterpret_cast<const float4*>(&As[st][kk][w * 4]);
                const float4 a1 = *reinterpret_cast<const float4*>(&As[st][kk][32 + w * 4]);
                const float4 b0 = *reinterpret_cast<const float4*>(&Ms[st][kk][lane * 4]);
                const float4 b1 = *reinterpret_cast<const float4*>(&Ms[st][kk][128 + lane * 4]);
                const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
            }
            if (more) {
                store(st ^ 1);
                __syncthreads();
                st ^= 1;
            }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float sq = 0.f;
#pragma unroll
            for (int j = 0; j < 8; ++j) sq = fmaf(acc[i][j], acc[i][j], sq);
            th[i] += sq;
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float v = warp_sum(th[i]);
        const int64_t r = row0 + (i < 4 ? w * 4 + i : 32 + w * 4 + (i - 4));
        if (lane == 0 && r < n) theta[r] = v;
    }
}

// ||a_i M||^2 of one CSR row (entries p0 .. p1), this lane's share (the caller sums the warp): lane
// owns columns q0 + lane*4 + {0..3} and q0 + 128 + lane*4 + {0..3} of each 256-column chunk.
template <bool VEC>
__device__ __forceinline__ float csr_row_norm(int64_t p0, int64_t p1, const int32_t* __restrict__ col,
                                              const float* __restrict__ val, int d, const float* __restrict__ M,
                                              int k, int lane) {
    float total = 0.f;
    for (int q0 = 0; q0 < k; q0 += 256) {
        float y[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) y[j] = 0.f;
        for (int64_t pb = p0; pb < p1; pb += 32) {
            const int cnt = (int)min((int64_t)32, p1 - pb);
            int my_c = -1;
            float my_v = 0.f;
            if (lane < cnt) {
                my_c = col[pb + lane];
                my_v = val[pb + lane];
                if ((unsigned)my_c >= (unsigned)d) { my_c = 0; my_v = 0.f; }
            }
            int u = 0;
            for (; u + 4 <= cnt; u += 4) {
                float4 m0[4], m1[4];
                float vv[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int c = __shfl_sync(0xffffffffu, my_c, u + e);
                    vv[e] = __shfl_sync(0xffffffffu, my_v, u + e);
                    const float* Mr = M + (int64_t)c * k + q0;
                    if (VEC) {
                        m0[e] = (q0 + lane * 4 < k) ? __ldg(reinterpret_cast<const float4*>(Mr + lane * 4))
                                                    : make_float4(0.f, 0.f, 0.f, 0.f);
                        m1[e] = (q0 + 128 + lane * 4 < k)
                                    ? __ldg(reinterpret_cast<const float4*>(Mr + 128 + lane * 4))
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
                    } else {
                        float tmp[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const int q = q0 + (j < 4 ? lane * 4 + j : 128 + lane * 4 + j - 4);
                            tmp[j] = (q < k) ? __ldg(M + (int64_t)c * k + q) : 0.f;
                        }
                        m0[e] = make_float4(tmp[0], tmp[1], tmp[2], tmp[3]);
                        m1[e] = make_float4(tmp[4], tmp[5], tmp[6], tmp[7]);
                    }
                }
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    y[0] = fmaf(vv[e], m0[e].x, y[0]); y[1] = fmaf(vv[e], m0[e].y, y[1]);
                    y[2] = fmaf(vv[e], m0[e].z, y[2]); y[3] = fmaf(vv[e], m0[e].w, y[3]);
                    y[4] = fmaf(vv[e], m1[e].x, y[4]); y[5] = fmaf(vv[e], m1[e].y, y[5]);
                    y[6] = fmaf(vv[e], m1[e].z, y[6]); y[7] = fmaf(vv[e], m1[e].w, y[7]);
                }
            }
            for (; u < cnt; ++u) {
                const int c = __shfl_sync(0xffffffffu, my_c, u);
                const float v = __shfl_sync(0xffffffffu, my_v, u);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int q = q0 + (j < 4 ? lane * 4 + j : 128 + lane * 4 + j - 4);
                    if (q < k) y[j] = fmaf(v, __ldg(M + (int64_t)c * k + q), y[j]);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) total = fmaf(y[j], y[j], total);
    }
    return total;
}

// CSR, warp per row: ||a_i Mfull||^2.
template <bool VEC>
__global__ void __launch_bounds__(256) k_final_csr_fp32(
        const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
        const float* __restrict__ val, int64_t n, int d, const float* __restrict__ M, int k,
        float* __restrict__ theta) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < n; i += nwarps) {
        const float total = warp_sum(csr_row_norm<VEC>(row_ptr[i], row_ptr[i + 1], col, val, d, M, k, lane));
        if (lane == 0) theta[i] = total;
    }
}

// CSR with the second form of Lemma 1 for short rows: theta~_i = a_i P a_i^T, P = Mfull Mfull^T
// (d x d), i.e. the sum over the entry pairs p <= q of (2 - [p = q]) a_p a_q P[c_p][c_q]:
// nnz_i^2 / 2 terms from a matrix that sits in L2, against nnz_i k products and nnz_i rows of
// Mfull for the first form. Repeated columns are handled as they stand (the double sum over the
// pairs is the quadratic form); columns outside [0, d) count as zero.
//
// The terms are summed in FP32 arithmetic with double-float accuracy (FP64 runs at 1/64 of the FP32
// rate here and made this pass FP64-bound): P is held as a pair hi + lo of FP32 matrices (the FP64
// Gram matrix of Mfull^T split once), each term's product is formed with its rounding errors
// (TwoProduct of the two entries, the pair of P multiplied in), and every lane accumulates its
// terms with TwoSum, so a row carries an error of a few 2^-48 of sum |terms| rather than 2^-24.
__device__ __forceinline__ void df_add(float& sh, float& sl, float th, float tl) {
    const float s = __fadd_rn(sh, th);
    const float bb = __fsub_rn(s, sh);
    float e = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(th, bb));
    e = __fadd_rn(e, __fadd_rn(sl, tl));
    sh = __fadd_rn(s, e);
    sl = __fsub_rn(e, __fsub_rn(sh, s));
}
// (w a b) (P_hi + P_lo) as an unevaluated pair (w = 1 or 2, exact).
__device__ __forceinline__ void df_term(float a, float b, float w, float2 P, float& th, float& tl) {
    const float x = __fmul_rn(a, b);
    const float xe = __fmaf_rn(a, b, -x);                             // a b = x + xe exactly
    const float xw = __fmul_rn(x, w), xwe = __fmul_rn(xe, w);          // exact (w a power of two)
    th = __fmul_rn(xw, P.x);
    tl = __fmaf_rn(xw, P.x, -th);
    tl = __fmaf_rn(xw, P.y, tl);
    tl = __fmaf_rn(xwe, P.x, tl);
}

// Rows with LO < len <= SEG entries (an empty row gets 0): SEG lanes a row, 32 / SEG rows a warp (a row is a short chain of
// dependent loads, bounds then entries then P, so a warp keeps several in flight, the next rows'
// bounds loaded ahead). Lane l of a row holds entry l; in step q the row's entry q is broadcast and
// lane p <= q adds the pair (p, q), so each pair is taken once; the lanes' pairs are summed by
// shuffles (TwoSum) at the end.
template <int SEG, int LO>
__global__ void __launch_bounds__(256) k_final_csr_pairs(const int64_t* __restrict__ row_ptr,
                                                         const int32_t* __restrict__ col,
                                                         const float* __restrict__ val, int64_t n, int d,
                                                         const float2* __restrict__ P, float* __restrict__ theta) {
    constexpr int RPW = 32 / SEG;
    const int lane = threadIdx.x & 31, seg = lane / SEG, sl = lane % SEG;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t rn = warp * RPW + seg;
    int64_t np0 = rn < n ? row_ptr[rn] : 0, np1 = rn < n ? row_ptr[rn + 1] : 0;
    for (int64_t r0 = warp * RPW; r0 < n; r0 += nwarps * RPW) {
        const int64_t r = r0 + seg;
        const int64_t p0 = np0, p1 = np1;
        const int len = (int)(p1 - p0);
        const bool mine = r < n && len > LO && len <= SEG;
        int c = -1;
        float a = 0.f;
        if (mine && sl < len) {
            c = col[p0 + sl];
            a = val[p0 + sl];
        }
        rn = r + nwarps * RPW;
        np0 = rn < n ? row_ptr[rn] : 0;
        np1 = rn < n ? row_ptr[rn + 1] : 0;
        if ((unsigned)c >= (unsigned)d) { c = -1; a = 0.f; }
        const int len_w = mine ? len : 0;
        int steps = len_w;                                            // the longest row of the warp
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) steps = max(steps, __shfl_xor_sync(0xffffffffu, steps, o));
        float sh = 0.f, sl2 = 0.f;
        const int64_t prow = c >= 0 ? (int64_t)c * d : 0;
        for (int q = 0; q < steps; ++q) {
            const int cq = __shfl_sync(0xffffffffu, c, seg * SEG + q);
            const float aq = __shfl_sync(0xffffffffu, a, seg * SEG + q);
            if (q < len_w && sl <= q && c >= 0 && cq >= 0) {
                float th, tl;
                df_term(a, aq, sl == q ? 1.f : 2.f, P[prow + cq], th, tl);
                df_add(sh, sl2, th, tl);
            }
        }
#pragma unroll
        for (int o = SEG / 2; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, sh, o), ol = __shfl_xor_sync(0xffffffffu, sl2, o);
            df_add(sh, sl2, oh, ol);
        }
        if (mine && sl == 0) theta[r] = __fadd_rn(sh, sl2);
    }
}

// Rows of more than 16 entries: a warp scans the bounds of 32 rows at once and takes each such row
// in turn with the whole warp: the second form (one entry per lane, the pair loop above) up to 32
// entries, the first form (csr_row_norm) above.
template <bool VEC>
__global__ void __launch_bounds__(256) k_final_csr_long(const int64_t* __restrict__ row_ptr,
                                                        const int32_t* __restrict__ col,
                                                        const float* __restrict__ val, int64_t n, int d,
                                                        const float* __restrict__ M, int k,
                                                        const float2* __restrict__ P, float* __restrict__ theta) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r0 = warp * 32; r0 < n; r0 += nwarps * 32) {
        const int64_t rl = r0 + lane;
        const int64_t lenl = rl < n ? row_ptr[rl + 1] - row_ptr[rl] : 0;
        unsigned todo = __ballot_sync(0xffffffffu, lenl > 16);
        while (todo) {
            const int b = __ffs(todo) - 1;
            todo &= todo - 1;
            const int64_t i = r0 + b;
            const int64_t p0 = row_ptr[i], p1 = row_ptr[i + 1];
            const int len = (int)(p1 - p0);
            if (len > 32) {
                const float total = warp_sum(csr_row_norm<VEC>(p0, p1, col, val, d, M, k, lane));
                if (lane == 0) theta[i] = total;
                continue;
            }
            int c = -1;
            float a = 0.f;
            if (lane < len) {
                c = col[p0 + lane];
                a = val[p0 + lane];
                if ((unsigned)c >= (unsigned)d) { c = -1; a = 0.f; }
            }
            float sh = 0.f, sl2 = 0.f;
            const int64_t prow = c >= 0 ? (int64_t)c * d : 0;
            for (int q = 0; q < len; ++q) {
                const int cq = __shfl_sync(0xffffffffu, c, q);
                const float aq = __shfl_sync(0xffffffffu, a, q);
                if (lane <= q && c >= 0 && cq >= 0) {
                    float th, tl;
                    df_term(a, aq, lane == q ? 1.f : 2.f, P[prow + cq], th, tl);
                    df_add(sh, sl2, th, tl);
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float oh = __shfl_xor_sync(0xffffffffu, sh, o), ol = __shfl_xor_sync(0xffffffffu, sl2, o);
                df_add(sh, sl2, oh, ol);
            }
            if (lane == 0) theta[i] = __fadd_rn(sh, sl2);
        }
    }
}

// Pdf (d x d pairs) = P split into FP32 hi + lo.
__global__ void k_split_pairs(const double* __restrict__ P, int64_t count, float2* __restrict__ Pdf) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
        const double x = P[e];
        const float h = (float)x;
        Pdf[e] = make_float2(h, (float)(x - (double)h));
    }
}

// MT (k x d) = Mfull^T (Mfull d x k, both row-major).
__global__ void k_transpose_mfull(const float* __restrict__ M, int d, int k, float* __restrict__ MT) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)d * k;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int q = (int)(e / d), c = (int)(e % d);
        MT[e] = M[(int64_t)c * k + q];
    }
}

}  // namespace

cudaError_t launch_final_dense_fp32(const float* A, int64_t lda, int64_t n, int64_t d,
                                    const float* Mfull, int64_t k, float* theta, cudaStream_t st) {
    const bool vec = (reinterpret_cast<uintptr_t>(A) % 16 == 0) && (reinterpret_cast<uintptr_t>(Mfull) % 16 == 0) &&
                     (lda % 4 == 0) && (d % 4 == 0) && (k % 4 == 0);
    const int64_t grid = (n + FD_BM - 1) / FD_BM;
    if (grid > 0x7fffffff) return cudaErrorInvalidValue;
    if (vec)
        k_final_dense_fp32<true><<<(unsigned)grid, 256, 0, st>>>(A, lda, n, (int)d, Mfull, (int)k, theta);
    else
        k_final_dense_fp32<false><<<(unsigned)grid, 256, 0, st>>>(A, lda, n, (int)d, Mfull, (int)k, theta);
    return cudaGetLastError();
}

size_t csr_gram_scratch_bytes(int64_t d, int64_t k) {
    return sizeof(double) * (size_t)(d * d + gram_partial_doubles(k, d)) + sizeof(float) * (size_t)(k * d) +
           sizeof(float2) * (size_t)(d * d) + 1024;
}

bool csr_gram_pays(int64_t n, int64_t d, int64_t nnz, int64_t k) {
    return d <= 1024 && n > 0 && nnz * 8 < n * k;      // short rows on average: nnz_i < k / 8
}

cudaError_t launch_final_csr_gram(const int64_t* row_ptr, const int32_t* col, const float* val, int64_t n, int64_t d,
                                  const float* Mfull, int64_t k, void* scratch, float* theta, cudaStream_t st) {
    double* P = reinterpret_cast<double*>(scratch);
    double* Gp = P + d * d;
    float* MT = reinterpret_cast<float*>(Gp + gram_partial_doubles(k, d));
    float2* Pdf = reinterpret_cast<float2*>(reinterpret_cast<uintptr_t>(MT + k * d + 3) & ~uintptr_t(7));
    int tg = (int)((d * k + 255) / 256);
    if (tg > 152 * 8) tg = 152 * 8;
    k_transpose_mfull<<<tg, 256, 0, st>>>(Mfull, (int)d, (int)k, MT);
    cudaError_t e = launch_gram_fp64(MT, d, k, d, Gp, P, st);           // P = Mfull Mfull^T (FP64-grade)
    if (e != cudaSuccess) return e;
    k_split_pairs<<<152 * 4, 256, 0, st>>>(P, d * d, Pdf);
    const bool vec = (reinterpret_cast<uintptr_t>(Mfull) % 16 == 0) && (k % 4 == 0);
    int64_t grid = (n * 8 + 255) / 256;                 // four rows of up to 8 entries a warp
    if (grid > 152 * 64) grid = 152 * 64;
    if (grid < 1) grid = 1;
    k_final_csr_pairs<8, -1><<<(unsigned)grid, 256, 0, st>>>(row_ptr, col, val, n, (int)d, Pdf, theta);  // empty rows too
    int64_t grid16 = (n * 16 + 255) / 256;              // two rows of 9 to 16 entries a warp
    if (grid16 > 152 * 64) grid16 = 152 * 64;
    if (grid16 < 1) grid16 = 1;
    k_final_csr_pairs<16, 8><<<(unsigned)grid16, 256, 0, st>>>(row_ptr, col, val, n, (int)d, Pdf, theta);
    int64_t grid_l = (n + 255) / 256;                   // 32 rows scanned a warp
    if (grid_l > 152 * 16) grid_l = 152 * 16;
    if (grid_l < 1) grid_l = 1;
    if (vec)
        k_final_csr_long<true><<<(unsigned)grid_l, 256, 0, st>>>(row_ptr, col, val, n, (int)d, Mfull, (int)k, Pdf,
                                                                theta);
    else
        k_final_csr_long<false><<<(unsigned)grid_l, 256, 0, st>>>(row_ptr, col, val, n, (int)d, Mfull, (int)k, Pdf,
                                                                 theta);
    return cudaGetLastError();
}

cudaError_t launch_final_csr_fp32(const int64_t* row_ptr, const int32_t* col, const float* val,
                                  int64_t n, int64_t d, const float* Mfull, int64_t k,
                                  float* theta, cudaStream_t st) {
    const bool vec = (reinterpret_cast<uintptr_t>(Mfull) % 16 == 0) && (k % 4 == 0);
    int64_t grid = (n * 32 + 255) / 256;
    if (grid > 152 * 64) grid = 152 * 64;
    if (grid < 1) grid = 1;
    if (vec)
        k_final_csr_fp32<true><<<(unsigned)grid, 256, 0, st>>>(row_ptr, col, val, n, (int)d, Mfull, (int)k, theta);
    else
        k_final_csr_fp32<false><<<(unsigned)grid, 256, 0, st>>>(row_ptr, col, val, n, (int)d, Mfull, (int)k, theta);
    return cudaGetLastError();
}

}  // namespace lev
