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

// CSR, warp per row, lane owns columns q0 + lane*4 + {0..3} and q0 + 128 + lane*4 + {0..3}.
template <bool VEC>
__global__ void __launch_bounds__(256) k_final_csr_fp32(
        const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
        const float* __restrict__ val, int64_t n, int d, const float* __restrict__ M, int k,
        float* __restrict__ theta) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < n; i += nwarps) {
        const int64_t p0 = row_ptr[i], p1 = row_ptr[i + 1];
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
        total = warp_sum(total);
        if (lane == 0) theta[i] = total;
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
