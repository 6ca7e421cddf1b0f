// Gradient of g(A) = sum_i w_i theta~_i(A) with respect to dense A (the
// reverse-mode adjoint of Alg. 10 with S, G, Omega, the pivots and the rank
// fixed). With A_K the selected columns, M = R_11^{-1} Omega, Y = A_K M,
// Z = 2 W Y and A~_K = G S A_K = Q_1 R_11:
//   C = A_K^T Z;  Rbar = -R_11^{-T} C M^T;  K = copyltu(R_11 Rbar^T)
//   (copyltu(X) = tril(X) + tril(X,-1)^T);  Xbar = Q_1 K R_11^{-T} = A~_K N with
//   N = R_11^{-1} K R_11^{-T};  T = G^T Xbar;
//   dg/dA_i = Z_i M^T + sigma_i T[h(i), :] on the columns of K, 0 elsewhere.
// Working over all d columns with Mfull (zero rows off K) and Xbar scattered
// into an m x d matrix (zero columns off K) makes both big passes plain dense
// products, and the columns off K come out 0 by construction.
//
// Kernels: pass 1 (Y recomputed per tile, C partials per row chunk), fixed-order
// reduction of C in FP64, the small FP64 steps (C M^T, two blocked triangular
// solves with R_11 and R_11^T, copyltu, Xbar), T = G^T Xbar (FP32), pass 2
// (Y recomputed, Z M^T plus the CountSketch adjoint gathered by hash, no atomics).
#include <cuda_bf16.h>

#include <algorithm>

#include "lev_common.cuh"
#include "lev_kernels.cuh"

namespace lev {

namespace {

constexpr int P1_RT = 32, P1_DB = 64, P1_KB = 64;

// C partial for (row chunk, d block, k block): C[a][q] = sum_i A[i][a] * 2 w_i (A_i Mfull)[q].
__global__ void __launch_bounds__(256) k_bwd_pass1(const float* __restrict__ A, int64_t lda, int64_t n, int d,
                                                   const float* __restrict__ Mf, int k, const float* __restrict__ w,
                                                   int rows_per_chunk, float* __restrict__ Cp) {
    extern __shared__ float sm[];
    const int dpad = (d + 3) & ~3;
    float* As = sm;                                 // P1_RT x dpad
    float* Ms = As + P1_RT * dpad;                  // d x P1_KB  (Mfull[:, kb])
    float* Zs = Ms + (size_t)d * P1_KB;             // P1_RT x P1_KB
    const int t = threadIdx.x;
    const int chunk = blockIdx.x, dbk = blockIdx.y, kbk = blockIdx.z;
    const int q0 = kbk * P1_KB, a0 = dbk * P1_DB;
    const int64_t r_begin = (int64_t)chunk * rows_per_chunk;
    const int64_t r_end = min(n, r_begin + rows_per_chunk);
    for (int e = t; e < d * P1_KB; e += 256) {
        const int j = e / P1_KB, q = e % P1_KB;
        Ms[e] = (q0 + q < k) ? Mf[(int64_t)j * k + q0 + q] : 0.f;
    }
    // thread tiles: Y: row ry = t / 8, columns qy .. qy+7; C: 4 x 4 at (ca, cq)
    const int ry = t >> 3, qy = (t & 7) * 8;
    const int ca = (t >> 4) * 4, cq = (t & 15) * 4;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int64_t r0 = r_begin; r0 < r_end; r0 += P1_RT) {
        __syncthreads();
        for (int e = t; e < P1_RT * dpad; e += 256) {
            const int r = e / dpad, j = e % dpad;
            const int64_t row = r0 + r;
            As[e] = (row < r_end && j < d) ? A[row * lda + j] : 0.f;
        }
        __syncthreads();
        float y[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) y[u] = 0.f;
        for (int j = 0; j < d; ++j) {
            const float a = As[ry * dpad + j];
#pragma unroll
            for (int u = 0; u < 8; ++u) y[u] = fmaf(a, Ms[j * P1_KB + qy + u], y[u]);
        }
        const int64_t row = r0 + ry;
        const float tw = (row < r_end) ? 2.f * w[row] : 0.f;
#pragma unroll
        for (int u = 0; u < 8; ++u) Zs[ry * P1_KB + qy + u] = tw * y[u];
        __syncthreads();
        for (int r = 0; r < P1_RT; ++r) {
            float av[4], zv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = (a0 + ca + i < d) ? As[r * dpad + a0 + ca + i] : 0.f;
#pragma unroll
            for (int j = 0; j < 4; ++j) zv[j] = Zs[r * P1_KB + cq + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], zv[j], acc[i][j]);
        }
    }
    float* out = Cp + (int64_t)chunk * d * k;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int a = a0 + ca + i, q = q0 + cq + j;
            if (a < d && q < k) out[(int64_t)a * k + q] = acc[i][j];
        }
}

__global__ void k_bwd_reduce_c(const float* __restrict__ Cp, int chunks, int d, int k, double* __restrict__ C) {
    const int64_t total = (int64_t)d * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int z = 0; z < chunks; ++z) s += (double)Cp[(int64_t)z * total + e];
        C[e] = s;
    }
}

// CMt[p][q] = sum_l C[P_p][l] Mfull[P_q][l] for p, q < r (d x d storage, ld = d).
__global__ void k_bwd_cmt(const double* __restrict__ C, const float* __restrict__ Mf, const int32_t* __restrict__ perm,
                          const int64_t* __restrict__ d_rank, int d, int k, double* __restrict__ CMt) {
    const int r = (int)min(*d_rank, (int64_t)d);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)d * d;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int p = (int)(e / d), q = (int)(e % d);
        double s = 0.0;
        if (p < r && q < r) {
            const double* cp = C + (int64_t)perm[p] * k;
            const float* mq = Mf + (int64_t)perm[q] * k;
            for (int l = 0; l < k; ++l) s = fma(cp[l], (double)mq[l], s);
        }
        CMt[e] = s;
    }
}

// Blocked triangular solve with R_11 (upper, row-major, ld = d), one warp per
// right-hand side column b, in place on X (element (p, b) at X[p*sp + b*sb]).
// upper: R_11 x = x (bottom-up). lower_t: R_11^T x = x (top-down). scale: applied to the rhs.
__global__ void k_trsm_r11(const double* __restrict__ R, const int64_t* __restrict__ d_rank, int d, double* X,
                           int64_t sp, int64_t sb, int lower_t, double scale) {
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int r = (int)min(*d_rank, (int64_t)d);
    if (b >= r) return;
    double* xb = X + (int64_t)b * sb;
    for (int p = lane; p < r; p += 32) xb[(int64_t)p * sp] *= scale;
    __syncwarp();
    const int nblk = (r + 31) / 32;
    for (int bi = 0; bi < nblk; ++bi) {
        const int blk = lower_t ? bi : nblk - 1 - bi;
        const int i0 = blk * 32;
        const int i = i0 + lane;
        const bool valid = i < r;
        double rhs = valid ? xb[(int64_t)i * sp] : 0.0;
        double acc = 0.0;
        if (valid) {
            if (lower_t) {
                for (int tt = 0; tt < i0; ++tt) acc = fma(R[(int64_t)tt * d + i], xb[(int64_t)tt * sp], acc);
            } else {
                for (int tt = i0 + 32; tt < r; ++tt) acc = fma(R[(int64_t)i * d + tt], xb[(int64_t)tt * sp], acc);
            }
        }
        rhs -= acc;
        double rb[32];
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) {
            const int c = i0 + jj;
            rb[jj] = (valid && c < r) ? (lower_t ? R[(int64_t)c * d + i] : R[(int64_t)i * d + c]) : 0.0;
        }
        const double inv = valid ? 1.0 / R[(int64_t)i * d + i] : 0.0;
        double x = 0.0;
        if (lower_t) {
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
                if (lane == jj) x = rhs * inv;
                const double xj = __shfl_sync(0xffffffffu, x, jj);
                if (lane > jj) rhs = fma(-rb[jj], xj, rhs);
            }
        } else {
#pragma unroll
            for (int jj = 31; jj >= 0; --jj) {
                if (lane == jj) x = rhs * inv;
                const double xj = __shfl_sync(0xffffffffu, x, jj);
                if (lane < jj) rhs = fma(-rb[jj], xj, rhs);
            }
        }
        if (valid) xb[(int64_t)i * sp] = x;
        __syncwarp();
    }
}

// K = copyltu(R_11 Rbar^T): K[a][b] = (R_11 Rbar^T)[max(a,b)][min(a,b)] (symmetric).
__global__ void k_copyltu(const double* __restrict__ R, const double* __restrict__ Rbar,
                          const int64_t* __restrict__ d_rank, int d, double* __restrict__ K) {
    const int r = (int)min(*d_rank, (int64_t)d);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)d * d;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(e / d), b = (int)(e % d);
        double s = 0.0;
        if (a < r && b < r) {
            const int hi = max(a, b), lo = min(a, b);
            for (int t = hi; t < r; ++t) s = fma(R[(int64_t)hi * d + t], Rbar[(int64_t)lo * d + t], s);
        }
        K[e] = s;
    }
}

// Xbar_full (m x d FP32): column P_p holds (A~_K N)[:, p]; other columns 0.
__global__ void k_xbar(const float* __restrict__ At, const double* __restrict__ N, const int32_t* __restrict__ perm,
                       const int64_t* __restrict__ d_rank, int m, int d, float* __restrict__ Xf) {
    const int r = (int)min(*d_rank, (int64_t)d);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)m * d;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / d), p = (int)(e % d);
        if (p >= r) continue;
        double s = 0.0;
        const float* arow = At + (int64_t)j * d;
        for (int q = 0; q < r; ++q) s = fma((double)arow[perm[q]], N[(int64_t)q * d + p], s);
        Xf[(int64_t)j * d + perm[p]] = (float)s;
    }
}

// T (s x d) = G^T Xbar_full, G (m x s, leading dimension ldg) as FP32 or BF16 hi + lo.
template <bool SPLIT>
__global__ void __launch_bounds__(256) k_gt_x(const float* __restrict__ G32, const __nv_bfloat16* __restrict__ Ghi,
                                              const __nv_bfloat16* __restrict__ Glo, int64_t ldg, int m, int64_t s,
                                              const float* __restrict__ Xf, int d, float* __restrict__ T) {
    __shared__ float Gs[16][64];
    __shared__ float Xs[16][64];
    const int t = threadIdx.x;
    const int64_t b0 = (int64_t)blockIdx.x * 64;
    const int c0 = blockIdx.y * 64;
    const int tb = (t >> 4) * 4, tc = (t & 15) * 4;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int j0 = 0; j0 < m; j0 += 16) {
        __syncthreads();
        for (int e = t; e < 16 * 64; e += 256) {
            const int jj = e / 64, u = e % 64;
            const int j = j0 + jj;
            const int64_t b = b0 + u;
            float g = 0.f;
            if (j < m && b < s) {
                if (SPLIT)
                    g = __bfloat162float(Ghi[(int64_t)j * ldg + b]) +
                        (Glo ? __bfloat162float(Glo[(int64_t)j * ldg + b]) : 0.f);
                else
                    g = G32[(int64_t)j * ldg + b];
            }
            Gs[jj][u] = g;
            Xs[jj][u] = (j < m && c0 + u < d) ? Xf[(int64_t)j * d + c0 + u] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
            float gv[4], xv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) gv[i] = Gs[jj][tb + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) xv[j] = Xs[jj][tc + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(gv[i], xv[j], acc[i][j]);
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t b = b0 + tb + i;
            const int c = c0 + tc + j;
            if (b < s && c < d) T[b * d + c] = acc[i][j];
        }
}

// Pass 2: gradA[i][c] = sum_q Z_iq Mfull[c][q] + sigma_i T[h(i)][c], Z_i = 2 w_i A_i Mfull.
// 32 rows per CTA. Phase A: Z (32 x k) from A (32 x d) and 64-column chunks of
// Mfull staged in shared memory; phase B: 64 x 64 chunks of Mfull^T staged
// (padded rows), 8 output columns per thread.
constexpr int P2_RT = 32, P2_QC = 64, P2_CC = 64;
__global__ void __launch_bounds__(256) k_bwd_pass2(const float* __restrict__ A, int64_t lda, int64_t n, int d,
                                                   const float* __restrict__ Mf, int k, const float* __restrict__ w,
                                                   const float* __restrict__ T, uint64_t key, uint32_t s,
                                                   int identity, float* __restrict__ gA) {
    extern __shared__ float sm[];
    const int dpad = (d + 3) & ~3, kz = ((k + P2_QC - 1) / P2_QC) * P2_QC + 4;
    float* As = sm;                       // P2_RT x dpad
    float* Zs = As + P2_RT * dpad;        // P2_RT x kz
    float* Ms = Zs + P2_RT * kz;          // phase A: d x P2_QC; phase B: P2_QC x (P2_CC + 4)
    const int t = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.x * P2_RT;
    for (int e = t; e < P2_RT * dpad; e += 256) {
        const int r = e / dpad, j = e % dpad;
        const int64_t row = r0 + r;
        As[e] = (row < n && j < d) ? A[row * lda + j] : 0.f;
    }
    const int ry = t >> 3, g8 = (t & 7) * 8;
    const int64_t row = r0 + ry;
    const float tw = (row < n) ? 2.f * w[row] : 0.f;
    for (int q0 = 0; q0 < k; q0 += P2_QC) {
        __syncthreads();
        for (int e = t; e < d * P2_QC; e += 256) {
            const int j = e / P2_QC, q = e % P2_QC;
            Ms[e] = (q0 + q < k) ? Mf[(int64_t)j * k + q0 + q] : 0.f;
        }
        __syncthreads();
        float y[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) y[u] = 0.f;
        for (int j = 0; j < d; ++j) {
            const float a = As[ry * dpad + j];
            const float4 m0 = *reinterpret_cast<const float4*>(&Ms[j * P2_QC + g8]);
            const float4 m1 = *reinterpret_cast<const float4*>(&Ms[j * P2_QC + g8 + 4]);
            y[0] = fmaf(a, m0.x, y[0]); y[1] = fmaf(a, m0.y, y[1]); y[2] = fmaf(a, m0.z, y[2]); y[3] = fmaf(a, m0.w, y[3]);
            y[4] = fmaf(a, m1.x, y[4]); y[5] = fmaf(a, m1.y, y[5]); y[6] = fmaf(a, m1.z, y[6]); y[7] = fmaf(a, m1.w, y[7]);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) Zs[ry * kz + q0 + g8 + u] = tw * y[u];
    }
    const uint64_t x = splitmix64(key, (uint64_t)row);
    const int64_t bucket = identity ? row : (int64_t)bucket_of(x, s);     // S = I: row i is bucket i
    const float sg = identity ? 1.f : sign_of(x);
    constexpr int MT = P2_CC + 4;
    for (int c0 = 0; c0 < d; c0 += P2_CC) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = 0.f;
        for (int q0 = 0; q0 < k; q0 += P2_QC) {
            __syncthreads();
            for (int e = t; e < P2_QC * P2_CC; e += 256) {
                const int c = e / P2_QC, q = e % P2_QC;             // coalesced over q of Mfull row c
                Ms[q * MT + c] = (c0 + c < d && q0 + q < k) ? Mf[(int64_t)(c0 + c) * k + q0 + q] : 0.f;
            }
            __syncthreads();
#pragma unroll 4
            for (int q = 0; q < P2_QC; ++q) {
                const float z = Zs[ry * kz + q0 + q];
                const float4 m0 = *reinterpret_cast<const float4*>(&Ms[q * MT + g8]);
                const float4 m1 = *reinterpret_cast<const float4*>(&Ms[q * MT + g8 + 4]);
                v[0] = fmaf(z, m0.x, v[0]); v[1] = fmaf(z, m0.y, v[1]); v[2] = fmaf(z, m0.z, v[2]); v[3] = fmaf(z, m0.w, v[3]);
                v[4] = fmaf(z, m1.x, v[4]); v[5] = fmaf(z, m1.y, v[5]); v[6] = fmaf(z, m1.z, v[6]); v[7] = fmaf(z, m1.w, v[7]);
            }
        }
        if (row < n) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int c = c0 + g8 + u;
                if (c < d) gA[row * d + c] = v[u] + sg * T[bucket * d + c];
            }
        }
    }
}

int grid_cap(int64_t work, int block, int cap) {
    int64_t g = (work + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

}  // namespace

size_t backward_scratch_bytes(int64_t n, int64_t d, int64_t k, int64_t s, int64_t m, int chunks) {
    size_t b = 0;
    b += sizeof(float) * (size_t)chunks * d * k;     // C partials
    b += sizeof(double) * (size_t)d * k;            // C
    b += 4 * sizeof(double) * (size_t)d * d;        // CMt/Rbar, K/V/N, spare
    b += sizeof(float) * (size_t)m * d;             // Xbar_full
    b += sizeof(float) * (size_t)s * d;             // T (unused in the identity-sketch mode)
    return b + 8 * 256;
}

int backward_chunks(int64_t n, int64_t d, int64_t k) {
    const int64_t dbk = (d + P1_DB - 1) / P1_DB, kbk = (k + P1_KB - 1) / P1_KB;
    int64_t c = (2 * 152 + dbk * kbk - 1) / (dbk * kbk);
    const int64_t max_c = (n + P1_RT - 1) / P1_RT;
    if (c > max_c) c = max_c;
    if (c < 1) c = 1;
    return (int)c;
}

cudaError_t launch_backward_dense(const float* A, int64_t lda, int64_t n, int64_t d, int64_t s, int64_t m, int64_t k,
                                  uint64_t seed, const float* Atilde, const int32_t* perm, const int64_t* d_rank,
                                  const double* R, const float* Mfull, const float* w, const float* G32,
                                  const __nv_bfloat16* Ghi, const __nv_bfloat16* Glo, int64_t ldg, bool identity,
                                  void* scratch, int chunks, float* gradA, cudaStream_t st) {
    char* p = static_cast<char*>(scratch);
    auto take = [&](size_t bytes) { char* r = p; p += (bytes + 255) / 256 * 256; return r; };
    float* Cp = reinterpret_cast<float*>(take(sizeof(float) * (size_t)chunks * d * k));
    double* C = reinterpret_cast<double*>(take(sizeof(double) * (size_t)d * k));
    double* B1 = reinterpret_cast<double*>(take(sizeof(double) * (size_t)d * d));
    double* B2 = reinterpret_cast<double*>(take(sizeof(double) * (size_t)d * d));
    float* Xf = reinterpret_cast<float*>(take(sizeof(float) * (size_t)m * d));
    float* T = reinterpret_cast<float*>(take(sizeof(float) * (size_t)s * d));
    cudaError_t e;
    // pass 1
    const int rows_per_chunk = (int)(((n + chunks - 1) / chunks + P1_RT - 1) / P1_RT * P1_RT);
    const int dpad = (int)((d + 3) & ~3);
    const size_t sm1 = sizeof(float) * ((size_t)P1_RT * dpad + (size_t)d * P1_KB + (size_t)P1_RT * P1_KB);
    if (sm1 > 48 * 1024)
        if ((e = cudaFuncSetAttribute(k_bwd_pass1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1)) != cudaSuccess)
            return e;
    dim3 g1((unsigned)chunks, (unsigned)((d + P1_DB - 1) / P1_DB), (unsigned)((k + P1_KB - 1) / P1_KB));
    k_bwd_pass1<<<g1, 256, sm1, st>>>(A, lda, n, (int)d, Mfull, (int)k, w, rows_per_chunk, Cp);
    k_bwd_reduce_c<<<grid_cap(d * k, 256, 1024), 256, 0, st>>>(Cp, chunks, (int)d, (int)k, C);
    // small FP64 steps
    k_bwd_cmt<<<grid_cap(d * d, 256, 1024), 256, 0, st>>>(C, Mfull, perm, d_rank, (int)d, (int)k, B1);
    // Rbar = -R^{-T} (C M^T): columns of CMt, in place in B1
    k_trsm_r11<<<(unsigned)d, 32, 0, st>>>(R, d_rank, (int)d, B1, d, 1, 1, -1.0);
    k_copyltu<<<grid_cap(d * d, 256, 1024), 256, 0, st>>>(R, B1, d_rank, (int)d, B2);
    // V = R^{-1} K (columns, in place), then N^T = R^{-1} V^T through the transposed view -> B2 holds N
    k_trsm_r11<<<(unsigned)d, 32, 0, st>>>(R, d_rank, (int)d, B2, d, 1, 0, 1.0);
    k_trsm_r11<<<(unsigned)d, 32, 0, st>>>(R, d_rank, (int)d, B2, 1, d, 0, 1.0);
    if ((e = cudaMemsetAsync(Xf, 0, sizeof(float) * (size_t)m * d, st)) != cudaSuccess) return e;
    k_xbar<<<grid_cap(m * d, 256, 152 * 8), 256, 0, st>>>(Atilde, B2, perm, d_rank, (int)m, (int)d, Xf);
    // T = G^T Xbar_full (G = I in the identity-sketch mode: T = Xbar_full)
    dim3 gt((unsigned)((s + 63) / 64), (unsigned)((d + 63) / 64));
    if (identity)
        T = Xf;
    else if (Ghi)
        k_gt_x<true><<<gt, 256, 0, st>>>(nullptr, Ghi, Glo, ldg, (int)m, s, Xf, (int)d, T);
    else
        k_gt_x<false><<<gt, 256, 0, st>>>(G32, nullptr, nullptr, ldg, (int)m, s, Xf, (int)d, T);
    // pass 2
    const int kz = (int)((k + P2_QC - 1) / P2_QC * P2_QC + 4);
    const size_t ms2 = std::max((size_t)d * P2_QC, (size_t)P2_QC * (P2_CC + 4));
    const size_t sm2 = sizeof(float) * ((size_t)P2_RT * dpad + (size_t)P2_RT * kz + ms2);
    if (sm2 > 48 * 1024)
        if ((e = cudaFuncSetAttribute(k_bwd_pass2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2)) != cudaSuccess)
            return e;
    k_bwd_pass2<<<(unsigned)((n + P2_RT - 1) / P2_RT), 256, sm2, st>>>(A, lda, n, (int)d, Mfull, (int)k, w, T,
                                                                       stream_key(seed, kStreamHash), (uint32_t)s,
                                                                       identity ? 1 : 0, gradA);
    return cudaGetLastError();
}

}  // namespace lev
