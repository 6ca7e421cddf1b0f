// Gradient of g(A) = sum_i w_i theta~_i(A) with respect to dense A (the
// reverse-mode adjoint of Alg. 10 with S, G, Omega, the pivots and the rank
// fixed). With A_K the selected columns, M = R_11^{-1} Omega, Y = A_K M,
// Z = 2 W Y and A~_K = G S A_K = Q_1 R_11:
//   C = A_K^T Z;  Rbar = -R_11^{-T} C M^T;  K = copyltu(R_11 Rbar^T)
//   (copyltu(X) = tril(X) + tril(X,-1)^T);  Xbar = Q_1 K R_11^{-T} = A~_K N with
//   N = R_11^{-1} K R_11^{-T};  T = G^T Xbar;
//   dg/dA_i = Z_i M^T + sigma_i T[h(i), :] on the columns of K, 0 elsewhere.
// Working over all d columns with Mfull (zero rows off K) and Xbar scattered
// into an m x d matrix (zero columns off K) makes both big passes dense
// products, and the columns off K come out 0 by construction. Both passes are
// reassociated around the two d x d matrices H = A^T W A and P = Mfull Mfull^T:
//   C = A^T Z = 2 (A^T W A) Mfull = 2 H Mfull,
//   Z M^T = 2 W A Mfull Mfull^T = 2 W A P,
// so the two passes over A cost 2 n d^2 flops each instead of 4 n d k.
//
// Kernels: pass 1 (H partials per row chunk, 8 x 8 register blocks, the upper
// 64 x 64 tiles only), fixed-order reduction of H, C = 2 H Mfull and P in FP64,
// the small FP64 steps (C M^T, two blocked triangular solves with R_11 and
// R_11^T, copyltu, Xbar), T = G^T Xbar (FP32), pass 2 (2 W A P plus the
// CountSketch adjoint gathered by hash, 8 x 4 register blocks, no atomics).
#include <cuda_bf16.h>

#include <algorithm>

#include "lev_common.cuh"
#include "lev_kernels.cuh"

namespace lev {

namespace {

constexpr int HT = 64;          // H tile
constexpr int H_RB = 32;        // rows staged per step of pass 1

__host__ __device__ inline int h_tiles(int d) {
    const int nt = (d + HT - 1) / HT;
    return nt * (nt + 1) / 2;
}

__device__ inline void h_tile_coords(int t, int nt, int& bi, int& bj) {
    bi = 0;
    while (t >= nt - bi) { t -= nt - bi; ++bi; }
    bj = bi + t;
}

// Pass 1: partial H = sum_i w_i A_i^T A_i over one row chunk, for the upper 64 x 64 tile
// (bi, bj) of H. Four groups of 64 threads take every fourth staged row; thread (ti, tj) of a
// group owns the 8 x 8 block (bi*64 + 8 ti .. , bj*64 + 8 tj ..). The groups' blocks are summed
// in shared memory and the CTA writes one 64 x 64 FP32 partial.
__global__ void __launch_bounds__(256) k_bwd_wgram(const float* __restrict__ A, int64_t lda, int64_t n, int d,
                                                   int vecA, const float* __restrict__ w, int rows_per_chunk,
                                                   float* __restrict__ Hp) {
    extern __shared__ __align__(16) float sm[];
    float* Ai = sm;                         // H_RB x 64: columns bi*64 ..
    float* Aj = Ai + H_RB * HT;             // H_RB x 64: columns bj*64 ..
    float* ws = Aj + H_RB * HT;             // H_RB
    const int nt = (d + HT - 1) / HT;
    int bi, bj;
    h_tile_coords(blockIdx.y, nt, bi, bj);
    const int t = threadIdx.x, g = t >> 6, tt = t & 63, ti = tt >> 3, tj = tt & 7;
    const int64_t r_begin = (int64_t)blockIdx.x * rows_per_chunk;
    const int64_t r_end = min(n, r_begin + rows_per_chunk);
    float acc[8][8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[u][v] = 0.f;
    for (int64_t r0 = r_begin; r0 < r_end; r0 += H_RB) {
        __syncthreads();
        // 32 rows x 64 columns per side; float4 loads when A is 16-byte aligned and lda % 4 == 0
        for (int e = t; e < H_RB * (HT / 4); e += 256) {
            const int r = e / (HT / 4), c4 = (e % (HT / 4)) * 4;
            const int64_t row = r0 + r;
            float4 vi = make_float4(0.f, 0.f, 0.f, 0.f), vj = vi;
            if (row < r_end) {
                const float* src = A + row * lda;
                const int ci = bi * HT + c4, cj = bj * HT + c4;
                if (vecA && ci + 3 < d) vi = *reinterpret_cast<const float4*>(src + ci);
                else {
                    vi.x = ci < d ? src[ci] : 0.f; vi.y = ci + 1 < d ? src[ci + 1] : 0.f;
                    vi.z = ci + 2 < d ? src[ci + 2] : 0.f; vi.w = ci + 3 < d ? src[ci + 3] : 0.f;
                }
                if (vecA && cj + 3 < d) vj = *reinterpret_cast<const float4*>(src + cj);
                else {
                    vj.x = cj < d ? src[cj] : 0.f; vj.y = cj + 1 < d ? src[cj + 1] : 0.f;
                    vj.z = cj + 2 < d ? src[cj + 2] : 0.f; vj.w = cj + 3 < d ? src[cj + 3] : 0.f;
                }
            }
            *reinterpret_cast<float4*>(Ai + r * HT + c4) = vi;
            *reinterpret_cast<float4*>(Aj + r * HT + c4) = vj;
        }
        for (int r = t; r < H_RB; r += 256) ws[r] = (r0 + r < r_end) ? w[r0 + r] : 0.f;
        __syncthreads();
#pragma unroll 2
        for (int r = g; r < H_RB; r += 4) {
            const float wr = ws[r];
            const float4 a0 = *reinterpret_cast<const float4*>(Ai + r * HT + ti * 8);
            const float4 a1 = *reinterpret_cast<const float4*>(Ai + r * HT + ti * 8 + 4);
            const float4 b0 = *reinterpret_cast<const float4*>(Aj + r * HT + tj * 8);
            const float4 b1 = *reinterpret_cast<const float4*>(Aj + r * HT + tj * 8 + 4);
            const float av[8] = {wr * a0.x, wr * a0.y, wr * a0.z, wr * a0.w, wr * a1.x, wr * a1.y, wr * a1.z, wr * a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int v = 0; v < 8; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
        }
    }
    // the four groups' blocks, summed in a fixed order
    __syncthreads();
    float* red = sm;                        // 4 x 64 x 64 (reuses the staging space)
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) red[(g * HT + ti * 8 + u) * HT + tj * 8 + v] = acc[u][v];
    __syncthreads();
    float* out = Hp + ((int64_t)blockIdx.x * gridDim.y + blockIdx.y) * (HT * HT);
    for (int e = t; e < HT * HT; e += 256)
        out[e] = ((red[e] + red[HT * HT + e]) + red[2 * HT * HT + e]) + red[3 * HT * HT + e];
}

// H (d x d FP64, both triangles) = sum over chunks of the partials, in chunk order.
__global__ void k_bwd_reduce_h(const float* __restrict__ Hp, int chunks, int d, double* __restrict__ H) {
    const int nt = (d + HT - 1) / HT;
    const int T = nt * (nt + 1) / 2;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)T * HT * HT;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int tile = (int)(e / (HT * HT)), x = (int)(e % (HT * HT));
        int bi, bj;
        h_tile_coords(tile, nt, bi, bj);
        const int a = bi * HT + x / HT, b = bj * HT + x % HT;
        // one writer per symmetric pair: in a diagonal tile the (a, b) and (b, a) partials
        // round differently ((w a_a) a_b against (w a_b) a_a), so only a <= b is summed
        if (a >= d || b >= d || a > b) continue;
        double sum = 0.0;
        for (int c = 0; c < chunks; ++c) sum += (double)Hp[((int64_t)c * T + tile) * (HT * HT) + x];
        H[(int64_t)a * d + b] = sum;
        H[(int64_t)b * d + a] = sum;
    }
}

// C (d x k FP64) = 2 H Mfull.
__global__ void k_bwd_hm(const double* __restrict__ H, const float* __restrict__ Mf, int d, int k,
                         double* __restrict__ C) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)d * k;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(e / k), q = (int)(e % k);
        double acc = 0.0;
        for (int b = 0; b < d; ++b) acc = fma(H[(int64_t)a * d + b], (double)Mf[(int64_t)b * k + q], acc);
        C[e] = 2.0 * acc;
    }
}

// P (d x d FP32, row stride ldp = d rounded up to 4) = Mfull Mfull^T, accumulated in FP64.
__global__ void k_bwd_pmat(const float* __restrict__ Mf, int d, int k, int ldp, float* __restrict__ P) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)d * d;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(e / d), c = (int)(e % d);
        double acc = 0.0;
        for (int q = 0; q < k; ++q) acc = fma((double)Mf[(int64_t)a * k + q], (double)Mf[(int64_t)c * k + q], acc);
        P[(int64_t)a * ldp + c] = (float)acc;
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

// T (s x d) = G^T Xbar_full, G = g_scale * (the image: FP32, or the BF16 pair hi + lo when B16, lo
// m ldg entries after hi; the sum is exact in FP32), m x s with leading dimension ldg.
template <bool B16>
__global__ void __launch_bounds__(256) k_gt_x(const float* __restrict__ G32, const __nv_bfloat16* __restrict__ Ghi,
                                              int64_t ldg, int m, int64_t s, float g_scale,
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
                const int64_t o = (int64_t)j * ldg + b;
                g = B16 ? __bfloat162float(Ghi[o]) + __bfloat162float(Ghi[(int64_t)m * ldg + o]) : G32[o];
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
            if (b < s && c < d) T[b * d + c] = acc[i][j] * g_scale;
        }
}

// Pass 2: gradA[i][c] = 2 w_i (A_i P)[c] + sigma_i T[h(i)][c] for a tile of 128 rows x 64
// columns. Thread (tr, tc) owns rows 8 tr .. 8 tr + 7 and columns 4 tc .. 4 tc + 3; A rows and
// P rows are staged 64 columns of A at a time; each step of 4 j's takes eight float4 of A
// and four of P for 128 FMAs.
constexpr int P2_R = 128, P2_C = 64, P2_J = 64, P2_AS = P2_J + 4;
__global__ void __launch_bounds__(256) k_bwd_pass2(const float* __restrict__ A, int64_t lda, int64_t n, int d,
                                                   int vecA, const float* __restrict__ P, int ldp,
                                                   const float* __restrict__ w,
                                                   const float* __restrict__ T, uint64_t key, uint32_t s,
                                                   int identity, float* __restrict__ gA) {
    extern __shared__ __align__(16) float sm[];
    float* As = sm;                          // P2_R x P2_AS
    float* Ps = As + P2_R * P2_AS;           // P2_J x P2_C
    const int t = threadIdx.x, tr = t >> 4, tc = t & 15;
    const int64_t r0 = (int64_t)blockIdx.x * P2_R;
    const int c0 = blockIdx.y * P2_C;
    float acc[8][4];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
    for (int j0 = 0; j0 < d; j0 += P2_J) {
        __syncthreads();
        for (int e = t; e < P2_R * (P2_J / 4); e += 256) {
            const int r = e / (P2_J / 4), j4 = (e % (P2_J / 4)) * 4;
            const int64_t row = r0 + r;
            const int j = j0 + j4;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (row < n) {
                const float* src = A + row * lda;
                if (vecA && j + 3 < d) v = *reinterpret_cast<const float4*>(src + j);
                else {
                    v.x = j < d ? src[j] : 0.f; v.y = j + 1 < d ? src[j + 1] : 0.f;
                    v.z = j + 2 < d ? src[j + 2] : 0.f; v.w = j + 3 < d ? src[j + 3] : 0.f;
                }
            }
            *reinterpret_cast<float4*>(As + r * P2_AS + j4) = v;
        }
        for (int e = t; e < P2_J * (P2_C / 4); e += 256) {
            const int j = e / (P2_C / 4), c4 = (e % (P2_C / 4)) * 4;
            const int jj = j0 + j, c = c0 + c4;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (jj < d) {
                const float* src = P + (int64_t)jj * ldp;          // ldp % 4 == 0, P 256-byte aligned
                if (c + 3 < d) v = *reinterpret_cast<const float4*>(src + c);
                else {
                    v.x = c < d ? src[c] : 0.f; v.y = c + 1 < d ? src[c + 1] : 0.f;
                    v.z = c + 2 < d ? src[c + 2] : 0.f; v.w = 0.f;
                }
            }
            *reinterpret_cast<float4*>(Ps + j * P2_C + c4) = v;
        }
        __syncthreads();
#pragma unroll 2
        for (int j = 0; j < P2_J; j += 4) {
            float4 a[8], p[4];
#pragma unroll
            for (int u = 0; u < 8; ++u) a[u] = *reinterpret_cast<const float4*>(As + (tr * 8 + u) * P2_AS + j);
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) p[jj] = *reinterpret_cast<const float4*>(Ps + (j + jj) * P2_C + tc * 4);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float av[4] = {a[u].x, a[u].y, a[u].z, a[u].w};
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    acc[u][0] = fmaf(av[jj], p[jj].x, acc[u][0]);
                    acc[u][1] = fmaf(av[jj], p[jj].y, acc[u][1]);
                    acc[u][2] = fmaf(av[jj], p[jj].z, acc[u][2]);
                    acc[u][3] = fmaf(av[jj], p[jj].w, acc[u][3]);
                }
            }
        }
    }
    const int c = c0 + tc * 4;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int64_t row = r0 + tr * 8 + u;
        if (row >= n) break;
        const uint64_t x = splitmix64(key, (uint64_t)row);
        const int64_t bucket = identity ? row : (int64_t)bucket_of(x, s);     // S = I: row i is bucket i
        const float sg = identity ? 1.f : sign_of(x);
        const float tw = 2.f * w[row];
        const float* trow = T + bucket * d;
        float* out = gA + row * d;
#pragma unroll
        for (int v = 0; v < 4; ++v)
            if (c + v < d) out[c + v] = fmaf(tw, acc[u][v], sg * trow[c + v]);
    }
}

int grid_cap(int64_t work, int block, int cap) {
    int64_t g = (work + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

}  // namespace

size_t backward_scratch_bytes(int64_t n, int64_t d, int64_t k, int64_t s, int64_t m, int64_t srht_t, int chunks) {
    size_t b = 0;
    b += sizeof(float) * (size_t)chunks * h_tiles((int)d) * HT * HT;   // H partials
    b += sizeof(double) * (size_t)d * d;            // H
    b += sizeof(double) * (size_t)d * k;            // C
    b += sizeof(float) * (size_t)d * ((d + 3) & ~3);   // P (row stride rounded up to 4)
    b += 2 * sizeof(double) * (size_t)d * d;        // CMt/Rbar, K/V/N
    b += sizeof(float) * (size_t)m * d;             // Xbar_full
    b += sizeof(float) * (size_t)s * d;             // T (unused in the identity-sketch mode)
    if (srht_t > 0) {
        b += sizeof(float) * (size_t)srht_t * d;    // G^T Xbar before the SRHT adjoint
        b += 2 * sizeof(int) * (size_t)(s + 1);     // draws per row of s, offsets
        b += 2 * sizeof(uint32_t) * (size_t)srht_t; // draws ordered by row, then by draw
    }
    return b + 14 * 256;
}

int backward_chunks(int64_t n, int64_t d, int64_t /*k*/) {
    const int64_t tiles = h_tiles((int)d);
    int64_t c = (2 * 152 + tiles - 1) / tiles;
    const int64_t max_c = (n + H_RB - 1) / H_RB;
    if (c > max_c) c = max_c;
    if (c < 1) c = 1;
    return (int)c;
}

cudaError_t launch_backward_dense(const float* A, int64_t lda, int64_t n, int64_t d, int64_t s, int64_t m, int64_t k,
                                  uint64_t seed, const float* Atilde, const int32_t* perm, const int64_t* d_rank,
                                  const double* R, const float* Mfull, const float* w, const float* G32,
                                  const __nv_bfloat16* Ghi, int64_t ldg, float g_scale, bool identity,
                                  int64_t srht_t, void* scratch, int chunks, float* gradA, cudaStream_t st) {
    char* p = static_cast<char*>(scratch);
    auto take = [&](size_t bytes) { char* r = p; p += (bytes + 255) / 256 * 256; return r; };
    const int ht = h_tiles((int)d);
    float* Hp = reinterpret_cast<float*>(take(sizeof(float) * (size_t)chunks * ht * HT * HT));
    double* H = reinterpret_cast<double*>(take(sizeof(double) * (size_t)d * d));
    double* C = reinterpret_cast<double*>(take(sizeof(double) * (size_t)d * k));
    const int ldp = (int)((d + 3) & ~3);
    float* P = reinterpret_cast<float*>(take(sizeof(float) * (size_t)d * ldp));
    const int vecA = ((reinterpret_cast<uintptr_t>(A) & 15u) == 0 && (lda & 3) == 0) ? 1 : 0;
    double* B1 = reinterpret_cast<double*>(take(sizeof(double) * (size_t)d * d));
    double* B2 = reinterpret_cast<double*>(take(sizeof(double) * (size_t)d * d));
    float* Xf = reinterpret_cast<float*>(take(sizeof(float) * (size_t)m * d));
    float* T = reinterpret_cast<float*>(take(sizeof(float) * (size_t)s * d));
    float* Tt = nullptr;
    int *cnt = nullptr, *off = nullptr;
    uint32_t *tmp = nullptr, *ord = nullptr;
    if (srht_t > 0) {
        Tt = reinterpret_cast<float*>(take(sizeof(float) * (size_t)srht_t * d));
        cnt = reinterpret_cast<int*>(take(sizeof(int) * (size_t)(s + 1)));
        off = reinterpret_cast<int*>(take(sizeof(int) * (size_t)(s + 1)));
        tmp = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * (size_t)srht_t));
        ord = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * (size_t)srht_t));
    }
    cudaError_t e;
    // pass 1: H = A^T W A, then C = 2 H Mfull and P = Mfull Mfull^T
    const int rows_per_chunk = (int)(((n + chunks - 1) / chunks + H_RB - 1) / H_RB * H_RB);
    const size_t sm1 = sizeof(float) * (size_t)4 * HT * HT;     // staging (2 x 32 x 64 + 32) fits inside
    if ((e = cudaFuncSetAttribute(k_bwd_wgram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1)) != cudaSuccess)
        return e;
    k_bwd_wgram<<<dim3((unsigned)chunks, (unsigned)ht), 256, sm1, st>>>(A, lda, n, (int)d, vecA, w, rows_per_chunk,
                                                                        Hp);
    k_bwd_reduce_h<<<grid_cap((int64_t)ht * HT * HT, 256, 1024), 256, 0, st>>>(Hp, chunks, (int)d, H);
    k_bwd_hm<<<grid_cap(d * k, 128, 1024), 128, 0, st>>>(H, Mfull, (int)d, (int)k, C);
    k_bwd_pmat<<<grid_cap(d * d, 128, 1024), 128, 0, st>>>(Mfull, (int)d, (int)k, ldp, P);
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
    // T = G^T Xbar_full (G = I in the identity-sketch mode: T = Xbar_full); after an SRHT, G is m x t and
    // T = F^T (G^T Xbar_full)
    const int64_t cg = srht_t > 0 ? srht_t : s;     // columns of G
    float* Tg = srht_t > 0 ? Tt : T;
    dim3 gt((unsigned)((cg + 63) / 64), (unsigned)((d + 63) / 64));
    if (identity)
        T = Xf;
    else if (Ghi)
        k_gt_x<true><<<gt, 256, 0, st>>>(nullptr, Ghi, ldg, (int)m, cg, g_scale, Xf, (int)d, Tg);
    else
        k_gt_x<false><<<gt, 256, 0, st>>>(G32, nullptr, ldg, (int)m, cg, g_scale, Xf, (int)d, Tg);
    if (!identity && srht_t > 0 &&
        (e = launch_srht_adjoint(Tt, s, d, srht_t, seed, cnt, off, tmp, ord, T, st)) != cudaSuccess)
        return e;
    // pass 2
    const size_t sm2 = sizeof(float) * ((size_t)P2_R * P2_AS + (size_t)P2_J * P2_C);
    if ((e = cudaFuncSetAttribute(k_bwd_pass2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2)) != cudaSuccess)
        return e;
    dim3 g2((unsigned)((n + P2_R - 1) / P2_R), (unsigned)((d + P2_C - 1) / P2_C));
    k_bwd_pass2<<<g2, 256, sm2, st>>>(A, lda, n, (int)d, vecA, P, ldp, w, T, stream_key(seed, kStreamHash),
                                      (uint32_t)s, identity ? 1 : 0, gradA);
    return cudaGetLastError();
}

}  // namespace lev
