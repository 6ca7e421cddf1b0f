// Rank-revealing QR of the sketch through its Gram matrix (FP64-grade), sm_103a.
//
// The pivoted QR of Alg. 4 (xGEQP3-style greatest-trailing-norm pivoting, Sec. 7)
// and the pivoted Cholesky factorisation of G = A~^T A~ produce the same
// permutation, rank and R in exact arithmetic: the squared trailing column
// norms of the QR are the diagonal of the Schur complement of G, and the rows
// of R are the scaled pivot rows of that Schur complement. On a GPU whose FP64
// rate is low, this moves the m d^2 FP64 work into one embarrassingly parallel
// product and leaves only d^3/3 of sequential work on a d x d matrix:
//
//   k_gram_dot2 / k_gram_reduce: G = A~^T A~ with FP64-grade sums from FP32
//     arithmetic (FP64 runs at 1/64 of the FP32 rate on this GPU): each product
//     of two FP32 entries is split exactly into p + e (p = a b rounded,
//     e = fma(a, b, -p)); the products of 64 rows are summed error-free
//     (TwoSum, s + q = s_old + p exactly), their rounding errors q and e
//     gathered in an FP32 correction c, and every 64 rows s + c is added into
//     FP64 (the compensated dot product of Ogita, Rump and Oishi, with an FP64
//     outer sum). Error: about 128 u_32^2 sum |a b| per block (4e-13) plus the
//     FP64 sum over blocks, comparable to the m u_64 sum |a b| of an FP64 FMA
//     chain at the sketch sizes (m = 1,024 to 4,096).
//     Upper 32 x 32 tiles split over rows, split partials reduced in a fixed
//     order and mirrored;
//   k_pchol_grid: one cooperative grid (at most one CTA per SM; ceil(d/3) CTAs
//     up to d = 256, where a step is latency-bound; above d = 256 one thread a
//     row, 512 or 1,024 threads a CTA); CTA c owns the
//     columns l = c mod gridDim of the Schur complement in shared memory, in
//     double-float arithmetic (FP32 pairs, about 48 bits; FP64 runs at 1/64 of
//     the FP32 rate here). All CTAs keep a replicated Schur diagonal and take the
//     same pivot p_j (largest diagonal, ties to the lowest column) and the same
//     rank decision S_pp <= tau^2 S_00 without exchanging them; the owner of each
//     pivot publishes its updated column, unscaled, as soon as it is up to date,
//     and the others wait for that row only (no flag, no grid barrier per step);
//   k_pchol_cluster: the same factorisation for d <= 256 on one thread-block
//     cluster of 8 or 16 CTAs, the columns in registers, the pivot column pulled
//     from the owner's shared memory (a remote hop of about 250 ns instead of an
//     L2 round trip); it holds 16 SMs instead of ceil(d/3), which the other
//     kernels of batches in flight use. The double-float helpers live in df.cuh.
//
// The Gram route resolves |R_jj| / |R_00| down to about sqrt(m u) ~ 1e-7; the
// caller uses the Householder kernel when tau is below 1e-6 or d > 1024.
#include <atomic>
#include <climits>

#include "df.cuh"
#include "lev_common.cuh"
#include "lev_kernels.cuh"

namespace lev {

namespace {

constexpr int GT = 32;                 // Gram tile
constexpr uint64_t kClusterWaitNs = 2000000000ull;
constexpr int32_t kStatusClusterTimeout = 3;

__host__ __device__ inline int gram_tiles(int d) {
    const int nt = (d + GT - 1) / GT;
    return nt * (nt + 1) / 2;
}

__device__ inline void tile_coords(int t, int nt, int& bi, int& bj) {
    bi = 0;
    while (t >= nt - bi) { t -= nt - bi; ++bi; }
    bj = bi + t;
}

constexpr int kDot2Rows = 64;         // rows per error-free block before the FP64 add
constexpr int kGramShort = 8;         // CSR rows of at most this many entries: k_gram_csr_short

__global__ void __launch_bounds__(256) k_gram_dot2(const float* __restrict__ At, int64_t lda, int m, int d,
                                                   int rows_per_split, double* __restrict__ Gp) {
    __shared__ __align__(16) float As[kDot2Rows][GT];
    __shared__ __align__(16) float Bs[kDot2Rows][GT];
    const int nt = (d + GT - 1) / GT;
    const int T = nt * (nt + 1) / 2;
    int bi, bj;
    tile_coords(blockIdx.x, nt, bi, bj);
    const int split = blockIdx.y;
    const int r_begin = split * rows_per_split, r_end = min(m, r_begin + rows_per_split);
    const int t = threadIdx.x;
    const int ty = t >> 3, tx = t & 7;           // 32 x 8 threads -> outputs (ty, tx*4 .. tx*4+3)
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int r0 = r_begin; r0 < r_end; r0 += kDot2Rows) {
        for (int e = t; e < kDot2Rows * GT; e += 256) {
            const int r = e / GT, c = e % GT;
            const int row = r0 + r;
            const bool rok = row < r_end;
            As[r][c] = (rok && bi * GT + c < d) ? At[(int64_t)row * lda + bi * GT + c] : 0.f;
            Bs[r][c] = (rok && bj * GT + c < d) ? At[(int64_t)row * lda + bj * GT + c] : 0.f;
        }
        __syncthreads();
        float sm[4] = {0.f, 0.f, 0.f, 0.f}, cm[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
        for (int r = 0; r < kDot2Rows; ++r) {
            const float a = As[r][ty];
            const float4 b4 = *reinterpret_cast<const float4*>(&Bs[r][tx * 4]);
            const float bq[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float p = __fmul_rn(a, bq[q]);
                const float ep = __fmaf_rn(a, bq[q], -p);          // a b = p + ep exactly
                const float s1 = __fadd_rn(sm[q], p);
                const float z = __fsub_rn(s1, sm[q]);
                const float es = __fadd_rn(__fsub_rn(sm[q], __fsub_rn(s1, z)), __fsub_rn(p, z));  // s + p = s1 + es
                sm[q] = s1;
                cm[q] = __fadd_rn(cm[q], __fadd_rn(es, ep));
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] += (double)sm[q] + (double)cm[q];
        __syncthreads();
    }
    double* out = Gp + ((int64_t)split * T + blockIdx.x) * (GT * GT);
#pragma unroll
    for (int q = 0; q < 4; ++q) out[ty * GT + tx * 4 + q] = acc[q];
}

__global__ void k_gram_reduce(const double* __restrict__ Gp, int d, int splits, double* __restrict__ G) {
    const int nt = (d + GT - 1) / GT;
    const int T = nt * (nt + 1) / 2;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)T * GT * GT;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int tile = (int)(e / (GT * GT)), w = (int)(e % (GT * GT));
        int bi, bj;
        tile_coords(tile, nt, bi, bj);
        const int i = bi * GT + w / GT, j = bj * GT + w % GT;
        if (i >= d || j >= d) continue;
        double s = 0.0;
        for (int z = 0; z < splits; ++z) s += Gp[((int64_t)z * T + tile) * (GT * GT) + w];
        G[(int64_t)i * d + j] = s;
        G[(int64_t)j * d + i] = s;
    }
}

// B = A^T A of a CSR matrix as the sum of its rows' outer products (Lemma 8, Sec. 5.1), FP64, into the
// upper triangle of G (d x d, zeroed by the caller). One warp per row: the first 32 entries of a
// chunk are held one per lane and broadcast in turn as entry p; the lanes take the entries q >= p
// of the row. A product of two FP32 values is exact in FP64; the sums are FP64 atomics in L2, so
// their order (and the last bits of G) varies between runs. Duplicate columns of a row add up
// (the pair p != q on one cell counts twice, once for each order); columns outside [0, d) are
// skipped.
// Rows with more than max_len entries are left to the dense route (k_heavy_rows, k_densify_rows,
// the compensated Gram of the densified rows), rows of at most kGramShort entries to
// k_gram_csr_short.
__global__ void __launch_bounds__(256) k_gram_csr_fp64(const int64_t* __restrict__ row_ptr,
                                                       const int32_t* __restrict__ col,
                                                       const float* __restrict__ val, int64_t n, int d,
                                                       int64_t max_len, double* __restrict__ G) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < n; i += nwarps) {
        const int64_t p0 = row_ptr[i], p1 = row_ptr[i + 1];
        if (p1 - p0 > max_len || p1 - p0 <= kGramShort) continue;
        for (int64_t pb = p0; pb < p1; pb += 32) {
            const int cnt = (int)min((int64_t)32, p1 - pb);
            int my_c = -1;
            float my_v = 0.f;
            if (lane < cnt) {
                my_c = col[pb + lane];
                my_v = val[pb + lane];
            }
            for (int u = 0; u < cnt; ++u) {
                const int cp = __shfl_sync(0xffffffffu, my_c, u);
                const double vp = (double)__shfl_sync(0xffffffffu, my_v, u);
                if ((unsigned)cp >= (unsigned)d) continue;                  // uniform over the warp
                for (int64_t q = pb + u + lane; q < p1; q += 32) {
                    const int cq = col[q];
                    if ((unsigned)cq >= (unsigned)d) continue;
                    double x = vp * (double)val[q];
                    if (cq == cp && q != pb + u) x *= 2.0;
                    const int a = cp < cq ? cp : cq, b = cp < cq ? cq : cp;
                    atomicAdd(&G[(int64_t)a * d + b], x);
                }
            }
        }
    }
}

// Rows of at most kGramShort (8) entries: 8 lanes a row, four rows a warp (a row is a short chain of
// dependent loads, so a warp keeps four in flight, the next four rows' bounds loaded ahead); lane
// l holds entry l, the pairs p <= q of the row (row-major upper triangle, at most 36) go round the
// 8 lanes in 5 fixed rounds, each adding its product by an FP64 atomic as in k_gram_csr_fp64.
__device__ __forceinline__ void tri_pair_g(int t, int len, int& p, int& q) {
    p = 0;
    while (t >= len - p) {
        t -= len - p;
        ++p;
    }
    q = p + t;
}

__global__ void __launch_bounds__(256) k_gram_csr_short(const int64_t* __restrict__ row_ptr,
                                                        const int32_t* __restrict__ col,
                                                        const float* __restrict__ val, int64_t n, int d,
                                                        double* __restrict__ G) {
    const int lane = threadIdx.x & 31, seg = lane >> 3, sl = lane & 7;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t rn = warp * 4 + seg;
    int64_t np0 = rn < n ? row_ptr[rn] : 0, np1 = rn < n ? row_ptr[rn + 1] : 0;
    for (int64_t r0 = warp * 4; r0 < n; r0 += nwarps * 4) {
        const int64_t r = r0 + seg;
        const int64_t p0 = np0, p1 = np1;
        const int len = (int)(p1 - p0);
        const bool mine = r < n && len <= kGramShort;
        int c = -1;
        double v = 0.0;
        if (mine && sl < len) {
            c = col[p0 + sl];
            v = (double)val[p0 + sl];
        }
        rn = r + nwarps * 4;
        np0 = rn < n ? row_ptr[rn] : 0;
        np1 = rn < n ? row_ptr[rn + 1] : 0;
        if ((unsigned)c >= (unsigned)d) { c = -1; v = 0.0; }
        const int npairs = mine ? len * (len + 1) / 2 : 0;
#pragma unroll
        for (int round = 0; round < 5; ++round) {
            const int t = round * 8 + sl;
            int pp = 0, qq = 0;
            if (t < npairs) tri_pair_g(t, len, pp, qq);
            const int cp = __shfl_sync(0xffffffffu, c, seg * 8 + pp), cq = __shfl_sync(0xffffffffu, c, seg * 8 + qq);
            const double vp = __shfl_sync(0xffffffffu, v, seg * 8 + pp), vq = __shfl_sync(0xffffffffu, v, seg * 8 + qq);
            if (t < npairs && cp >= 0 && cq >= 0) {
                double x = vp * vq;
                if (cq == cp && qq != pp) x *= 2.0;
                const int a = cp < cq ? cp : cq, b = cp < cq ? cq : cp;
                atomicAdd(&G[(int64_t)a * d + b], x);
            }
        }
    }
}

// Indices of the rows with more than max_len entries (in no fixed order) and their count.
__global__ void k_heavy_rows(const int64_t* __restrict__ row_ptr, int64_t n, int64_t max_len,
                             unsigned long long* __restrict__ count, int32_t* __restrict__ idx) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (row_ptr[i + 1] - row_ptr[i] > max_len) idx[atomicAdd(count, 1ull)] = (int32_t)i;
}

// H (nh x d FP32, zeroed by the caller): row h = CSR row idx[h]; a repeated column adds.
__global__ void k_densify_rows(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                               const float* __restrict__ val, const int32_t* __restrict__ idx,
                               const unsigned long long* __restrict__ count, int d, float* __restrict__ H) {
    const int64_t nh = (int64_t)*count;
    for (int64_t hr = blockIdx.x; hr < nh; hr += gridDim.x) {
        const int64_t i = idx[hr];
        for (int64_t e = row_ptr[i] + threadIdx.x; e < row_ptr[i + 1]; e += blockDim.x) {
            const int c = col[e];
            if ((unsigned)c < (unsigned)d) atomicAdd(H + hr * d + c, val[e]);
        }
    }
}

// G[i][j] += D[i][j] for i <= j.
__global__ void k_add_upper(double* __restrict__ G, const double* __restrict__ D, int d) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)d * d;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / d), j = (int)(e % d);
        if (i <= j) G[e] += D[e];
    }
}

// G[j][i] = G[i][j] for i < j.
__global__ void k_mirror_upper(double* __restrict__ G, int d) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)d * d;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / d), j = (int)(e % d);
        if (i > j) G[e] = G[(int64_t)j * d + i];
    }
}

// ---------------------------------------------------------------- helpers

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Pivoted Cholesky of G (d x d FP64, symmetric) on one cooperative grid (at
// most one CTA per SM). CTA c owns the columns l = c mod gridDim and keeps them in shared
// memory. Every CTA keeps a replicated copy of the Schur diagonal, updated with
// the same FMAs as the owners' columns, so all CTAs take the same pivots and the
// same rank decisions without exchanging them.
//
// Step j with pivot p (Schur diagonal s_pp): row j of R is u / sqrt(s_pp), u the
// pivot column of the Schur complement. The owner of p publishes u UNSCALED in
// row j of U as soon as its column is up to date, so no square root or division
// sits between its update and its stores; every CTA has already computed
// 1 / sqrt(s_pp) from its own copy of the diagonal while it waited. A reader
// takes each entry of the row once it no longer holds the "unwritten" pattern
// (bounded spin); rows of U are written once, so a slow reader never races a
// fast writer. Thread t handles the indices i = t, t + 256, ... in every phase
// (read, scale, diagonal update, local argmax, column updates), which leaves two
// block barriers per step: one for the argmax, one after the column updates.
// The owner writes row j of R (scaled, original column order) to Rorig off the
// critical path; nothing reads Rorig before the kernel ends.
constexpr unsigned long long kUnwritten = 0xFFF40000DEADBEEFull;
constexpr int kGridMaxD = 1024;                    // rows of the grid factorisation
__device__ __forceinline__ unsigned long long ld_relaxed_gpu_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__global__ void k_fill_unwritten(unsigned long long* R, int64_t count) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
        R[e] = kUnwritten;
}

__device__ __forceinline__ void st_relaxed_gpu_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// The Schur complement is held in double-float: G is first scaled by 2^-e (e even, the largest
// diagonal entry in [1, 4)), so that every value the factorisation can pivot on stays inside FP32's
// exponent range (a forced pivot whose Schur diagonal falls below about 2^-126 of the largest
// diagonal entry stops the factorisation as a non-positive one would). Rows of R are written as
// double-float pairs into the bytes of Rorig, scaled by 2^(-e/2); k_df_to_fp64 turns them into
// FP64 with rscale_out = 2^(e/2) afterwards. The published rows U hold the pairs' 8-byte patterns
// (the "unwritten" sentinel has a NaN low part, which no pair has).
template <int NT>
__global__ void __launch_bounds__(NT, 1) k_pchol_grid(const double* __restrict__ Gm, int d, int m, double tau,
                                                       const int32_t* __restrict__ forced, int forced_rank,
                                                       unsigned long long* __restrict__ U, float2* __restrict__ Rdf,
                                                       double* __restrict__ rscale_out, int32_t* __restrict__ piv,
                                                       int64_t* __restrict__ rank_out, int32_t* status,
                                                       int withhold) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int G = gridDim.x, me = blockIdx.x;
    const int ncl = (d - me + G - 1) / G;                        // columns me, me + G, ...
    float2* S = reinterpret_cast<float2*>(smem);                  // ncl x d (own columns)
    float2* ubuf = S + (size_t)ncl * d;                           // d: unscaled row (owner's own entries)
    float2* rbuf = ubuf + d;                                      // d: row j of R
    float2* diag = rbuf + d;                                      // d: replicated Schur diagonal
    int* active = reinterpret_cast<int*>(diag + d);               // d
    constexpr int NW = NT / 32, RPT = kGridMaxD / NT;           // warps; rows a thread
    __shared__ __align__(16) uint4 red4[NW];                     // per warp: key lo, key hi, index
    __shared__ double red_d[NW];
    __shared__ volatile int s_abort;
    __shared__ float2 s_inv;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    // prescale 2^-e from the largest diagonal entry (the same in every CTA)
    double mx = 0.0;
    for (int i = tid; i < d; i += NT) mx = fmax(mx, Gm[(int64_t)i * d + i]);
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red_d[wid] = mx;
    __syncthreads();
    mx = red_d[0];
    for (int w = 1; w < NW; ++w) mx = fmax(mx, red_d[w]);
    int ex = 0;
    if (mx > 0.0 && mx < 1.0e300) ex = ilogb(mx) & ~1;
    const double scale = ldexp(1.0, -ex);
    if (me == 0 && tid == 0) *rscale_out = ldexp(1.0, ex / 2);
    for (int lc = 0; lc < ncl; ++lc) {
        const double* src = Gm + (int64_t)(lc * G + me) * d;     // column = row (symmetric)
        for (int i = tid; i < d; i += NT) S[(size_t)lc * d + i] = df_from_double(src[i] * scale);
    }
    for (int i = tid; i < d; i += NT) {
        active[i] = 1;
        diag[i] = df_from_double(Gm[(int64_t)i * d + i] * scale);
    }
    if (tid == 0) s_abort = 0;
    __syncthreads();
    // largest active diagonal entry, ties to the lowest index: per thread over its own indices,
    // per warp by three redux operations (max of the key's high and low words, min index among
    // the maxima), one barrier, then every warp reduces the eight warp results the same way
    auto pick = [&]() -> int {
        unsigned long long bk = 0;
        int bi = INT_MAX;
        for (int i = tid; i < d; i += NT)
            if (active[i]) {
                const unsigned long long k = df_key(diag[i]);
                if (k > bk) { bk = k; bi = i; }                       // i increases: ties keep the lowest
            }
        const unsigned hi = (unsigned)(bk >> 32), lo = (unsigned)bk;
        const unsigned mh = __reduce_max_sync(0xffffffffu, hi);
        const unsigned ml = __reduce_max_sync(0xffffffffu, hi == mh ? lo : 0u);
        const unsigned mi = __reduce_min_sync(0xffffffffu, (hi == mh && lo == ml) ? (unsigned)bi : 0xffffffffu);
        if (lane == 0) red4[wid] = make_uint4(ml, mh, mi, 0u);
        __syncthreads();
        // lane w reads warp w's result (one 16-byte load), three redux operations combine the NW
        const uint4 e = red4[lane & (NW - 1)];
        const unsigned bh = __reduce_max_sync(0xffffffffu, e.y);
        const unsigned bl = __reduce_max_sync(0xffffffffu, e.y == bh ? e.x : 0u);
        const unsigned bm = __reduce_min_sync(0xffffffffu, (e.y == bh && e.x == bl) ? e.z : 0xffffffffu);
        return (bh == 0u && bl == 0u) ? INT_MAX : (int)bm;
    };
    // rank test on the pivot's squared trailing norm: stop at a pivot that is not positive and
    // finite, or (unforced) at s_pp <= tau^2 s_00, compared through keys; the same in every thread
    unsigned long long thr = 0;
    auto stops = [&](int j, int p) -> bool {
        const float2 v = diag[p];
        if (!(v.x > 0.f) || !(v.x < 3.0e38f)) return true;
        if (j == 0) thr = df_key(df_from_double(tau * tau * df_to_double(v)));
        return !forced && df_key(v) <= thr;
    };
    const int steps = forced ? min(forced_rank, min(m, d)) : min(m, d);
    int j = 0;
    int p = -1;
    bool go = false;
    if (steps > 0) {
        p = forced ? forced[0] : pick();
        go = p >= 0 && p < d && !stops(0, p);
    }
    if (go) {
        if (p % G == me) {
            const float2* col = S + (size_t)(p / G) * d;
            for (int i = tid; i < d; i += NT)
                if (i != p) {
                    ubuf[i] = col[i];
                    st_relaxed_gpu_u64(U + i, df_bits(col[i]));
                }
        }
        if (tid == 0) s_inv = df_inv_sqrt(diag[p]);
        __syncthreads();
    }
    for (; go && j < steps; ++j) {
        const float2 inv = s_inv;
        const bool owner = (p % G) == me;
        // 1. row j of R: unscaled entries (own copy or the published row, bounded spin), scaled,
        //    and the replicated diagonal updated, index by index
        const unsigned long long* urow = U + (int64_t)j * d;
        // the published entries of this thread (at most RPT), all loads issued before any
        // is waited on, so that they share one L2 round trip
        unsigned long long first[RPT];
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int i = tid + NT * k;
            first[k] = (!owner && i < d && active[i] && i != p) ? ld_relaxed_gpu_u64(urow + i) : 0ull;
        }
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int i = tid + NT * k;
            if (i >= d) break;
            float2 r = make_float2(0.f, 0.f);
            if (active[i] && i != p) {
                float2 u;
                if (owner) {
                    u = ubuf[i];
                } else {
                    unsigned long long bits = first[k];
                    if (bits == kUnwritten) {
                        const uint64_t t0 = gtimer();
                        for (uint32_t it = 0;; ++it) {
                            bits = ld_relaxed_gpu_u64(urow + i);
                            if (bits != kUnwritten) break;
                            if ((it & 15u) == 15u && (s_abort || gtimer() - t0 > kClusterWaitNs)) {
                                if (!s_abort) atomicExch(status, kStatusClusterTimeout);
                                s_abort = 1;
                                break;
                            }
                        }
                    }
                    u = df_of_bits(bits);
                }
                r = df_mul(u, inv);
                diag[i] = df_sub_mul(diag[i], r, r);
            }
            if (i == p) active[i] = 0;
            rbuf[i] = r;
        }
        if (owner) {
            float2* row = Rdf + (int64_t)j * d;
            for (int i = tid; i < d; i += NT)
                if (i != p && active[i]) row[i] = rbuf[i];
            if (tid == 0) row[p] = df_mul(diag[p], inv);              // R_jj = s_pp / sqrt(s_pp)
        }
        if (me == 0 && tid == 0) piv[j] = p;
        // 2. the next pivot and its rank test (one barrier)
        int pn;
        if (forced) {
            pn = j + 1 < steps ? forced[j + 1] : -1;
            __syncthreads();
        } else {
            pn = pick();
        }
        if (s_abort) break;
        const bool go_on = j + 1 < steps && pn >= 0 && pn < d && active[pn] && !stops(j + 1, pn);
        // 3. owner of the next pivot: its column first, published unscaled entry by entry
        if (go_on && pn % G == me) {
            float2* col = S + (size_t)(pn / G) * d;
            const float2 rc = rbuf[pn];
            unsigned long long* urow_n = U + (int64_t)(j + 1) * d;
            for (int i = tid; i < d; i += NT)
                if (active[i]) {
                    const float2 v = df_sub_mul(col[i], rbuf[i], rc);
                    col[i] = v;
                    if (i != pn) {
                        ubuf[i] = v;
                        if (j + 1 != withhold) st_relaxed_gpu_u64(urow_n + i, df_bits(v));
                    }
                }
        }
        // 4. the next step's scale factor (every CTA, while the row travels)
        if (go_on && tid == 0) s_inv = df_inv_sqrt(diag[pn]);
        // 5. the other own columns
        for (int lc = 0; lc < ncl; ++lc) {
            const int c = lc * G + me;
            if (c == pn || !active[c]) continue;
            const float2 rc = rbuf[c];
            float2* col = S + (size_t)lc * d;
            for (int i = tid; i < d; i += NT)
                if (active[i]) col[i] = df_sub_mul(col[i], rbuf[i], rc);
        }
        __syncthreads();
        if (!go_on) { ++j; break; }
        p = pn;
    }
    if (me == 0 && tid == 0) *rank_out = j;
}

// ---- the same factorisation on one thread-block cluster (d <= 256) ----
// C CTAs (8 or 16) of 256 T threads. CTA me owns the columns c = q C + me (q < NCL) of the Schur
// complement; row i of them is held in registers by the T threads i + 256 t (t < T), NCL / T columns
// each. The Schur diagonal is replicated: entry i is held by thread i (t = 0) in every CTA. A step
// with pivot p: thread i of an active row reads entry i of column p from the owner's array F (shared
// memory; each column written once when it becomes a pivot, sentinel-filled before; a remote load
// repeated, bounded, until it is not the sentinel), forms r_i = u_i / sqrt(s_pp) and the new
// diagonal entry, and writes r_i to the CTA's row buffer and its warp's argmax to shared memory;
// one block barrier, after which the row's other threads read r_i; every thread takes the next
// pivot from the eight warp results (ties to the lowest index, the same in every CTA). The thread
// holding the next pivot's column applies row j to it first and publishes it; every thread then
// applies row j to its other columns while that column travels, skipping the held columns that
// were pivots (a warp's threads hold the same columns, so the skip is uniform). A retired row has
// r = 0, so its updates leave it unchanged. Same arithmetic, outputs and stopping rule as
// k_pchol_grid.
constexpr int kClRows = 256;

__device__ __forceinline__ uint32_t cl_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cl_size() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cl_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t cl_mapa(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
__device__ __forceinline__ unsigned long long cl_ld_u64(uint32_t addr) {
    unsigned long long v;
    asm volatile("ld.relaxed.cluster.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ void cl_st_local_u64(uint32_t addr, unsigned long long v) {
    asm volatile("st.relaxed.cluster.shared::cta.u64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
}
// Inverse of order_key32: the FP32 value a key was made from.
__device__ __forceinline__ float key32_value(unsigned k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

template <int NCL, int T>
__global__ void __launch_bounds__(kClRows * T, 1) k_pchol_cluster(const double* __restrict__ Gm, int d, int m,
                                                                  double tau, const int32_t* __restrict__ forced,
                                                                  int forced_rank, float2* __restrict__ Rdf,
                                                                  double* __restrict__ rscale_out,
                                                                  int32_t* __restrict__ piv,
                                                                  int64_t* __restrict__ rank_out, int32_t* status,
                                                                  int withhold) {
    constexpr int NQ = NCL / T;                                           // columns a thread holds
    static_assert(NQ * T == NCL, "columns split evenly over a row's threads");
    extern __shared__ __align__(16) uint8_t smem[];
    const int C = (int)cl_size(), me = (int)cl_rank();
    unsigned long long* F = reinterpret_cast<unsigned long long*>(smem);   // NCL x d: published columns
    float2* rb = reinterpret_cast<float2*>(F + (size_t)NCL * d);          // 2 x d: row j of R, by parity
    __shared__ __align__(16) uint4 red[2][8];                              // per warp: key lo, key hi, index
    __shared__ float2 s_next[2];                                          // forced: the next pivot's s_pp
    __shared__ double red_d[8];
    __shared__ volatile int s_abort;
    const int i = threadIdx.x % kClRows, t = threadIdx.x / kClRows;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;            // warps 0..7: t = 0
    const bool row_ok = i < d;
    // prescale 2^-e from the largest diagonal entry (the same in every CTA)
    if (t == 0) {
        double mx = row_ok ? Gm[(int64_t)i * d + i] : 0.0;
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) red_d[wid] = mx;
    }
    __syncthreads();
    double mx = red_d[0];
#pragma unroll
    for (int w = 1; w < 8; ++w) mx = fmax(mx, red_d[w]);
    int ex = 0;
    if (mx > 0.0 && mx < 1.0e300) ex = ilogb(mx) & ~1;
    const double scale = ldexp(1.0, -ex);
    if (me == 0 && threadIdx.x == 0) *rscale_out = ldexp(1.0, ex / 2);
    float2 S[NQ];                                                         // columns (t NQ + k) C + me
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
        const int c = (t * NQ + k) * C + me;
        S[k] = (row_ok && c < d) ? df_from_double(Gm[(int64_t)c * d + i] * scale) : make_float2(0.f, 0.f);
    }
    float2 dg = row_ok ? df_from_double(Gm[(int64_t)i * d + i] * scale) : make_float2(0.f, 0.f);
    bool active = row_ok;
    for (int e = threadIdx.x; e < NCL * d; e += kClRows * T) F[e] = kUnwritten;
    if (threadIdx.x == 0) s_abort = 0;
    __syncthreads();
    cl_sync();                                       // every CTA's F is filled before any is read

    // the warp's largest active diagonal entry (key, lowest index among equal keys) into buffer b
    auto warp_pick = [&](int b) {
        const unsigned long long k = active ? df_key(dg) : 0ull;
        const unsigned hi = (unsigned)(k >> 32), lo = (unsigned)k;
        const unsigned mh = __reduce_max_sync(0xffffffffu, hi);
        const unsigned ml = __reduce_max_sync(0xffffffffu, hi == mh ? lo : 0u);
        const unsigned mi = __reduce_min_sync(0xffffffffu, (hi == mh && lo == ml && k != 0ull) ? (unsigned)i : 0xffffffffu);
        if (lane == 0) red[b][wid] = make_uint4(ml, mh, mi, 0u);
    };
    // after the barrier: the block's pick (INT_MAX if no active row) and its diagonal entry; lane w of
    // every warp reads warp w's result (one 16-byte load), three redux operations combine them
    auto block_pick = [&](int b, float2& val) -> int {
        const uint4 e = red[b][lane & 7];
        const unsigned mh = __reduce_max_sync(0xffffffffu, e.y);
        const unsigned ml = __reduce_max_sync(0xffffffffu, e.y == mh ? e.x : 0u);
        const unsigned mi = __reduce_min_sync(0xffffffffu, (e.y == mh && e.x == ml) ? e.z : 0xffffffffu);
        val = make_float2(key32_value(mh), key32_value(ml));
        return (mh == 0u && ml == 0u) ? INT_MAX : (int)mi;
    };
    // entry i of column c's slot in the owner's F (shared::cluster address)
    auto remote_entry = [&](int c) -> uint32_t {
        return cl_mapa((uint32_t)__cvta_generic_to_shared(F + (size_t)(c / C) * d + i), (uint32_t)(c % C));
    };
    // this thread's copy of column c (held by thread t = (c / C) / NQ of the owner), or 0
    auto own_value = [&](int c) -> float2 {
        float2 v = make_float2(0.f, 0.f);
        const int q = c / C;
#pragma unroll
        for (int k = 0; k < NQ; ++k)
            if (t * NQ + k == q) v = S[k];
        return v;
    };

    const int steps = forced ? min(forced_rank, min(m, d)) : min(m, d);
    unsigned long long thr = 0;
    int j = 0, p = -1;
    float2 sp = make_float2(0.f, 0.f);
    bool go = false;
    if (steps > 0) {
        const int f0 = forced ? forced[0] : -1;
        if (forced) {
            if (t == 0 && i == f0) s_next[0] = active ? dg : make_float2(0.f, 0.f);
        } else if (t == 0) {
            warp_pick(0);
        }
        __syncthreads();
        if (forced) {
            p = f0;
            sp = (p >= 0 && p < d) ? s_next[0] : make_float2(0.f, 0.f);
        } else {
            p = block_pick(0, sp);
        }
        go = p >= 0 && p < d && sp.x > 0.f && sp.x < 3.0e38f;
        if (go) thr = df_key(df_from_double(tau * tau * df_to_double(sp)));
        go = go && (forced || df_key(sp) > thr);
        // the thread holding the first pivot's column publishes it (unscaled)
        if (go && p % C == me && (p / C) / NQ == t && active && i != p)
            cl_st_local_u64((uint32_t)__cvta_generic_to_shared(F + (size_t)(p / C) * d + i), df_bits(own_value(p)));
    }
    float2 inv = go ? df_inv_sqrt(sp) : make_float2(0.f, 0.f);
    unsigned retired = 0u;                            // held columns that were pivots (no longer read)
    for (; go && j < steps; ++j) {
        const int b = j & 1;
        if (p % C == me && (p / C) / NQ == t) retired |= 1u << ((p / C) - t * NQ);
        // 1. (threads t = 0) entry i of the pivot column (own copy, or the owner's F), row j of R, the
        //    diagonal; the other threads of the row take r_i from the row buffer after the barrier
        float2 r = make_float2(0.f, 0.f);
        const bool was_active = active;
        if (t == 0 && active && i != p) {
            float2 u;
            const int q = p / C;
            if (p % C == me && q / NQ == 0) {
                u = own_value(p);
            } else {
                // the owner's F: this CTA's (where thread q / NQ of the row published it) or another's
                const uint32_t a = p % C == me ? (uint32_t)__cvta_generic_to_shared(F + (size_t)q * d + i)
                                               : remote_entry(p);
                unsigned long long bits = cl_ld_u64(a);
                if (bits == kUnwritten) {
                    const uint64_t t0 = gtimer();
                    for (uint32_t it = 0;; ++it) {
                        bits = cl_ld_u64(a);
                        if (bits != kUnwritten) break;
                        if ((it & 15u) == 15u && (s_abort || gtimer() - t0 > kClusterWaitNs)) {
                            if (!s_abort) atomicExch(status, kStatusClusterTimeout);
                            s_abort = 1;
                            break;
                        }
                    }
                }
                u = df_of_bits(bits);
            }
            r = df_mul(u, inv);
            dg = df_sub_mul(dg, r, r);
        }
        if (i == p) active = false;
        if (t == 0) {
            if (row_ok) rb[b * d + i] = r;
            if (j % C == me && was_active) Rdf[(int64_t)j * d + i] = i == p ? df_mul(sp, inv) : r;   // R_jj = sqrt(s_pp)
            if (me == 0 && i == 0) piv[j] = p;
        }
        // 2. the next pivot (one barrier)
        const int fn = forced ? (j + 1 < steps ? forced[j + 1] : -1) : -1;
        if (forced) {
            if (t == 0 && i == fn) s_next[b ^ 1] = active ? dg : make_float2(0.f, 0.f);
        } else if (t == 0) {
            warp_pick(b);
        }
        __syncthreads();
        if (s_abort) break;
        int pn;
        float2 spn;
        if (forced) {
            pn = fn;
            spn = (pn >= 0 && pn < d) ? s_next[b ^ 1] : make_float2(0.f, 0.f);
        } else {
            pn = block_pick(b, spn);
        }
        const bool go_on = j + 1 < steps && pn >= 0 && pn < d && spn.x > 0.f && spn.x < 3.0e38f &&
                           (forced || df_key(spn) > thr);
        const float2* rj = rb + (size_t)b * d;
        if (t != 0 && row_ok) r = rj[i];
        // 3. the thread holding the next pivot's column: that column first, published unscaled
        int kn = -1;
        if (go_on && pn % C == me && (pn / C) / NQ == t) {
            kn = (pn / C) - t * NQ;
            const float2 rc = rj[pn];
            float2 v = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < NQ; ++k)
                if (k == kn) {
                    S[k] = df_sub_mul(S[k], r, rc);
                    v = S[k];
                }
            if (active && i != pn && j + 1 != withhold)
                cl_st_local_u64((uint32_t)__cvta_generic_to_shared(F + (size_t)(pn / C) * d + i), df_bits(v));
        }
        // 4. the other held columns that are not yet pivots (the same for the whole warp)
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
            const int c = (t * NQ + k) * C + me;
            if (k != kn && c < d && !((retired >> k) & 1u)) S[k] = df_sub_mul(S[k], r, rj[c]);
        }
        if (!go_on) {
            ++j;
            break;
        }
        inv = df_inv_sqrt(spn);
        sp = spn;
        p = pn;
    }
    if (me == 0 && threadIdx.x == 0) *rank_out = j;
    // no CTA leaves while another may still read its F
    __syncthreads();
    cl_sync();
}

// R (d x d) from the double-float rows k_pchol_grid wrote into the same bytes: (hi + lo) rscale.
__global__ void k_df_to_fp64(double* __restrict__ R, const double* __restrict__ rscale, int64_t count) {
    const double sc = *rscale;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = reinterpret_cast<const float2*>(R)[e];
        R[e] = ((double)v.x + (double)v.y) * sc;
    }
}

}  // namespace

// Row splits of the Gram product. The FP64 pipe of an SM is shared by its resident CTAs, so the
// SM with the most CTAs sets the time: take the split count whose CTA total fills its last wave
// over the SMs best (the largest such count within 1%), with the FP64 partials held to 4 MB.
int gram_splits(int64_t m, int64_t d) {
    static std::atomic<int> sms_cached{0};               // host threads share it
    int sms = sms_cached.load(std::memory_order_relaxed);
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                      cudaSuccess || sms < 1)
            sms = 152;
        sms_cached.store(sms, std::memory_order_relaxed);
    }
    const int64_t T = gram_tiles((int)d);
    const int64_t blocks = (m + 15) / 16;
    int64_t cap = ((int64_t)4 << 20) / (T * GT * GT * (int64_t)sizeof(double));
    if (cap > blocks) cap = blocks;
    if (cap < 1) cap = 1;
    int64_t best = 1;
    double best_eff = -1.0;
    for (int64_t sp = 1; sp <= cap; ++sp) {
        const int64_t ctas = T * sp, waves = (ctas + sms - 1) / sms;
        const double eff = (double)ctas / ((double)sms * (double)waves);
        if (eff > best_eff + 0.01 || eff >= best_eff - 0.01) {
            if (eff > best_eff) best_eff = eff;
            best = sp;
        }
    }
    return (int)best;
}

size_t gram_partial_doubles(int64_t m, int64_t d) {
    return (size_t)gram_splits(m, d) * gram_tiles((int)d) * GT * GT;
}

cudaError_t launch_gram_fp64(const float* A, int64_t lda, int64_t m, int64_t d, double* Gp, double* G,
                             cudaStream_t st) {
    const int splits = gram_splits(m, d);
    const int rows_per_split = (int)(((m + splits - 1) / splits + kDot2Rows - 1) / kDot2Rows * kDot2Rows);
    dim3 grid((unsigned)gram_tiles((int)d), (unsigned)splits);
    k_gram_dot2<<<grid, 256, 0, st>>>(A, lda, (int)m, (int)d, rows_per_split, Gp);
    k_gram_reduce<<<152 * 4, 256, 0, st>>>(Gp, (int)d, splits, G);
    return cudaGetLastError();
}

cudaError_t launch_gram_csr_fp64(const int64_t* row_ptr, const int32_t* col, const float* val, int64_t n,
                                 int64_t d, double* G, cudaStream_t st) {
    return launch_gram_csr_light(row_ptr, col, val, n, d, INT64_MAX, nullptr, G, st);
}

cudaError_t launch_gram_csr_light(const int64_t* row_ptr, const int32_t* col, const float* val, int64_t n, int64_t d,
                                  int64_t max_len, const double* Gheavy, double* G, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(G, 0, sizeof(double) * (size_t)(d * d), st);
    if (e != cudaSuccess) return e;
    int64_t grid = (n * 32 + 255) / 256;
    if (grid > 152 * 16) grid = 152 * 16;
    if (grid < 1) grid = 1;
    k_gram_csr_fp64<<<(unsigned)grid, 256, 0, st>>>(row_ptr, col, val, n, (int)d, max_len, G);
    int64_t grid_s = (n * 8 + 255) / 256;               // four rows a warp
    if (grid_s > 152 * 64) grid_s = 152 * 64;
    if (grid_s < 1) grid_s = 1;
    k_gram_csr_short<<<(unsigned)grid_s, 256, 0, st>>>(row_ptr, col, val, n, (int)d, G);
    if (Gheavy) k_add_upper<<<152 * 4, 256, 0, st>>>(G, Gheavy, (int)d);
    k_mirror_upper<<<152 * 4, 256, 0, st>>>(G, (int)d);
    return cudaGetLastError();
}

cudaError_t launch_heavy_rows(const int64_t* row_ptr, int64_t n, int64_t max_len, unsigned long long* count,
                              int32_t* idx, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    int64_t grid = (n + 255) / 256;
    if (grid > 152 * 16) grid = 152 * 16;
    if (grid < 1) grid = 1;
    k_heavy_rows<<<(unsigned)grid, 256, 0, st>>>(row_ptr, n, max_len, count, idx);
    return cudaGetLastError();
}

cudaError_t launch_densify_rows(const int64_t* row_ptr, const int32_t* col, const float* val, const int32_t* idx,
                                const unsigned long long* count, int64_t nh, int64_t d, float* H, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(H, 0, sizeof(float) * (size_t)(nh * d), st);
    if (e != cudaSuccess) return e;
    const int64_t grid = nh < 152 * 16 ? (nh > 0 ? nh : 1) : 152 * 16;
    k_densify_rows<<<(unsigned)grid, 256, 0, st>>>(row_ptr, col, val, idx, count, (int)d, H);
    return cudaGetLastError();
}

cudaError_t launch_gram_pivoted_cholesky(const float* Atilde, int64_t m, int64_t d, double tau,
                                         const int32_t* forced, int64_t forced_rank, const QrScratch& q,
                                         int32_t* status, cudaStream_t st, cudaEvent_t after_gram) {
    cudaError_t e = launch_gram_fp64(Atilde, d, m, d, q.Gp, q.G, st);
    if (e != cudaSuccess) return e;
    if (after_gram && (e = cudaEventRecord(after_gram, st)) != cudaSuccess) return e;
    return launch_pivoted_cholesky(m, d, tau, forced, forced_rank, q, status, st);
}

// The cluster form for d <= 256: C CTAs of one cluster, NCL columns a CTA. Returns
// cudaErrorNotSupported (nothing launched) when no such cluster can be resident on this GPU.
template <int NCL, int T>
cudaError_t launch_pchol_cluster(int C, int64_t m, int64_t d, double tau, const int32_t* forced, int64_t forced_rank,
                                 const QrScratch& q, int32_t* status, cudaStream_t st) {
    static std::atomic<int> resident[2][64] = {};         // per (C > 8, device): 1 yes, -1 no, 0 unknown
    const size_t smem = sizeof(unsigned long long) * (size_t)NCL * d + sizeof(float2) * 2 * (size_t)d;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)C);
    cfg.blockDim = dim3(kClRows * T);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    std::atomic<int>* known = dev >= 0 && dev < 64 ? &resident[C > 8 ? 1 : 0][dev] : nullptr;
    if (known && known->load(std::memory_order_relaxed) < 0) return cudaErrorNotSupported;
    if (C > 8 && (e = cudaFuncSetAttribute(k_pchol_cluster<NCL, T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) !=
                     cudaSuccess) {
        cudaGetLastError();
        if (known) known->store(-1, std::memory_order_relaxed);
        return cudaErrorNotSupported;
    }
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(k_pchol_cluster<NCL, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
        return e;
    if (!known || known->load(std::memory_order_relaxed) == 0) {
        int clusters = 0;
        e = cudaOccupancyMaxActiveClusters(&clusters, k_pchol_cluster<NCL, T>, &cfg);
        if (e != cudaSuccess || clusters < 1) {
            cudaGetLastError();
            if (known) known->store(-1, std::memory_order_relaxed);
            return cudaErrorNotSupported;
        }
        if (known) known->store(1, std::memory_order_relaxed);
    }
    const double* S = q.G;
    float2* Rdf = reinterpret_cast<float2*>(q.Rorig);
    double* rscale = q.norms;
    const int withhold = fault_pivot_wait() ? 1 : -1;    // LEV_FAULT=pivwait: step 1's column is never published
    e = cudaLaunchKernelEx(&cfg, k_pchol_cluster<NCL, T>, S, (int)d, (int)m, tau, forced, (int)forced_rank, Rdf, rscale,
                           (int32_t*)q.piv, (int64_t*)q.rank, status, withhold);
    if (e != cudaSuccess) return e;
    k_df_to_fp64<<<152 * 2, 256, 0, st>>>(q.Rorig, q.norms, d * d);
    return cudaGetLastError();
}

cudaError_t launch_pivoted_cholesky(int64_t m, int64_t d, double tau, const int32_t* forced, int64_t forced_rank,
                                    const QrScratch& q, int32_t* status, cudaStream_t st) {
    cudaError_t e;
    // d <= 256: one cluster (16 columns a CTA: 8 CTAs up to d = 128, 16 above; 32 columns on 8 CTAs
    // where a 16-CTA cluster cannot be resident)
    if (d >= 1 && d <= 256) {
        if (d <= 128)
            e = launch_pchol_cluster<16, 2>(8, m, d, tau, forced, forced_rank, q, status, st);
        else if ((e = launch_pchol_cluster<16, 2>(16, m, d, tau, forced, forced_rank, q, status, st)) ==
                 cudaErrorNotSupported)
            e = launch_pchol_cluster<32, 2>(8, m, d, tau, forced, forced_rank, q, status, st);
        if (e != cudaErrorNotSupported) return e;
    }
    // cooperative grid over the SMs (at most one CTA per SM), own columns in shared memory. Up to
    // d = 256 a step is bound by the latency of the published row, not by the FP64 work, so each
    // CTA takes three columns (ceil(d / 3) CTAs): a factorisation alone takes about 7% longer, and
    // the SMs it leaves free run the kernels of other batches in flight. The grid does not change
    // the result (every CTA takes the same pivots; each entry sees the same operations).
    int sms = 0, dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if (sms < 1 || d < 1 || d > kGridMaxD) return cudaErrorInvalidValue;
    int pgrid = sms < (int)d ? sms : (int)d;
    if (d <= 256 && pgrid > (int)(d + 2) / 3) pgrid = (int)(d + 2) / 3;
    const size_t ncl = ((size_t)d + pgrid - 1) / pgrid;
    if (ncl > 32) return cudaErrorInvalidConfiguration;          // per-CTA bookkeeping holds 32 columns
    const size_t smem = sizeof(float2) * (ncl * d + 3 * (size_t)d) + sizeof(int) * (size_t)d + 64;
    // one row of the sketch's Gram matrix a thread where d > 256 (512 or 1,024 threads): the Schur
    // updates of a step are a chain of dependent FP32 operations per row, so more threads shorten it
    const int nt = d <= 256 ? 256 : d <= 512 ? 512 : 1024;
    const void* fn = nt == 256 ? (const void*)k_pchol_grid<256>
                   : nt == 512 ? (const void*)k_pchol_grid<512> : (const void*)k_pchol_grid<1024>;
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
    k_fill_unwritten<<<152 * 4, 256, 0, st>>>(reinterpret_cast<unsigned long long*>(q.U), d * d);
    const double* S = q.G;
    const int32_t* fp = forced;
    int fr = (int)forced_rank, di = (int)d, mi = (int)m;
    unsigned long long* U = reinterpret_cast<unsigned long long*>(q.U);
    float2* Rdf = reinterpret_cast<float2*>(q.Rorig);
    double* rscale = q.norms;                                    // unused by the Gram route otherwise
    int withhold = fault_pivot_wait() ? 1 : -1;          // LEV_FAULT=pivwait: step 1's column is never published
    void* kargs[] = {&S, &di, &mi, &tau, &fp, &fr, &U, &Rdf, &rscale, (void*)&q.piv, (void*)&q.rank, &status, &withhold};
    e = cudaLaunchCooperativeKernel(fn, dim3((unsigned)pgrid), dim3((unsigned)nt), kargs, smem, st);
    if (e != cudaSuccess) return e;
    k_df_to_fp64<<<152 * 2, 256, 0, st>>>(q.Rorig, q.norms, d * d);
    return cudaGetLastError();
}

}  // namespace lev
