// CountGauss sketch A~ = G (S A) (Alg. 3) on sm_103a.
//
//  * bucket permutation: counting sort of the rows by their CountSketch bucket
//    (hash and sign of Sec. 3.4.3), rows ascending inside a bucket, so that the
//    sums below run in a fixed order (bit-identical repeat runs);
//  * CountSketch: one warp per bucket gathers its rows with 128-bit loads and
//    writes the bucket row of B = S A once (no atomics), or, for the BF16 forms
//    of the Gaussian stage, writes B directly as that stage's K-major operand;
//  * G: Box-Muller by counter, generated once per (seed, m, s) into a cache;
//  * Gaussian stage A~ = G B: FP32 SIMT split-K GEMM with a fixed-order
//    reduction of the split partials (tensor-core forms live in tc_sketch.cu).
#include <cuda_bf16.h>

#include "lev_common.cuh"
#include "lev_kernels.cuh"

namespace lev {

namespace {

constexpr uint32_t kSignBit = 0x80000000u;

// Local row i of a row shard is hashed by its global index row0 + i, so the shards' sketches
// are column blocks of one S and add up to the sketch of the whole matrix.
__global__ void k_bucket_hist(int64_t n, int64_t row0, uint32_t s, uint64_t key, int* count) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; i < n; i += stride) {
        uint64_t x = splitmix64(key, (uint64_t)(row0 + i));
        atomicAdd(&count[bucket_of(x, s)], 1);
    }
}

// Exclusive scan of count[0..s) into off[0..s], single CTA of 1024 threads:
// tiles of 4096 counts loaded as int4 (coalesced), warp-shuffle scans, a
// running carry between tiles.
__global__ void __launch_bounds__(1024) k_scan_offsets(const int* count, int* off, int s) {
    __shared__ int warp_tot[32];
    __shared__ int carry_s;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (t == 0) carry_s = 0;
    __syncthreads();
    for (int base = 0; base < s; base += 4096) {
        const int i0 = base + t * 4;
        int v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = (i0 + q < s) ? count[i0 + q] : 0;
        const int local = v[0] + v[1] + v[2] + v[3];
        int incl = local;                                   // inclusive warp scan of the thread sums
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) warp_tot[w] = incl;
        __syncthreads();
        if (w == 0) {
            int wt = warp_tot[lane];
            int wi = wt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += y;
            }
            warp_tot[lane] = wi - wt;                       // exclusive prefix of warp totals
        }
        __syncthreads();
        int run = carry_s + warp_tot[w] + incl - local;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (i0 + q < s) off[i0 + q] = run;
            run += v[q];
        }
        __syncthreads();
        if (t == 1023) carry_s = run;                       // thread 1023 holds the tile's end
        __syncthreads();
    }
    if (t == 0) off[s] = carry_s;
}

__global__ void k_bucket_scatter(int64_t n, int64_t row0, uint32_t s, uint64_t key, const int* off,
                                 int* cursor, uint32_t* out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; i < n; i += stride) {
        uint64_t x = splitmix64(key, (uint64_t)(row0 + i));
        uint32_t b = bucket_of(x, s);
        int pos = off[b] + atomicAdd(&cursor[b], 1);
        out[pos] = (uint32_t)i | ((x & 1ull) ? kSignBit : 0u);
    }
}

// Sort each bucket segment by row index (rank sort; rows are distinct).
__global__ void k_segment_sort(const int* off, int s, const uint32_t* in, uint32_t* out) {
    const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    const int nwarps = (int)((gridDim.x * (int64_t)blockDim.x) >> 5);
    for (int b = warp; b < s; b += nwarps) {
        const int o0 = off[b], len = off[b + 1] - o0;
        for (int e = lane; e < len; e += 32) {
            const uint32_t ve = in[o0 + e];
            const uint32_t ke = ve & ~kSignBit;
            int rank = 0;
            for (int f = 0; f < len; ++f) rank += ((in[o0 + f] & ~kSignBit) < ke);
            out[o0 + rank] = ve;
        }
    }
}

__device__ __forceinline__ float4 ld_stream_f4(const float* p) {
    float4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
    return v;
}

// Warp per bucket; lane holds columns c*128 + lane*4 .. +3 for c < NC.
// Rows are taken U at a time so that U*NC 128-bit loads are in flight.
template <int NC, int U>
__global__ void __launch_bounds__(256) k_countsketch_dense_v4(
        const float* __restrict__ A, int64_t lda, int d, const int* __restrict__ off,
        const uint32_t* __restrict__ perm, int s, float* __restrict__ B) {
    const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    const int nwarps = (int)((gridDim.x * (int64_t)blockDim.x) >> 5);
    for (int b = warp; b < s; b += nwarps) {
        float4 acc[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = make_float4(0.f, 0.f, 0.f, 0.f);
        const int t0 = off[b], t1 = off[b + 1];
        for (int t = t0; t < t1; t += U) {
            float4 v[U][NC];
            float sg[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool ok = (t + u) < t1;
                const uint32_t e = ok ? perm[t + u] : 0u;
                sg[u] = ok ? ((e & kSignBit) ? -1.f : 1.f) : 0.f;
                const float* row = A + (int64_t)(e & ~kSignBit) * lda;
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const int col = c * 128 + lane * 4;
                    v[u][c] = (ok && col < d) ? ld_stream_f4(row + col) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    acc[c].x = fmaf(sg[u], v[u][c].x, acc[c].x);
                    acc[c].y = fmaf(sg[u], v[u][c].y, acc[c].y);
                    acc[c].z = fmaf(sg[u], v[u][c].z, acc[c].z);
                    acc[c].w = fmaf(sg[u], v[u][c].w, acc[c].w);
                }
            }
        }
        float* out = B + (int64_t)b * d;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int col = c * 128 + lane * 4;
            if (col < d) *reinterpret_cast<float4*>(out + col) = acc[c];
        }
    }
}

// Octet o of buckets (rows: 8 x d FP32 in shared memory, bucket 8 o + w in row w) written into
// the blocked K-major operand img[g][c][k] = B[64 g + k][c]: thread c writes the eight buckets of
// column c as one 16-byte piece of hi (and of lo), rounded pairwise: hi = bf16(x), lo = bf16(x - hi).
template <bool SPLIT>
__device__ __forceinline__ void write_operand_octet(const float* rows, int d, int o, __nv_bfloat16* __restrict__ hi,
                                                    __nv_bfloat16* __restrict__ lo) {
    const int64_t base = ((int64_t)(o >> 3) * d) * 64 + (o & 7) * 8;
    for (int c = threadIdx.x; c < d; c += blockDim.x) {
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float x0 = rows[(2 * k) * d + c], x1 = rows[(2 * k + 1) * d + c];
            const __nv_bfloat162 h2 = __floats2bfloat162_rn(x0, x1);
            hw[k] = *reinterpret_cast<const uint32_t*>(&h2);
            if constexpr (SPLIT) {
                const float2 hf = __bfloat1622float2(h2);
                const __nv_bfloat162 l2 = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
                lw[k] = *reinterpret_cast<const uint32_t*>(&l2);
            }
        }
        const int64_t at = base + (int64_t)c * 64;
        *reinterpret_cast<uint4*>(hi + at) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        if constexpr (SPLIT) *reinterpret_cast<uint4*>(lo + at) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
}

// The same sums, written as the K-major operand of the tensor-core Gaussian stage instead of B:
// the BF16 image (and, split, the BF16 image of the remainder) of B^T, blocked by 64 buckets,
//   img[g][c][k] = B[64 g + k][c]   (g < ld / 64, c < d, k < 64; buckets s..ld zero),
// so that a 2-D tensor copy of 64 x rows over (ld / 64) d rows of 64 elements takes K block g of
// rows c. A CTA takes eight consecutive buckets (one a warp, the loop of k_countsketch_dense_v4),
// stages their rows in shared memory (two buffers, one barrier an octet) and writes them with
// write_operand_octet, whose rounding is the transpose kernel's.
template <int NC, int U, bool SPLIT>
__global__ void __launch_bounds__(256) k_countsketch_dense_op(
        const float* __restrict__ A, int64_t lda, int d, const int* __restrict__ off,
        const uint32_t* __restrict__ perm, int s, int64_t ld, __nv_bfloat16* __restrict__ hi,
        __nv_bfloat16* __restrict__ lo) {
    extern __shared__ float4 stage4[];                           // [2][8][d / 4]
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int dq = d >> 2;
    const int noct = (int)(ld >> 3);
    int buf = 0;
    for (int o = blockIdx.x; o < noct; o += gridDim.x, buf ^= 1) {
        const int b = 8 * o + w;
        float4 acc[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (b < s) {
            const int t0 = off[b], t1 = off[b + 1];
            for (int t = t0; t < t1; t += U) {
                float4 v[U][NC];
                float sg[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const bool ok = (t + u) < t1;
                    const uint32_t e = ok ? perm[t + u] : 0u;
                    sg[u] = ok ? ((e & kSignBit) ? -1.f : 1.f) : 0.f;
                    const float* row = A + (int64_t)(e & ~kSignBit) * lda;
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        const int col = c * 128 + lane * 4;
                        v[u][c] = (ok && col < d) ? ld_stream_f4(row + col) : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        acc[c].x = fmaf(sg[u], v[u][c].x, acc[c].x);
                        acc[c].y = fmaf(sg[u], v[u][c].y, acc[c].y);
                        acc[c].z = fmaf(sg[u], v[u][c].z, acc[c].z);
                        acc[c].w = fmaf(sg[u], v[u][c].w, acc[c].w);
                    }
                }
            }
        }
        float4* mine = stage4 + (size_t)(buf * 8 + w) * dq;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int q = c * 32 + lane;
            if (q < dq) mine[q] = acc[c];
        }
        // the buffer written here was last read two octets ago, before the previous barrier
        __syncthreads();
        write_operand_octet<SPLIT>(reinterpret_cast<const float*>(stage4 + (size_t)buf * 8 * dq), d, o, hi, lo);
    }
}

// Any alignment: lane j holds columns j, j+32, ...; one column block at a time.
__global__ void __launch_bounds__(256) k_countsketch_dense_scalar(
        const float* __restrict__ A, int64_t lda, int d, const int* __restrict__ off,
        const uint32_t* __restrict__ perm, int s, float* __restrict__ B) {
    const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    const int nwarps = (int)((gridDim.x * (int64_t)blockDim.x) >> 5);
    for (int b = warp; b < s; b += nwarps) {
        const int t0 = off[b], t1 = off[b + 1];
        for (int c0 = 0; c0 < d; c0 += 256) {
            float acc[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[c] = 0.f;
            for (int t = t0; t < t1; ++t) {
                const uint32_t e = perm[t];
                const float sg = (e & kSignBit) ? -1.f : 1.f;
                const float* row = A + (int64_t)(e & ~kSignBit) * lda;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int col = c0 + c * 32 + lane;
                    if (col < d) acc[c] = fmaf(sg, __ldg(row + col), acc[c]);
                }
            }
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int col = c0 + c * 32 + lane;
                if (col < d) B[(int64_t)b * d + col] = acc[c];
            }
        }
    }
}

// CSR: warp per bucket, dense accumulator row of d floats in shared memory.
// Rows of a bucket are added one after the other (__syncwarp between rows),
// so a column's sum runs in row order. The bounds of up to 32 rows are fetched
// at once (lane r holds row r's), and the first 32 entries of eight rows are
// loaded before any of them is added, so the dependent global loads of a
// bucket overlap instead of running one row at a time; entries past the 32nd
// of a row (the heavy rows) follow in that row's turn.
constexpr int CS_PF = 8;
// Bucket b added into the warp's zeroed accumulator row sacc (d floats).
__device__ __forceinline__ void csr_bucket_sum(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                               const float* __restrict__ val, int d, const int* __restrict__ off,
                                               const uint32_t* __restrict__ perm, int b, int lane, float* sacc) {
    const int t0 = off[b], t1 = off[b + 1];
    for (int tb = t0; tb < t1; tb += 32) {
        const int nr = min(32, t1 - tb);
        int64_t my_p0 = 0, my_p1 = 0;
        float my_sg = 0.f;
        if (lane < nr) {
            const uint32_t e = perm[tb + lane];
            const int64_t row = e & ~kSignBit;
            my_sg = (e & kSignBit) ? -1.f : 1.f;
            my_p0 = row_ptr[row];
            my_p1 = row_ptr[row + 1];
        }
        for (int r0 = 0; r0 < nr; r0 += CS_PF) {
            int cc[CS_PF];
            float vv[CS_PF];
#pragma unroll
            for (int u = 0; u < CS_PF; ++u) {                // loads of CS_PF rows in flight together
                const int r = r0 + u;
                const int64_t p0 = __shfl_sync(0xffffffffu, my_p0, r & 31);
                const int64_t p1 = __shfl_sync(0xffffffffu, my_p1, r & 31);
                cc[u] = -1;
                vv[u] = 0.f;
                if (r < nr && p0 + lane < p1) {
                    cc[u] = col[p0 + lane];
                    vv[u] = val[p0 + lane];
                }
            }
#pragma unroll
            for (int u = 0; u < CS_PF; ++u) {                // rows added in order
                const int r = r0 + u;
                const int64_t p0 = __shfl_sync(0xffffffffu, my_p0, r & 31);
                const int64_t p1 = __shfl_sync(0xffffffffu, my_p1, r & 31);
                const float sg = __shfl_sync(0xffffffffu, my_sg, r & 31);
                if (r < nr) {
                    if ((unsigned)cc[u] < (unsigned)d) atomicAdd(&sacc[cc[u]], sg * vv[u]);
                    for (int64_t p = p0 + 32 + lane; p < p1; p += 32) {
                        const int c = col[p];
                        if ((unsigned)c < (unsigned)d) atomicAdd(&sacc[c], sg * val[p]);
                    }
                }
                __syncwarp();
            }
        }
    }
}

__global__ void __launch_bounds__(128) k_countsketch_csr(
        const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
        const float* __restrict__ val, int d, const int* __restrict__ off,
        const uint32_t* __restrict__ perm, int s, float* __restrict__ B) {
    extern __shared__ float sacc_all[];
    const int wib = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    float* sacc = sacc_all + (int64_t)wib * d;
    const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * (int64_t)blockDim.x) >> 5);
    for (int b = warp; b < s; b += nwarps) {
        for (int c = lane; c < d; c += 32) sacc[c] = 0.f;
        __syncwarp();
        csr_bucket_sum(row_ptr, col, val, d, off, perm, b, lane, sacc);
        float* out = B + (int64_t)b * d;
        for (int c = lane; c < d; c += 32) out[c] = sacc[c];
        __syncwarp();
    }
}


// G (m x s) by counter into an image with leading dimension ld (columns s..ld are 0). G[j, b] =
// N_{j s + b} / sqrt(m), N the Box-Muller draw of stream 2 evaluated in FP32 (box_muller_f32: a
// few FP32 ulp of the FP64 draw). Images: g32 with form 0, fl32(N / sqrt(m)) (the FP32 SIMT
// stage); g32 with form 1, the TF32 rounding (nearest, ties away) of N, unscaled; ghi (form 2), the
// BF16 pair hi = bf16(N), lo = bf16(N - hi) at ghi and ghi + m ld, unscaled (hi + lo carries N
// to about 2^-17 of itself). The unscaled images leave 1 / sqrt(m) to the Gaussian stage's
// reduction.
__global__ void k_gen_gaussian(int64_t m, int64_t s, int64_t ld, uint64_t key, float scale, float* g32,
                               int form, __nv_bfloat16* ghi) {
    const int64_t total = m * ld;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; i < total; i += stride) {
        const int64_t j = i / ld, b = i % ld;
        const float gf = b < s ? box_muller_f32(key, (uint64_t)(j * s + b)) : 0.0f;   // draw j*s + b
        if (form == 0) {
            g32[i] = gf * scale;
        } else if (form == 1) {
            uint32_t t;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(gf));
            g32[i] = __uint_as_float(t);
        } else {
            const __nv_bfloat16 hi = __float2bfloat16_rn(gf);
            ghi[i] = hi;
            ghi[total + i] = __float2bfloat16_rn(gf - __bfloat162float(hi));
        }
    }
}

// ---------------------------------------------------------------------------
// FP32 SIMT split-K GEMM: P[z] (M x N) = G[:, kz] (M x Kz) * B[kz, :] (Kz x N).
// 128x128 tile, BK = 8, 256 threads, 8x8 outputs per thread, two smem stages.
// ---------------------------------------------------------------------------
constexpr int SG_BM = 128, SG_BN = 128, SG_BK = 8;

__global__ void __launch_bounds__(256) k_sgemm_splitk(
        const float* __restrict__ G, const float* __restrict__ B, int M, int N, int64_t K,
        int64_t kchunk, float* __restrict__ P) {
    __shared__ __align__(16) float As[2][SG_BK][SG_BM];
    __shared__ __align__(16) float Bs[2][SG_BK][SG_BN];
    const int t = threadIdx.x;
    const int m0 = blockIdx.y * SG_BM, n0 = blockIdx.x * SG_BN;
    const int64_t kb = (int64_t)blockIdx.z * kchunk;
    const int64_t ke = min(K, kb + kchunk);
    // loader coordinates
    const int a_row = t >> 1, a_k = (t & 1) * 4;
    const int b_k = t >> 5, b_col = (t & 31) * 4;
    const int ty = t >> 4, tx = t & 15;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    float ra[4], rb[4];
    auto load_regs = [&](int64_t k0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t kk = k0 + a_k + i;
            const int row = m0 + a_row;
            ra[i] = (row < M && kk < ke) ? __ldg(G + (int64_t)row * K + kk) : 0.f;
        }
        const int64_t kr = k0 + b_k;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int c = n0 + b_col + i;
            rb[i] = (kr < ke && c < N) ? __ldg(B + kr * N + c) : 0.f;
        }
    };
    auto store_smem = [&](int st) {
#pragma unroll
        for (int i = 0; i < 4; ++i) As[st][a_k + i][a_row] = ra[i];
        *reinterpret_cast<float4*>(&Bs[st][b_k][b_col]) = make_float4(rb[0], rb[1], rb[2], rb[3]);
    };

    int st = 0;
    if (kb < ke) {
        load_regs(kb);
        store_smem(0);
    }
    __syncthreads();
    for (int64_t k0 = kb; k0 < ke; k0 += SG_BK) {
        const bool more = (k0 + SG_BK) < ke;
        if (more) load_regs(k0 + SG_BK);
#pragma unroll
        for (int kk = 0; kk < SG_BK; ++kk) {
            float a[8], b[8];
            const float4 a0 = *reinterpret_cast<const float4*>(&As[st][kk][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[st][kk][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[st][kk][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[st][kk][64 + tx * 4]);
            a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
            a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
            b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w;
            b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[7] = b1.w;
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        if (more) {
            store_smem(st ^ 1);
            __syncthreads();
            st ^= 1;
        }
    }
    float* out = P + (int64_t)blockIdx.z * M * N;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int row = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
        if (row >= M) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
            if (c < N) out[(int64_t)row * N + c] = acc[i][j];
        }
    }
}

__global__ void k_reduce_splits(const float* __restrict__ P, int splits, int64_t count,
                                float* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; i < count; i += stride) {
        float acc = 0.f;
        for (int z = 0; z < splits; ++z) acc += P[(int64_t)z * count + i];
        out[i] = acc;
    }
}

__global__ void k_copy_dense(const float* __restrict__ A, int64_t lda, int64_t n, int d,
                             float* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; i < n * d; i += stride) out[i] = A[(i / d) * lda + (i % d)];
}

int grid_for(int64_t work, int block, int cap = 1 << 20) {
    int64_t g = (work + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

template <int NC, int U>
cudaError_t launch_op(const float* A, int64_t lda, int d, int s, int64_t ld, const int* off, const uint32_t* perm,
                      __nv_bfloat16* hi, __nv_bfloat16* lo, cudaStream_t st) {
    const size_t smem = sizeof(float) * 16 * (size_t)d;
    // one octet a CTA: the block scheduler balances the buckets' lengths (a grid-stride loop over
    // fewer CTAs left a tail of about 15%)
    const int64_t noct = ld / 8;
    const int grid = (int)noct;
    cudaError_t e;
    if (lo) {
        if ((e = cudaFuncSetAttribute(k_countsketch_dense_op<NC, U, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem)) != cudaSuccess)
            return e;
        k_countsketch_dense_op<NC, U, true><<<grid, 256, smem, st>>>(A, lda, d, off, perm, s, ld, hi, lo);
    } else {
        if ((e = cudaFuncSetAttribute(k_countsketch_dense_op<NC, U, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem)) != cudaSuccess)
            return e;
        k_countsketch_dense_op<NC, U, false><<<grid, 256, smem, st>>>(A, lda, d, off, perm, s, ld, hi, lo);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_scan_offsets(const int* count, int* off, int64_t s, cudaStream_t st) {
    k_scan_offsets<<<1, 1024, 0, st>>>(count, off, (int)s);
    return cudaGetLastError();
}

cudaError_t launch_segment_sort(const int* off, int64_t s, const uint32_t* in, uint32_t* out, cudaStream_t st) {
    k_segment_sort<<<grid_for(s * 32, 256), 256, 0, st>>>(off, (int)s, in, out);
    return cudaGetLastError();
}

cudaError_t launch_bucket_perm(int64_t n, int64_t s, uint64_t seed, int64_t row0, int* count, int* off,
                               uint32_t* tmp, uint32_t* perm, cudaStream_t st) {
    const uint64_t key = stream_key(seed, kStreamHash);
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int) * (size_t)(s + 1), st);
    if (e != cudaSuccess) return e;
    k_bucket_hist<<<grid_for(n, 256, 152 * 16), 256, 0, st>>>(n, row0, (uint32_t)s, key, count);
    k_scan_offsets<<<1, 1024, 0, st>>>(count, off, (int)s);
    e = cudaMemsetAsync(count, 0, sizeof(int) * (size_t)(s + 1), st);
    if (e != cudaSuccess) return e;
    k_bucket_scatter<<<grid_for(n, 256, 152 * 16), 256, 0, st>>>(n, row0, (uint32_t)s, key, off, count, tmp);
    k_segment_sort<<<grid_for(s * 32, 256), 256, 0, st>>>(off, (int)s, tmp, perm);
    return cudaGetLastError();
}

cudaError_t launch_countsketch_dense(const float* A, int64_t lda, int64_t d, int64_t s,
                                     const int* off, const uint32_t* perm, float* B, cudaStream_t st) {
    const bool vec = (reinterpret_cast<uintptr_t>(A) % 16 == 0) && (lda % 4 == 0) && (d % 4 == 0);
    const int grid = grid_for(s * 32, 256);
    if (vec && d <= 128) {
        k_countsketch_dense_v4<1, 8><<<grid, 256, 0, st>>>(A, lda, (int)d, off, perm, (int)s, B);
    } else if (vec && d <= 256) {
        k_countsketch_dense_v4<2, 4><<<grid, 256, 0, st>>>(A, lda, (int)d, off, perm, (int)s, B);
    } else if (vec && d <= 512) {
        k_countsketch_dense_v4<4, 2><<<grid, 256, 0, st>>>(A, lda, (int)d, off, perm, (int)s, B);
    } else if (vec && d <= 1024) {
        k_countsketch_dense_v4<8, 1><<<grid, 256, 0, st>>>(A, lda, (int)d, off, perm, (int)s, B);
    } else {
        k_countsketch_dense_scalar<<<grid, 256, 0, st>>>(A, lda, (int)d, off, perm, (int)s, B);
    }
    return cudaGetLastError();
}

cudaError_t launch_countsketch_dense_op(const float* A, int64_t lda, int64_t d, int64_t s, int64_t ld,
                                        const int* off, const uint32_t* perm, __nv_bfloat16* hi, __nv_bfloat16* lo,
                                        cudaStream_t st) {
    const bool vec = (reinterpret_cast<uintptr_t>(A) % 16 == 0) && (lda % 4 == 0) && (d % 4 == 0);
    if (!vec || d < 4 || d > 1024 || ld % 64 != 0 || ld < s || (reinterpret_cast<uintptr_t>(hi) % 16) != 0 ||
        (lo && reinterpret_cast<uintptr_t>(lo) % 16 != 0))
        return cudaErrorNotSupported;
    if (d <= 128) return launch_op<1, 8>(A, lda, (int)d, (int)s, ld, off, perm, hi, lo, st);
    if (d <= 256) return launch_op<2, 4>(A, lda, (int)d, (int)s, ld, off, perm, hi, lo, st);
    if (d <= 512) return launch_op<4, 2>(A, lda, (int)d, (int)s, ld, off, perm, hi, lo, st);
    return launch_op<8, 1>(A, lda, (int)d, (int)s, ld, off, perm, hi, lo, st);
}


cudaError_t launch_countsketch_csr(const int64_t* row_ptr, const int32_t* col, const float* val,
                                   int64_t d, int64_t s, const int* off, const uint32_t* perm,
                                   float* B, cudaStream_t st) {
    const int warps = 4;
    const size_t smem = sizeof(float) * (size_t)d * warps;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_countsketch_csr,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_countsketch_csr<<<grid_for(s * 32, 32 * warps), 32 * warps, smem, st>>>(
        row_ptr, col, val, (int)d, off, perm, (int)s, B);
    return cudaGetLastError();
}

cudaError_t launch_gen_gaussian(int64_t m, int64_t s, int64_t ld, uint64_t seed, float* g32, int form,
                                __nv_bfloat16* ghi, cudaStream_t st) {
    const float scale = (float)(1.0 / sqrt((double)m));
    k_gen_gaussian<<<grid_for(m * ld, 256, 152 * 32), 256, 0, st>>>(
        m, s, ld, stream_key(seed, kStreamG), scale, g32, form, ghi);
    return cudaGetLastError();
}

int gaussian_stage_splits(int64_t m, int64_t d, int64_t s) {
    const int64_t tiles = ((m + SG_BM - 1) / SG_BM) * ((d + SG_BN - 1) / SG_BN);
    int64_t splits = (152 * 4 + tiles - 1) / tiles;          // about 4 CTAs per SM
    const int64_t max_by_k = (s + 255) / 256;                 // at least 256 k per split
    if (splits > max_by_k) splits = max_by_k;
    if (splits < 1) splits = 1;
    return (int)splits;
}

cudaError_t launch_gaussian_stage_fp32(const float* G, const float* B, int64_t m, int64_t s,
                                       int64_t d, float* partial, int splits, float* Atilde,
                                       cudaStream_t st) {
    int64_t kchunk = (s + splits - 1) / splits;
    kchunk = (kchunk + SG_BK - 1) / SG_BK * SG_BK;
    dim3 grid((unsigned)((d + SG_BN - 1) / SG_BN), (unsigned)((m + SG_BM - 1) / SG_BM), (unsigned)splits);
    k_sgemm_splitk<<<grid, 256, 0, st>>>(G, B, (int)m, (int)d, s, kchunk, partial);
    k_reduce_splits<<<grid_for(m * d, 256, 152 * 8), 256, 0, st>>>(partial, splits, m * d, Atilde);
    return cudaGetLastError();
}

// The CSR structure of the input contract: bad |= 1 if row_ptr[0] != 0, 2 if row_ptr decreases
// somewhere, 4 if row_ptr[n] != nnz. Reads row_ptr[0..n] only.
__global__ void k_check_csr(const int64_t* __restrict__ rp, int64_t n, int64_t nnz, int32_t* bad) {
    int flags = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = rp[i];
        if (i == 0 && a != 0) flags |= 1;
        if (i < n && rp[i + 1] < a) flags |= 2;
        if (i == n && a != nnz) flags |= 4;
    }
    if (flags) atomicOr(bad, flags);
}

cudaError_t launch_check_csr(const int64_t* row_ptr, int64_t n, int64_t nnz, int32_t* bad, cudaStream_t st) {
    k_check_csr<<<grid_for(n + 1, 256, 152 * 8), 256, 0, st>>>(row_ptr, n, nnz, bad);
    return cudaGetLastError();
}

cudaError_t launch_copy_dense(const float* A, int64_t lda, int64_t n, int64_t d, float* out,
                              cudaStream_t st) {
    k_copy_dense<<<grid_for(n * d, 256, 152 * 8), 256, 0, st>>>(A, lda, n, (int)d, out);
    return cudaGetLastError();
}

}  // namespace lev
