// Tensor-core (tcgen05, sm_103a) Gaussian stage of the CountGauss sketch
// (Alg. 3 step 3): A~ (m x d) = G (m x s) B (s x d), a long-K GEMM.
//
// CTA pairs (cta_group::2) with split-K over the grid: a pair covers 256 rows of G (128 in each
// CTA) and a tile of up to 256 columns of B (each CTA holds half of the tile's rows of B^T), so
// every CTA loads 128 rows of G and only half of the B tile per K block. One thread of the even
// CTA issues M = 256 MMAs for the pair; each CTA's TMEM receives its own 128 rows of the
// accumulator with all the tile's columns. The pair accumulates its 256 x NT block over its slice
// of s and writes the FP32 partial (row-major, one slice after another); a second kernel adds the
// partials of the slices in a fixed order. Operands are K-major: rows of G, and rows of B^T. For
// the BF16 forms B^T is blocked by K block (K block g of rows c.. is a run of 128-byte rows at row
// g d + c), written by the dense CountSketch itself or by k_transpose_blocked from the FP32 B; for
// TF32 it is d x ld from k_transpose_operand. Both are loaded by 2-D tensor TMA with the 128-byte
// swizzle into a ring of stages:
//   warp 0: TMA producer (one thread); warp 1: TMEM allocation, and in the even CTA the MMA issuer
//   (one thread), in the odd CTA the relay that reports each landed stage to the even CTA;
//   warps 2..5: epilogue (tcgen05.ld, partial stores).
// G = N / sqrt(m) with N the FP32 rounding of the counter draws; the MMAs take N and the reduction
// applies 1 / sqrt(m). Forms: BF16 (N and B rounded to BF16, one MMA per K step), BF16X3 (N and B
// split into BF16 hi + lo: N_hi B_hi + N_lo B_hi + N_hi B_lo, three MMAs), TF32 (N and B rounded to
// TF32).
#include <atomic>
#include <cuda.h>
#include <cuda_bf16.h>

#include "lev_common.cuh"
#include "lev_kernels.cuh"
#include "lev_tc.cuh"
#include "tc_common.cuh"

namespace lev {

namespace {

using namespace tcx;

enum GForm { gBF16 = 0, gBF16X3 = 1, gTF32 = 2 };

template <int F>
struct GTraits;
template <>
struct GTraits<gBF16> {
    static constexpr bool kTf32 = false, kSplit = false;
    static constexpr int kElem = 2, kKbe = 64;
};
template <>
struct GTraits<gBF16X3> {
    static constexpr bool kTf32 = false, kSplit = true;
    static constexpr int kElem = 2, kKbe = 64;
};
template <>
struct GTraits<gTF32> {
    static constexpr bool kTf32 = true, kSplit = false;
    static constexpr int kElem = 4, kKbe = 32;
};

constexpr int kRowsM = 128;                   // rows of G per CTA (TMEM lanes)
constexpr int kMaxNt = 256;                   // MMA N: columns of the accumulator tile
constexpr int kMaxStages = 6;
constexpr int kMaxSliceKb = 54;               // K blocks in one accumulation chain (3,456 BF16 / 1,728 TF32 products)
constexpr int kStageBudget = 200 * 1024;      // shared memory for the ring of stages
constexpr uint64_t kWaitNs = 2000000000ull;
constexpr uint64_t kExitWaitNs = 5000000000ull;
constexpr int32_t kStatusGaussTimeout = 4;

struct GCtl {
    uint64_t full[kMaxStages], empty[kMaxStages], tfull, mdone, xbar;
    uint32_t tmem_base;
    int32_t abort;
};

// Bounded wait on an mbarrier phase (acquire at cluster scope); false if this CTA gave up.
__device__ __forceinline__ bool gwait(uint32_t bar, uint32_t parity, GCtl* ctl, int32_t* status) {
    if (mbar_try_wait_cluster(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait_cluster(bar, parity)) return true;
        if ((it & 63u) == 0) {
            if (*(volatile int32_t*)&ctl->abort) return false;
            if (global_ns() - t0 > kWaitNs) {
                *(volatile int32_t*)&ctl->abort = 1;
                atomicExch(status, kStatusGaussTimeout);
                return false;
            }
        }
    }
}

// Bounded wait that an abort does not cut short (copies, MMAs and arrivals still in flight).
__device__ __forceinline__ bool gdrain(uint32_t bar, uint32_t parity, uint64_t limit_ns, int32_t* status) {
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait_cluster(bar, parity)) {
        if (global_ns() - t0 > limit_ns) {
            atomicExch(status, kStatusGaussTimeout);
            return false;
        }
    }
    return true;
}

// Grid: x = 2 * (pair tile * n_tiles + n tile) + CTA rank in the pair (clusters of 2 along x),
// y = K slice. Partial P[z][i][c] (i < m, c < d), row-major per slice.
template <int F>
__global__ void __launch_bounds__(192, 1) k_gauss_tc(const __grid_constant__ CUtensorMap tmG,
                                                     const __grid_constant__ CUtensorMap tmGlo,
                                                     const __grid_constant__ CUtensorMap tmB,
                                                     const __grid_constant__ CUtensorMap tmBlo, int m, int d, int nt,
                                                     int n_tiles, int stages, int kb_per_slice, int kb_total,
                                                     int bd, float* __restrict__ P, int32_t* status) {
    using T = GTraits<F>;
    constexpr int NOPS = T::kSplit ? 2 : 1;               // hi (and lo) images of each operand
    const int A_BYTES = kRowsM * 128;                     // one image of this CTA's rows of G
    const int B_BYTES = (nt / 2) * 128;                   // one image of this CTA's half of the B tile
    const int STAGE_BYTES = NOPS * (A_BYTES + B_BYTES);   // [G hi][G lo][B hi][B lo]
    const uint32_t idesc = make_idesc(T::kTf32, 2 * kRowsM, nt);
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
    uint8_t* base = smem_raw + pad;
    GCtl* ctl = reinterpret_cast<GCtl*>(base + stages * STAGE_BYTES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t me = cluster_ctarank();
    const int unit = blockIdx.x >> 1;
    const int pt = unit / n_tiles, ntile = unit % n_tiles;
    const int kb0 = blockIdx.y * kb_per_slice;
    const int kb1 = min(kb_total, kb0 + kb_per_slice);
    const int nkb = max(0, kb1 - kb0);

    if (threadIdx.x == 0) {
        for (int q = 0; q < stages; ++q) {
            // the even CTA's full barrier also takes the odd CTA's "landed" report
            mbar_init(smem_u32(&ctl->full[q]), me == 0 ? 2 : 1);
            mbar_init(smem_u32(&ctl->empty[q]), 1);
        }
        mbar_init(smem_u32(&ctl->tfull), 1);
        mbar_init(smem_u32(&ctl->mdone), 1);
        mbar_init(smem_u32(&ctl->xbar), 2);
        ctl->abort = 0;
        fence_mbar_init();
    }
    __syncthreads();
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    if (warp == 1) {
        tmem_alloc_cg<2>(smem_u32(&ctl->tmem_base), 256);
        tmem_relinquish_cg<2>();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = ctl->tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            int q = 0;
            uint32_t phase = 0;
            int issued = 0;
            const int32_t yg = pt * 2 * kRowsM + (int32_t)me * kRowsM;
            const int32_t yb = ntile * nt + (int32_t)me * (nt / 2);
            for (int i = 0; i < nkb; ++i) {
                if (!gwait(smem_u32(&ctl->empty[q]), phase ^ 1u, ctl, status)) break;
                const uint32_t sb = smem_u32(base + q * STAGE_BYTES);
                const uint32_t bar = smem_u32(&ctl->full[q]);
                mbar_arrive_expect_tx(bar, (uint32_t)STAGE_BYTES);
                const int x = (kb0 + i) * T::kKbe;
                // B^T rows yb.. of K block kb0 + i: plain (d x ld) or blocked by K block (rows of
                // 64 elements, block kb at rows kb d..; a box that runs past d takes rows of the next
                // block, which only reach accumulator columns >= d, never stored)
                const int xb = bd ? 0 : x, ybk = bd ? (kb0 + i) * bd + yb : yb;
                tma_load_2d(sb, &tmG, x, yg, bar);
                if constexpr (T::kSplit) tma_load_2d(sb + A_BYTES, &tmGlo, x, yg, bar);
                tma_load_2d(sb + NOPS * A_BYTES, &tmB, xb, ybk, bar);
                if constexpr (T::kSplit) tma_load_2d(sb + NOPS * A_BYTES + B_BYTES, &tmBlo, xb, ybk, bar);
                ++issued;
                if (++q == stages) { q = 0; phase ^= 1u; }
            }
            // no copy may still be landing in this CTA's shared memory when it exits
            for (int j = issued > stages ? issued - stages : 0; j < issued; ++j)
                gdrain(smem_u32(&ctl->full[j % stages]), (uint32_t)((j / stages) & 1), kWaitNs, status);
            // and every MMA that reads it has finished (the "stage free" commits, multicast to the
            // pair, have landed here)
            if (issued == nkb && !*(volatile int32_t*)&ctl->abort) {
                for (int u = 0; u < stages; ++u) {
                    const int k_uses = nkb / stages + (u < nkb % stages ? 1 : 0);
                    if (k_uses > 0) gdrain(smem_u32(&ctl->empty[u]), (uint32_t)((k_uses - 1) & 1), kWaitNs, status);
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0 && me != 0) {
            // odd CTA: report each landed stage to the even CTA, whose MMAs read this CTA's half. The
            // stage's bytes were written by TMA and are read by the MMAs (both the async proxy) and
            // this thread has seen them land, so the report is a relaxed arrival (a cluster-scope
            // release arrive costs about a microsecond under load)
            int q = 0;
            uint32_t phase = 0;
            for (int i = 0; i < nkb; ++i) {
                if (!gwait(smem_u32(&ctl->full[q]), phase, ctl, status)) break;
                mbar_arrive_relaxed_cluster(mapa_shared(smem_u32(&ctl->full[q]), 0));
                if (++q == stages) { q = 0; phase ^= 1u; }
            }
        } else if (lane == 0) {
            int q = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int i = 0; i < nkb; ++i) {
                if (!gwait(smem_u32(&ctl->full[q]), phase, ctl, status)) { ok = false; break; }
                tc_fence_after();
                const uint32_t sb = smem_u32(base + q * STAGE_BYTES);
                const uint32_t ghi = sb, glo = sb + A_BYTES;
                const uint32_t bhi = sb + NOPS * A_BYTES, blo = bhi + B_BYTES;
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                    const uint32_t ko = (uint32_t)ks * 32u;
                    const uint32_t acc = (i | ks) != 0 ? 1u : 0u;
                    if constexpr (T::kSplit) {
                        tc_mma_cg<2, false>(tmem, sw128_desc(glo + ko), sw128_desc(bhi + ko), idesc, acc);
                        tc_mma_cg<2, false>(tmem, sw128_desc(ghi + ko), sw128_desc(blo + ko), idesc, 1u);
                        tc_mma_cg<2, false>(tmem, sw128_desc(ghi + ko), sw128_desc(bhi + ko), idesc, 1u);
                    } else {
                        tc_mma_cg<2, T::kTf32>(tmem, sw128_desc(ghi + ko), sw128_desc(bhi + ko), idesc, acc);
                    }
                }
                // stage q is free again in both CTAs once these MMAs finish
                tc_commit_mc<2>(smem_u32(&ctl->empty[q]), (uint16_t)0x3);
                if (++q == stages) { q = 0; phase ^= 1u; }
            }
            if (ok && nkb > 0) tc_commit_mc<2>(smem_u32(&ctl->tfull), (uint16_t)0x3);
            // every MMA has finished before TMEM is freed
            tc_commit_mc<2>(smem_u32(&ctl->mdone), (uint16_t)0x1);
            gdrain(smem_u32(&ctl->mdone), 0, kWaitNs, status);
        }
        __syncwarp();
    } else {
        // epilogue: warps 2..5 cover TMEM lane groups (warp % 4); TMEM lane = row of this CTA
        const int lg = warp & 3;
        const int row = pt * 2 * kRowsM + (int)me * kRowsM + lg * 32 + lane;
        float* out = P + (int64_t)blockIdx.y * m * d + (int64_t)row * d;
        const bool vec = (d & 3) == 0;
        if (nkb == 0) {
            if (row < m)
                for (int c = 0; c < nt; ++c) {
                    const int col = ntile * nt + c;
                    if (col < d) out[col] = 0.f;
                }
        } else if (gwait(smem_u32(&ctl->tfull), 0, ctl, status)) {
            tc_fence_after();
            for (int c0 = 0; c0 < nt; c0 += 32) {
                uint32_t r[32];
                tmem_ld32(tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)c0, r);
                tmem_ld_wait();
                const int col0 = ntile * nt + c0;
                if (row >= m) continue;
                if (vec && col0 + 32 <= d) {
#pragma unroll
                    for (int j = 0; j < 32; j += 4)
                        *reinterpret_cast<float4*>(out + col0 + j) =
                            make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]), __uint_as_float(r[j + 2]),
                                        __uint_as_float(r[j + 3]));
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (col0 + j < d) out[col0 + j] = __uint_as_float(r[j]);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc_cg<2>(tmem, 256);
    }
    // neither CTA leaves while its peer may still signal its mbarriers or read its shared memory
    if (threadIdx.x == 0) {
        const uint32_t xb = smem_u32(&ctl->xbar);
        mbar_arrive_cluster(xb);
        mbar_arrive_cluster(mapa_shared(xb, me ^ 1u));
        gdrain(xb, 0, kExitWaitNs, status);
    }
    __syncthreads();
}

// A~ = scale * (sum of the K-slice partials, in slice order); scale = 1 / sqrt(m) (G = N / sqrt(m)).
// Partials and A~ are row-major m x d.
__global__ void k_gauss_reduce(const float* __restrict__ P, int splits, int m, int d, float scale,
                               float* __restrict__ At) {
    const int64_t total = (int64_t)m * d;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        float acc = 0.f;
        for (int z = 0; z < splits; ++z) acc += P[(int64_t)z * total + e];
        At[e] = acc * scale;
    }
}

// B (s x d FP32 row-major) -> B^T (d x ld) in the operand type; columns s..ld zero. Tiles of 64 k
// x 32 columns: a warp reads 32 consecutive floats of a row of B, and writes two consecutive k of
// one column per lane (a BF16 pair, or two TF32 words), so both sides move whole 128-byte lines.
template <int F>
__global__ void k_transpose_operand(const float* __restrict__ B, int64_t s, int d, int64_t ld, void* __restrict__ hi,
                                    void* __restrict__ lo) {
    using T = GTraits<F>;
    __shared__ float tile[64][33];
    const int64_t k0 = (int64_t)blockIdx.x * 64;
    const int c0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;     // 32 x 8
    for (int yy = ty; yy < 64; yy += 8) {
        const int64_t k = k0 + yy;
        const int c = c0 + tx;
        tile[yy][tx] = (k < s && c < d) ? B[k * d + c] : 0.f;
    }
    __syncthreads();
    const int64_t k = k0 + 2 * tx;                               // even; ld is a multiple of 64
    if (k >= ld) return;
    for (int cc = ty; cc < 32; cc += 8) {
        const int c = c0 + cc;
        if (c >= d) continue;
        const float x0 = tile[2 * tx][cc], x1 = tile[2 * tx + 1][cc];
        const int64_t o = (int64_t)c * ld + k;
        if constexpr (T::kTf32) {
            reinterpret_cast<uint2*>(static_cast<uint32_t*>(hi) + o)[0] = make_uint2(f32_to_tf32(x0), f32_to_tf32(x1));
        } else {
            const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
            reinterpret_cast<__nv_bfloat162*>(static_cast<__nv_bfloat16*>(hi) + o)[0] = h;
            if constexpr (T::kSplit) {
                const float2 hf = __bfloat1622float2(h);
                reinterpret_cast<__nv_bfloat162*>(static_cast<__nv_bfloat16*>(lo) + o)[0] =
                    __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
            }
        }
    }
}

// B (s x d FP32 row-major) -> the blocked K-major BF16 operand img[g][c][k] = B[64 g + k][c]
// (rows s..ld zero): hi, and lo = bf16(x - hi) when SPLIT, rounded pairwise as above. A tile is one
// K block g by 64 columns, whose image rows are 64 consecutive 128-byte rows: read as 16-byte
// pieces of rows of B, written as 8 KB runs per image (four threads a 128-byte row).
template <bool SPLIT>
__global__ void __launch_bounds__(256) k_transpose_blocked(const float* __restrict__ B, int64_t s, int d,
                                                           __nv_bfloat16* __restrict__ hi,
                                                           __nv_bfloat16* __restrict__ lo) {
    __shared__ float tile[64][65];
    const int g = blockIdx.x, c0 = blockIdx.y * 64;
    const int64_t k0 = (int64_t)g * 64;
    const bool vec = (d & 3) == 0;                               // rows of B start on 16-byte boundaries
    const int cq = (threadIdx.x & 15) * 4;
    for (int r = threadIdx.x >> 4; r < 64; r += 16) {
        const int64_t k = k0 + r;
        const int c = c0 + cq;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (k < s) {
            const float* row = B + k * d;
            if (vec && c < d) {
                v = *reinterpret_cast<const float4*>(row + c);
            } else {
                v.x = c < d ? row[c] : 0.f;
                v.y = c + 1 < d ? row[c + 1] : 0.f;
                v.z = c + 2 < d ? row[c + 2] : 0.f;
                v.w = c + 3 < d ? row[c + 3] : 0.f;
            }
        }
        tile[r][cq] = v.x;
        tile[r][cq + 1] = v.y;
        tile[r][cq + 2] = v.z;
        tile[r][cq + 3] = v.w;
    }
    __syncthreads();
    const int cc = threadIdx.x >> 2, q = threadIdx.x & 3;         // column, quarter of the K block
    const int c = c0 + cc;
    if (c >= d) return;
    uint32_t hw[8], lw[8];
#pragma unroll
    for (int p = 0; p < 8; ++p) {
        const float x0 = tile[q * 16 + 2 * p][cc], x1 = tile[q * 16 + 2 * p + 1][cc];
        const __nv_bfloat162 h2 = __floats2bfloat162_rn(x0, x1);
        hw[p] = *reinterpret_cast<const uint32_t*>(&h2);
        if constexpr (SPLIT) {
            const float2 hf = __bfloat1622float2(h2);
            const __nv_bfloat162 l2 = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
            lw[p] = *reinterpret_cast<const uint32_t*>(&l2);
        }
    }
    const int64_t at = ((int64_t)g * d + c) * 64 + q * 16;
    uint4* dh = reinterpret_cast<uint4*>(hi + at);
    dh[0] = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    dh[1] = make_uint4(hw[4], hw[5], hw[6], hw[7]);
    if constexpr (SPLIT) {
        uint4* dl = reinterpret_cast<uint4*>(lo + at);
        dl[0] = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        dl[1] = make_uint4(lw[4], lw[5], lw[6], lw[7]);
    }
}

// Row-major matrix rows x cols (elements) with leading dimension ld, box (box_cols x box_rows).
bool make_map(CUtensorMap* map, const void* ptr, bool tf32, int64_t rows, int64_t cols, int64_t ld, int box_cols,
              int box_rows) {
    return make_map_2d(map, ptr, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, tf32 ? 4 : 2,
                       rows, cols, ld, box_cols, box_rows);
}

// Resident 2-CTA clusters of k_gauss_tc<F> with `smem` bytes each, per device (cached; host threads
// share it).
template <int F>
int resident_pairs(size_t smem, cudaLaunchConfig_t cfg, int sms) {
    static std::atomic<int> cached[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    int pairs = dev >= 0 && dev < 64 ? cached[dev].load(std::memory_order_relaxed) : 0;
    if (pairs > 0) return pairs;
    cfg.gridDim = dim3((unsigned)(sms & ~1));
    cfg.dynamicSmemBytes = smem;
    if (cudaOccupancyMaxActiveClusters(&pairs, k_gauss_tc<F>, &cfg) != cudaSuccess || pairs < 1) {
        cudaGetLastError();
        return -1;
    }
    if (dev >= 0 && dev < 64) cached[dev].store(pairs, std::memory_order_relaxed);
    return pairs;
}

// B == nullptr: the operand is already in scratch slot 2, blocked by K block (tc_gaussian_operand);
// otherwise it is made here from the FP32 B.
template <int F>
int run_gauss_tc(lev_handle* h, const float* B, int64_t m, int64_t s, int64_t d, uint64_t seed, float* Atilde,
                 cudaStream_t st) {
    using T = GTraits<F>;
    const int64_t ld = (s + 63) / 64 * 64;                // padded K: 16-byte row strides, whole 128-byte rows
    // G image (cached in the handle): kind 2 = the BF16 pair of N (ld), kind 3 = N rounded to TF32 (ld)
    const float* g32 = nullptr;
    const __nv_bfloat16* ghi = nullptr;
    int rc = handle_gaussian(h, m, s, seed, T::kTf32 ? 3 : 2, st, &g32, &ghi);
    if (rc != LEV_OK) return rc;
    // B^T in the operand type
    const size_t bt_elems = (size_t)d * ld;
    void* bt = nullptr;
    rc = handle_scratch(h, 2, bt_elems * T::kElem * (T::kSplit ? 2 : 1), &bt);
    if (rc != LEV_OK) return rc;
    void* bt_lo = T::kSplit ? static_cast<void*>(static_cast<uint8_t*>(bt) + bt_elems * T::kElem) : nullptr;
    // BF16 forms: B^T blocked by K block (written by the CountSketch, B == nullptr, or here); TF32:
    // plain d x ld
    const bool blocked = !T::kTf32;
    if (!B && !blocked) return handle_fail(LEV_EINVAL, "blocked operand needs a BF16 form");
    if (B && blocked) {
        dim3 tg((unsigned)(ld / 64), (unsigned)((d + 63) / 64));
        k_transpose_blocked<T::kSplit><<<tg, 256, 0, st>>>(B, s, (int)d, static_cast<__nv_bfloat16*>(bt),
                                                           static_cast<__nv_bfloat16*>(bt_lo));
    } else if (B) {
        dim3 tg((unsigned)((ld + 63) / 64), (unsigned)((d + 31) / 32));
        k_transpose_operand<F><<<tg, 256, 0, st>>>(B, s, (int)d, ld, bt, bt_lo);
    }
    // tiles: a pair covers 256 rows of G and nt columns of B (nt a multiple of 16, each CTA nt / 2)
    const int nt_full = (int)std::min<int64_t>(kMaxNt, (d + 15) / 16 * 16);
    const int n_tiles = (int)((d + nt_full - 1) / nt_full);
    const int nt = (int)(((d + n_tiles - 1) / n_tiles + 15) / 16 * 16);
    const int pair_tiles = (int)((m + 2 * kRowsM - 1) / (2 * kRowsM));
    const int kb_total = (int)(ld / T::kKbe);
    const int nops = T::kSplit ? 2 : 1;
    const int stage_bytes = nops * (kRowsM * 128 + (nt / 2) * 128);
    const int stages = std::min(kMaxStages, kStageBudget / stage_bytes);
    const size_t smem = 1024 + (size_t)stages * stage_bytes + sizeof(GCtl) + 64;
    cudaError_t e = cudaFuncSetAttribute(k_gauss_tc<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return handle_fail(LEV_ECUDA, cudaGetErrorString(e));
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(192);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const int pairs = resident_pairs<F>(smem, cfg, handle_num_sms(h));
    if (pairs < 1) return handle_fail(LEV_ECUDA, "no resident 2-CTA cluster for the Gaussian stage");
    // K slices: the count z that minimises (waves of pairs) x (K blocks a slice + a fixed cost of
    // about six K blocks for the pipeline fill and the epilogue), among the counts that keep a slice
    // at most kMaxSliceKb K blocks long: each slice is one accumulation chain in TMEM, whose error
    // grows with its length, and the partials of the slices are summed apart in a fixed order
    const int64_t units = (int64_t)pair_tiles * n_tiles;
    const int z_min = (int)std::min<int64_t>(kb_total, (kb_total + kMaxSliceKb - 1) / kMaxSliceKb);
    int splits = z_min;
    int64_t best = -1;
    for (int z = z_min; z <= std::min(kb_total, std::max(256, z_min)); ++z) {
        const int64_t per = (kb_total + z - 1) / z;
        const int64_t cost = ((units * z + pairs - 1) / pairs) * (per + 6);
        if (best < 0 || cost < best) { best = cost; splits = z; }
    }
    const int kb_per_slice = (kb_total + splits - 1) / splits;
    splits = (kb_total + kb_per_slice - 1) / kb_per_slice;
    void* part = nullptr;
    rc = handle_scratch(h, 1, sizeof(float) * (size_t)splits * m * d, &part);
    if (rc != LEV_OK) return rc;
    CUtensorMap mG, mGlo, mB, mBlo;
    const void* gimg = T::kTf32 ? static_cast<const void*>(g32) : static_cast<const void*>(ghi);
    // B^T: d rows of ld, or (blocked) ld / 64 d rows of 64
    const int64_t b_rows = blocked ? (ld / 64) * d : d, b_cols = blocked ? 64 : ld;
    bool ok = make_map(&mG, gimg, T::kTf32, m, ld, ld, T::kKbe, kRowsM) &&
              make_map(&mB, bt, T::kTf32, b_rows, b_cols, b_cols, T::kKbe, nt / 2);
    if (T::kSplit)
        ok = ok && make_map(&mGlo, ghi + (size_t)m * ld, false, m, ld, ld, T::kKbe, kRowsM) &&
             make_map(&mBlo, bt_lo, false, b_rows, b_cols, b_cols, T::kKbe, nt / 2);
    else {
        mGlo = mG;
        mBlo = mB;
    }
    if (!ok) return handle_fail(LEV_ECUDA, "cuTensorMapEncodeTiled failed for the Gaussian stage");
    cfg.gridDim = dim3((unsigned)(2 * units), (unsigned)splits);
    e = cudaLaunchKernelEx(&cfg, k_gauss_tc<F>, mG, mGlo, mB, mBlo, (int)m, (int)d, nt, n_tiles, stages, kb_per_slice,
                           kb_total, blocked ? (int)d : 0, static_cast<float*>(part), handle_status(h));
    if (e != cudaSuccess) return handle_fail(LEV_ECUDA, cudaGetErrorString(e));
    k_gauss_reduce<<<152 * 4, 256, 0, st>>>(static_cast<const float*>(part), splits, (int)m, (int)d,
                                            (float)(1.0 / std::sqrt((double)m)), Atilde);
    e = cudaGetLastError();
    if (e != cudaSuccess) return handle_fail(LEV_ECUDA, cudaGetErrorString(e));
    return LEV_OK;
}

}  // namespace

int tc_gaussian_operand(lev_handle* h, int64_t s, int64_t d, int32_t prec, __nv_bfloat16** hi, __nv_bfloat16** lo,
                        int64_t* ld_out) {
    if (prec != LEV_BF16 && prec != LEV_BF16X3) return handle_fail(LEV_EINVAL, "blocked operand needs a BF16 form");
    const int64_t ld = (s + 63) / 64 * 64;
    const size_t elems = (size_t)d * ld;
    void* bt = nullptr;
    // the same slot and size as run_gauss_tc asks for, so that the stage finds this buffer
    const int rc = handle_scratch(h, 2, elems * 2 * (prec == LEV_BF16X3 ? 2 : 1), &bt);
    if (rc != LEV_OK) return rc;
    *hi = static_cast<__nv_bfloat16*>(bt);
    *lo = prec == LEV_BF16X3 ? static_cast<__nv_bfloat16*>(bt) + elems : nullptr;
    *ld_out = ld;
    return LEV_OK;
}

int tc_gaussian_stage_blocked(lev_handle* h, int64_t m, int64_t s, int64_t d, uint64_t seed, int32_t prec,
                              float* Atilde, cudaStream_t st) {
    switch (prec) {
        case LEV_BF16: return run_gauss_tc<gBF16>(h, nullptr, m, s, d, seed, Atilde, st);
        case LEV_BF16X3: return run_gauss_tc<gBF16X3>(h, nullptr, m, s, d, seed, Atilde, st);
        default: return handle_fail(LEV_EINVAL, "blocked operand needs a BF16 form");
    }
}

int tc_gaussian_stage(lev_handle* h, const float* B, int64_t m, int64_t s, int64_t d, uint64_t seed, int32_t prec,
                      float* Atilde, cudaStream_t st) {
    if (!B) return handle_fail(LEV_EINVAL, "null B for the Gaussian stage");
    switch (prec) {
        case LEV_BF16: return run_gauss_tc<gBF16>(h, B, m, s, d, seed, Atilde, st);
        case LEV_BF16X3: return run_gauss_tc<gBF16X3>(h, B, m, s, d, seed, Atilde, st);
        case LEV_TF32: return run_gauss_tc<gTF32>(h, B, m, s, d, seed, Atilde, st);
        default: return handle_fail(LEV_EINVAL, "unknown tensor-core precision for the Gaussian stage");
    }
}

}  // namespace lev
