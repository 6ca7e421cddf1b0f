// Tensor-core (tcgen05, sm_103a) Gaussian stage of the CountGauss sketch
// (Alg. 3 step 3): A~ (m x d) = G (m x s) B (s x d), a long-K GEMM.
//
// Split-K over the grid: CTA (tile of 128 rows of G, tile of up to 256 columns
// of B, K slice) accumulates its 128 x NT block in TMEM over its slice of s and
// writes the FP32 partial; a second kernel adds the partials of the slices in
// a fixed order. Operands are K-major (rows of G; rows of B^T, produced by a
// transpose kernel), loaded by 2-D tensor TMA with the 128-byte swizzle into a
// ring of shared-memory stages:
//   warp 0: TMA producer (one thread); warp 1: TMEM allocation and the MMA
//   issuer (one thread); warps 2..5: epilogue (tcgen05.ld, partial stores).
// G = Z / sqrt(m) with Z exact in BF16 (the BF16 rounding of the counter draws), so G is never
// split: the MMAs take Z and the reduction applies 1 / sqrt(m). Forms: BF16 (Z times B rounded to
// BF16, one MMA per K step), BF16X3 (Z B_hi + Z B_lo, B split into BF16 hi + lo: two MMAs), TF32
// (Z, exact in TF32, times B rounded to TF32).
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
    static constexpr int kElem = 2, kKbe = 64, kStages = 4;
};
template <>
struct GTraits<gBF16X3> {
    static constexpr bool kTf32 = false, kSplit = true;
    static constexpr int kElem = 2, kKbe = 64, kStages = 2;
};
template <>
struct GTraits<gTF32> {
    static constexpr bool kTf32 = true, kSplit = false;
    static constexpr int kElem = 4, kKbe = 32, kStages = 4;
};

constexpr int kRowsM = 128;
constexpr int kMaxNt = 256;
constexpr uint64_t kWaitNs = 2000000000ull;
constexpr int32_t kStatusGaussTimeout = 4;

struct GCtl {
    uint64_t full[4], empty[4], tfull;
    uint32_t tmem_base;
    int32_t abort;
};

__device__ __forceinline__ bool gwait(uint32_t bar, uint32_t parity, GCtl* ctl, int32_t* status) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
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

// Grid: x = m tile * n_tiles + n tile, y = K slice. Partial P[z][c][i] (c < d, i < m).
template <int F>
__global__ void __launch_bounds__(192, 1) k_gauss_tc(const __grid_constant__ CUtensorMap tmG,
                                                     const __grid_constant__ CUtensorMap tmB,
                                                     const __grid_constant__ CUtensorMap tmBlo, int m, int d, int nt,
                                                     int n_tiles, int kb_per_slice, int kb_total,
                                                     float* __restrict__ P, int32_t* status) {
    using T = GTraits<F>;
    constexpr int STAGES = T::kStages;
    const int A_BYTES = kRowsM * 128;
    const int B_BYTES = nt * 128;
    const int STAGE_BYTES = A_BYTES + B_BYTES * (T::kSplit ? 2 : 1);   // Z tile, B_hi (and B_lo) tile
    const uint32_t idesc = make_idesc(T::kTf32, kRowsM, nt);
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
    uint8_t* base = smem_raw + pad;
    GCtl* ctl = reinterpret_cast<GCtl*>(base + STAGES * STAGE_BYTES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mt = blockIdx.x / n_tiles, ntile = blockIdx.x % n_tiles;
    const int kb0 = blockIdx.y * kb_per_slice;
    const int kb1 = min(kb_total, kb0 + kb_per_slice);
    const int nkb = max(0, kb1 - kb0);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(smem_u32(&ctl->full[s]), 1);
            mbar_init(smem_u32(&ctl->empty[s]), 1);
        }
        mbar_init(smem_u32(&ctl->tfull), 1);
        ctl->abort = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (warp == 1) {
        tmem_alloc(smem_u32(&ctl->tmem_base), 256);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = ctl->tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            for (int i = 0; i < nkb; ++i) {
                if (!gwait(smem_u32(&ctl->empty[stage]), phase ^ 1u, ctl, status)) break;
                const uint32_t sb = smem_u32(base + stage * STAGE_BYTES);
                const uint32_t bar = smem_u32(&ctl->full[stage]);
                mbar_arrive_expect_tx(bar, (uint32_t)STAGE_BYTES);
                const int x = (kb0 + i) * T::kKbe;
                tma_load_2d(sb, &tmG, x, mt * kRowsM, bar);
                tma_load_2d(sb + A_BYTES, &tmB, x, ntile * nt, bar);
                if constexpr (T::kSplit) tma_load_2d(sb + A_BYTES + B_BYTES, &tmBlo, x, ntile * nt, bar);
                if (++stage == STAGES) { stage = 0; phase ^= 1u; }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int i = 0; i < nkb; ++i) {
                if (!gwait(smem_u32(&ctl->full[stage]), phase, ctl, status)) { ok = false; break; }
                tc_fence_after();
                const uint32_t sb = smem_u32(base + stage * STAGE_BYTES);
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                    const uint32_t ko = (uint32_t)ks * 32u;
                    const uint32_t acc = (i | ks) != 0 ? 1u : 0u;
                    tc_mma<T::kTf32>(tmem, sw128_desc(sb + ko), sw128_desc(sb + A_BYTES + ko), idesc, acc);
                    if constexpr (T::kSplit)
                        tc_mma<false>(tmem, sw128_desc(sb + ko), sw128_desc(sb + A_BYTES + B_BYTES + ko), idesc, 1u);
                }
                tc_commit(smem_u32(&ctl->empty[stage]));
                if (++stage == STAGES) { stage = 0; phase ^= 1u; }
            }
            if (ok) tc_commit(smem_u32(&ctl->tfull));
        }
        __syncwarp();
    } else {
        // epilogue: warps 2..5 cover TMEM lane groups (warp % 4)
        const int lg = warp & 3;
        const int row = mt * kRowsM + lg * 32 + lane;
        float* out = P + (int64_t)blockIdx.y * d * m;
        if (nkb == 0) {
            for (int c = 0; c < nt; ++c) {
                const int col = ntile * nt + c;
                if (row < m && col < d) out[(int64_t)col * m + row] = 0.f;
            }
        } else if (gwait(smem_u32(&ctl->tfull), 0, ctl, status)) {
            tc_fence_after();
            for (int c0 = 0; c0 < nt; c0 += 32) {
                uint32_t r[32];
                tmem_ld32(tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)c0, r);
                tmem_ld_wait();
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int col = ntile * nt + c0 + j;
                    if (row < m && col < d) out[(int64_t)col * m + row] = __uint_as_float(r[j]);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 256);
    }
}

// A~ = scale * (sum of the K-slice partials, in slice order); scale = 1 / sqrt(m) (G = Z / sqrt(m)).
__global__ void k_gauss_reduce(const float* __restrict__ P, int splits, int m, int d, float scale,
                               float* __restrict__ At) {
    const int64_t total = (int64_t)m * d;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / m), i = (int)(e % m);        // i fastest: coalesced partial reads
        float acc = 0.f;
        for (int z = 0; z < splits; ++z) acc += P[(int64_t)z * total + e];
        At[(int64_t)i * d + c] = acc * scale;
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

// Row-major matrix rows x cols (elements) with leading dimension ld, box (box_cols x box_rows).
bool make_map(CUtensorMap* map, const void* ptr, bool tf32, int64_t rows, int64_t cols, int64_t ld, int box_cols,
              int box_rows) {
    return make_map_2d(map, ptr, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, tf32 ? 4 : 2,
                       rows, cols, ld, box_cols, box_rows);
}

template <int F>
int run_gauss_tc(lev_handle* h, const float* B, int64_t m, int64_t s, int64_t d, uint64_t seed, float* Atilde,
                 cudaStream_t st) {
    using T = GTraits<F>;
    const int64_t ld = (s + 63) / 64 * 64;                // padded K: 16-byte row strides, whole 128-byte rows
    // G image (cached in the handle): kind 2 = Z in BF16 (ld), kind 3 = Z in FP32 (ld; exact in TF32)
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
    dim3 tg((unsigned)((ld + 63) / 64), (unsigned)((d + 31) / 32));
    k_transpose_operand<F><<<tg, 256, 0, st>>>(B, s, (int)d, ld, bt, bt_lo);
    // tiles and K slices
    const int nt_full = (int)std::min<int64_t>(kMaxNt, (d + 15) / 16 * 16);
    const int n_tiles = (int)((d + nt_full - 1) / nt_full);
    const int nt = (int)(((d + n_tiles - 1) / n_tiles + 15) / 16 * 16);
    const int m_tiles = (int)((m + kRowsM - 1) / kRowsM);
    const int kb_total = (int)(ld / T::kKbe);
    const int sms = handle_num_sms(h);
    int splits = std::max(1, (sms + m_tiles * n_tiles - 1) / (m_tiles * n_tiles));
    splits = std::min(splits, kb_total);
    const int kb_per_slice = (kb_total + splits - 1) / splits;
    splits = (kb_total + kb_per_slice - 1) / kb_per_slice;
    void* part = nullptr;
    rc = handle_scratch(h, 1, sizeof(float) * (size_t)splits * m * d, &part);
    if (rc != LEV_OK) return rc;
    CUtensorMap mG, mB, mBlo;
    const void* gimg = T::kTf32 ? static_cast<const void*>(g32) : static_cast<const void*>(ghi);
    bool ok = make_map(&mG, gimg, T::kTf32, m, ld, ld, T::kKbe, kRowsM) &&
              make_map(&mB, bt, T::kTf32, d, ld, ld, T::kKbe, nt);
    if (T::kSplit)
        ok = ok && make_map(&mBlo, bt_lo, false, d, ld, ld, T::kKbe, nt);
    else
        mBlo = mB;
    if (!ok) return handle_fail(LEV_ECUDA, "cuTensorMapEncodeTiled failed for the Gaussian stage");
    const int stage_bytes = kRowsM * 128 + nt * 128 * (T::kSplit ? 2 : 1);
    const size_t smem = 1024 + (size_t)T::kStages * stage_bytes + sizeof(GCtl) + 64;
    cudaError_t e = cudaFuncSetAttribute(k_gauss_tc<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return handle_fail(LEV_ECUDA, cudaGetErrorString(e));
    dim3 grid((unsigned)(m_tiles * n_tiles), (unsigned)splits);
    k_gauss_tc<F><<<grid, 192, smem, st>>>(mG, mB, mBlo, (int)m, (int)d, nt, n_tiles, kb_per_slice, kb_total,
                                           static_cast<float*>(part), handle_status(h));
    k_gauss_reduce<<<152 * 4, 256, 0, st>>>(static_cast<const float*>(part), splits, (int)m, (int)d,
                                            (float)(1.0 / std::sqrt((double)m)), Atilde);
    e = cudaGetLastError();
    if (e != cudaSuccess) return handle_fail(LEV_ECUDA, cudaGetErrorString(e));
    return LEV_OK;
}

}  // namespace

int tc_gaussian_stage(lev_handle* h, const float* B, int64_t m, int64_t s, int64_t d, uint64_t seed, int32_t prec,
                      float* Atilde, cudaStream_t st) {
    switch (prec) {
        case LEV_BF16: return run_gauss_tc<gBF16>(h, B, m, s, d, seed, Atilde, st);
        case LEV_BF16X3: return run_gauss_tc<gBF16X3>(h, B, m, s, d, seed, Atilde, st);
        case LEV_TF32: return run_gauss_tc<gTF32>(h, B, m, s, d, seed, Atilde, st);
        default: return handle_fail(LEV_EINVAL, "unknown tensor-core precision for the Gaussian stage");
    }
}

}  // namespace lev
