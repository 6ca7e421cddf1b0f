// Tensor-core (tcgen05, sm_103a) form of the fused final pass (Alg. 8 step 5):
// theta~_i = ||A_i Mfull||^2 with the product accumulated in TMEM and squared
// in the epilogue, so the n x k product never reaches memory.
//
// One persistent CTA per SM (one pair of CTAs for the half-width forms):
//   * warp 12 (MMA warp): allocates TMEM (two accumulators), loads the packed
//     operand image of Mfull^T into shared memory once with bulk TMA copies,
//     and one thread issues tcgen05.mma (M = 128 rows, N = NT columns, 32 bytes
//     of K per instruction) for every K block of every tile;
//   * warps 4..11 (converters): coalesced 128-bit loads of A rows, rounding to
//     the operand type (BF16, BF16 hi + lo, or TF32), stores into the 128-byte
//     swizzled K-major operand layout, one K block (128 bytes of K per row) per
//     pipeline stage;
//   * warps 0..3 (epilogue): tcgen05.ld of the accumulator (TMEM lane = row),
//     sum of squares per row, one FP32 store (or atomic add of the half-width
//     partial) per row.
// Forms: BF16 (N = 256, one CTA per tile); BF16X3 (hi*hi + lo*hi + hi*lo,
// N = 128 per CTA, a pair of CTAs per tile); TF32 (N = 128 per CTA, pair).
// The half-width forms exist because a K x 256 operand of 4-byte (TF32) or
// split (2 x 2-byte) values is 256 KB, more than a CTA's shared memory.
// Every wait is bounded (2 s of %globaltimer); on expiry the CTA records the
// failure in the status word and leaves its loops.
#include <cuda_bf16.h>

#include "lev_common.cuh"
#include "lev_tc.cuh"
#include "tc_common.cuh"

namespace lev {

namespace {

using namespace tcx;

// ------------------------------------------------------------------ forms

enum Form { kBF16 = 0, kBF16X3 = 1, kTF32 = 2 };

template <int F>
struct FormTraits;
template <>
struct FormTraits<kBF16> {
    static constexpr bool kTf32 = false, kSplit = false;
    static constexpr int kElem = 2, kKbe = 64, kNt = 256, kStages = 4, kPair = 1;
};
template <>
struct FormTraits<kBF16X3> {
    static constexpr bool kTf32 = false, kSplit = true;
    static constexpr int kElem = 2, kKbe = 64, kNt = 128, kStages = 2, kPair = 2;
};
template <>
struct FormTraits<kTF32> {
    static constexpr bool kTf32 = true, kSplit = false;
    static constexpr int kElem = 4, kKbe = 32, kNt = 128, kStages = 4, kPair = 2;
};

constexpr int kTileRows = 128;
constexpr int kKBlockBytes = kTileRows * 128;     // one K block of the A operand: 16 KB
constexpr int kEpiWarps = 4, kCvtWarps = 8;
constexpr int kMmaWarp = kEpiWarps + kCvtWarps;   // warp 12
constexpr int kThreads = (kMmaWarp + 1) * 32;     // 416
constexpr uint64_t kWaitNs = 2000000000ull;       // 2 s
constexpr int32_t kStatusTcTimeout = 2;

struct TcSmemCtl {
    uint64_t full[4], empty[4], tfull[2], tempty[2], mfull;
    uint32_t tmem_base;
    int32_t abort;
};

// Bounded wait on an mbarrier phase; false if this CTA gave up.
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, TcSmemCtl* ctl, int32_t* status) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 0) {
            if (*(volatile int32_t*)&ctl->abort) return false;
            if (global_ns() - t0 > kWaitNs) {
                *(volatile int32_t*)&ctl->abort = 1;
                atomicExch(status, kStatusTcTimeout);
                return false;
            }
        }
    }
}

template <int F>
__global__ void __launch_bounds__(kThreads, 1) k_final_tc(const float* __restrict__ A, int64_t lda, int64_t n,
                                                          int d, int nkb, const uint8_t* __restrict__ image,
                                                          uint32_t image_bytes, float* __restrict__ theta,
                                                          int32_t* status) {
    using T = FormTraits<F>;
    constexpr int NT = T::kNt;
    constexpr int STAGES = T::kStages;
    constexpr int A_STAGE_BYTES = kKBlockBytes * (T::kSplit ? 2 : 1);
    constexpr uint32_t IDESC = make_idesc(T::kTf32, kTileRows, NT);
    extern __shared__ uint8_t smem_raw[];
    // 1024-byte aligned operand area: [image | A stages], control block after it
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
    uint8_t* base = smem_raw + pad;
    uint8_t* img = base;                                   // image_bytes (multiple of 1024)
    uint8_t* astage = base + image_bytes;                  // STAGES x A_STAGE_BYTES
    TcSmemCtl* ctl = reinterpret_cast<TcSmemCtl*>(astage + STAGES * A_STAGE_BYTES);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int half = (T::kPair == 2) ? (int)(blockIdx.x & 1) : 0;
    const int group = (T::kPair == 2) ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
    const int ngroups = (T::kPair == 2) ? (int)(gridDim.x >> 1) : (int)gridDim.x;
    const int64_t ntiles = (n + kTileRows - 1) / kTileRows;
    const uint32_t img_half_bytes = image_bytes;           // this CTA's half (or the whole image)

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(smem_u32(&ctl->full[s]), kCvtWarps);
            mbar_init(smem_u32(&ctl->empty[s]), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(smem_u32(&ctl->tfull[a]), 1);
            mbar_init(smem_u32(&ctl->tempty[a]), kEpiWarps);
        }
        mbar_init(smem_u32(&ctl->mfull), 1);
        ctl->abort = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (warp == kMmaWarp) {
        tmem_alloc(smem_u32(&ctl->tmem_base), 2 * NT);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = ctl->tmem_base;

    if (warp == kMmaWarp) {
        if (lane == 0) {
            // Operand image of Mfull^T for this CTA's column half: bulk TMA copies, 16 KB each.
            const uint8_t* src = image + (size_t)half * img_half_bytes;
            const uint32_t mbar = smem_u32(&ctl->mfull);
            mbar_arrive_expect_tx(mbar, img_half_bytes);
            for (uint32_t off = 0; off < img_half_bytes; off += 16384u) {
                const uint32_t len = min(16384u, img_half_bytes - off);
                bulk_g2s(smem_u32(img + off), src + off, len, mbar);
            }
            bool ok = wait_bar(mbar, 0, ctl, status);
            int stage = 0;
            uint32_t phase = 0;
            int acc = 0;
            uint32_t acc_phase = 0;
            const uint32_t img_addr = smem_u32(img);
            const uint32_t a_addr = smem_u32(astage);
            const uint32_t kb_img_bytes = (uint32_t)NT * 128u;     // one K block of the image
            for (int64_t t = group; ok && t < ntiles; t += ngroups) {
                if (!wait_bar(smem_u32(&ctl->tempty[acc]), acc_phase ^ 1u, ctl, status)) { ok = false; break; }
                tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(acc * NT);
                for (int kb = 0; kb < nkb; ++kb) {
                    if (!wait_bar(smem_u32(&ctl->full[stage]), phase, ctl, status)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t a_hi = a_addr + (uint32_t)stage * A_STAGE_BYTES;
                    const uint32_t m_hi = img_addr + (uint32_t)kb * kb_img_bytes;
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint32_t koff = (uint32_t)ks * 32u;
                        const uint32_t first = (kb | ks) != 0 ? 1u : 0u;
                        tc_mma<T::kTf32>(d_tmem, sw128_desc(a_hi + koff), sw128_desc(m_hi + koff), IDESC, first);
                        if constexpr (T::kSplit) {
                            const uint32_t a_lo = a_hi + kKBlockBytes;
                            const uint32_t m_lo = m_hi + (uint32_t)nkb * kb_img_bytes;
                            tc_mma<false>(d_tmem, sw128_desc(a_lo + koff), sw128_desc(m_hi + koff), IDESC, 1u);
                            tc_mma<false>(d_tmem, sw128_desc(a_hi + koff), sw128_desc(m_lo + koff), IDESC, 1u);
                        }
                    }
                    tc_commit(smem_u32(&ctl->empty[stage]));      // frees the A stage when these MMAs finish
                    if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                }
                if (!ok) break;
                tc_commit(smem_u32(&ctl->tfull[acc]));            // accumulator ready for the epilogue
                acc ^= 1;
                if (acc == 0) acc_phase ^= 1u;
            }
        }
        __syncwarp();
    } else if (warp >= kEpiWarps) {
        // ---------------- converters: A rows -> operand layout
        // Work items are (tile, K block) in order. The loads of the next PD items
        // are in flight while the current item is rounded and stored.
        const int cw = warp - kEpiWarps;                   // 0..7, 16 rows each
        constexpr int LPR = T::kKbe / 4;                   // lanes per row (one float4 each)
        constexpr int RPI = 32 / LPR;                      // rows per warp iteration
        constexpr int ITERS = 16 / RPI;
        constexpr int PD = T::kTf32 ? 4 : 2;               // K blocks of loads in flight
        const int sub = lane % LPR, rsub = lane / LPR;
        const int64_t my_tiles = (ntiles - group + ngroups - 1) / ngroups;
        const int64_t total = (my_tiles > 0 ? my_tiles : 0) * nkb;
        float4 v[PD][ITERS];
        auto load_item = [&](int64_t item, float4 (&dst)[ITERS]) {
            const int64_t t = group + (item / nkb) * ngroups;
            const int kb = (int)(item % nkb);
            const int64_t row0 = t * kTileRows;
            const int col = kb * T::kKbe + sub * 4;
#pragma unroll
            for (int it = 0; it < ITERS; ++it) {
                const int64_t gr = row0 + cw * 16 + it * RPI + rsub;
                dst[it] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (gr < n && col < d) dst[it] = __ldg(reinterpret_cast<const float4*>(A + gr * lda + col));
            }
        };
#pragma unroll
        for (int p = 0; p < PD; ++p)
            if (p < total) load_item(p, v[p]);
        int stage = 0;
        uint32_t phase = 0;
        bool ok = true;
        for (int64_t i0 = 0; ok && i0 < total; i0 += PD) {
#pragma unroll
            for (int p = 0; p < PD; ++p) {
                const int64_t item = i0 + p;
                if (item >= total) break;
                if (!wait_bar(smem_u32(&ctl->empty[stage]), phase ^ 1u, ctl, status)) { ok = false; break; }
                uint8_t* dst = astage + stage * A_STAGE_BYTES;
#pragma unroll
                for (int it = 0; it < ITERS; ++it) {
                    const uint32_t r = (uint32_t)(cw * 16 + it * RPI + rsub);
                    const float4 x = v[p][it];
                    if constexpr (T::kTf32) {
                        uint4 w = make_uint4(f32_to_tf32(x.x), f32_to_tf32(x.y), f32_to_tf32(x.z), f32_to_tf32(x.w));
                        *reinterpret_cast<uint4*>(dst + sw128_offset(r, (uint32_t)sub * 16u)) = w;
                    } else {
                        const __nv_bfloat16 h0 = __float2bfloat16_rn(x.x), h1 = __float2bfloat16_rn(x.y);
                        const __nv_bfloat16 h2 = __float2bfloat16_rn(x.z), h3 = __float2bfloat16_rn(x.w);
                        uint2 w;
                        w.x = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
                        w.y = (uint32_t)__bfloat16_as_ushort(h2) | ((uint32_t)__bfloat16_as_ushort(h3) << 16);
                        const uint32_t off = sw128_offset(r, (uint32_t)sub * 8u);
                        *reinterpret_cast<uint2*>(dst + off) = w;
                        if constexpr (T::kSplit) {
                            const __nv_bfloat16 l0 = __float2bfloat16_rn(x.x - __bfloat162float(h0));
                            const __nv_bfloat16 l1 = __float2bfloat16_rn(x.y - __bfloat162float(h1));
                            const __nv_bfloat16 l2 = __float2bfloat16_rn(x.z - __bfloat162float(h2));
                            const __nv_bfloat16 l3 = __float2bfloat16_rn(x.w - __bfloat162float(h3));
                            uint2 u;
                            u.x = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
                            u.y = (uint32_t)__bfloat16_as_ushort(l2) | ((uint32_t)__bfloat16_as_ushort(l3) << 16);
                            *reinterpret_cast<uint2*>(dst + kKBlockBytes + off) = u;
                        }
                    }
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&ctl->full[stage]));
                if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                if (item + PD < total) load_item(item + PD, v[p]);
            }
        }
    } else {
        // ---------------- epilogue: TMEM lane = tile row
        int acc = 0;
        uint32_t acc_phase = 0;
        for (int64_t t = group; t < ntiles; t += ngroups) {
            if (!wait_bar(smem_u32(&ctl->tfull[acc]), acc_phase, ctl, status)) break;
            tc_fence_after();
            float sum = 0.f;
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(acc * NT);
#pragma unroll
            for (int c = 0; c < NT; c += 32) {
                uint32_t r[32];
                tmem_ld32(taddr + (uint32_t)c, r);
                tmem_ld_wait();
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const float y = __uint_as_float(r[j]);
                    sum = fmaf(y, y, sum);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&ctl->tempty[acc]));
            const int64_t row = t * kTileRows + warp * 32 + lane;
            if (row < n) {
                if constexpr (T::kPair == 2)
                    atomicAdd(theta + row, sum);
                else
                    theta[row] = sum;
            }
            acc ^= 1;
            if (acc == 0) acc_phase ^= 1u;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc_fence_after();
        tmem_dealloc(tmem, 2 * NT);
    }
}

// Pack Mfull (d x k FP32, row-major) into the operand image of Mfull^T:
// per column half h, per K block kb, NT rows (columns q of Mfull) of 128 bytes,
// 128-byte swizzled; split forms store the hi image then the lo image.
template <int F>
__global__ void k_pack_image(const float* __restrict__ M, int d, int k, int nkb, uint8_t* __restrict__ image,
                             uint32_t half_bytes) {
    using T = FormTraits<F>;
    constexpr int NT = T::kNt;
    const int64_t per_half = (int64_t)nkb * NT * T::kKbe;
    const int64_t total = per_half * T::kPair;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int h = (int)(e / per_half);
        int64_t rem = e % per_half;
        const int kb = (int)(rem / (NT * T::kKbe));
        rem %= NT * T::kKbe;
        const int nl = (int)(rem / T::kKbe), el = (int)(rem % T::kKbe);
        const int q = h * NT + nl, kk = kb * T::kKbe + el;
        const float x = (q < k && kk < d) ? M[(int64_t)kk * k + q] : 0.f;
        uint8_t* dst = image + (size_t)h * half_bytes + (size_t)kb * NT * 128;
        const uint32_t off = sw128_offset((uint32_t)nl, (uint32_t)(el * T::kElem));
        if constexpr (T::kTf32) {
            *reinterpret_cast<uint32_t*>(dst + off) = f32_to_tf32(x);
        } else {
            const __nv_bfloat16 hi = __float2bfloat16_rn(x);
            *reinterpret_cast<__nv_bfloat16*>(dst + off) = hi;
            if constexpr (T::kSplit) {
                const __nv_bfloat16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
                *reinterpret_cast<__nv_bfloat16*>(dst + (size_t)nkb * NT * 128 + off) = lo;
            }
        }
    }
}

template <int F>
int run_final_tc(lev_handle* h, const float* A, int64_t n, int64_t d, int64_t lda, const float* Mfull, int64_t k,
                 float* theta, int32_t* status, cudaStream_t st) {
    using T = FormTraits<F>;
    const int nkb = (int)((d + T::kKbe - 1) / T::kKbe);
    const uint32_t half_bytes = (uint32_t)nkb * T::kNt * 128u * (T::kSplit ? 2u : 1u);
    void* ws = nullptr;
    int rc = handle_scratch(h, 0, (size_t)half_bytes * T::kPair, &ws);
    if (rc != LEV_OK) return rc;
    uint8_t* image = static_cast<uint8_t*>(ws);
    k_pack_image<F><<<64, 256, 0, st>>>(Mfull, (int)d, (int)k, nkb, image, half_bytes);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return handle_fail(LEV_ECUDA, cudaGetErrorString(e));
    if (T::kPair == 2) {
        e = cudaMemsetAsync(theta, 0, sizeof(float) * (size_t)n, st);
        if (e != cudaSuccess) return handle_fail(LEV_ECUDA, cudaGetErrorString(e));
    }
    const int stage_bytes = kKBlockBytes * (T::kSplit ? 2 : 1);
    const size_t smem = 1024 + (size_t)half_bytes + (size_t)T::kStages * stage_bytes + sizeof(TcSmemCtl) + 64;
    e = cudaFuncSetAttribute(k_final_tc<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return handle_fail(LEV_ECUDA, cudaGetErrorString(e));
    const int64_t ntiles = (n + kTileRows - 1) / kTileRows;
    const int sms = handle_num_sms(h);
    int64_t groups = T::kPair == 2 ? sms / 2 : sms;
    if (groups > ntiles) groups = ntiles;
    if (groups < 1) groups = 1;
    k_final_tc<F><<<(unsigned)(groups * T::kPair), kThreads, smem, st>>>(A, lda, n, (int)d, nkb, image, half_bytes,
                                                                          theta, status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return handle_fail(LEV_ECUDA, cudaGetErrorString(e));
    return LEV_OK;
}

}  // namespace

int tc_final_dense(lev_handle* h, const float* A, int64_t n, int64_t d, int64_t lda, const float* Mfull, int64_t k,
                   int32_t prec, float* theta, cudaStream_t st) {
    if ((reinterpret_cast<uintptr_t>(A) & 15u) != 0 || (lda & 3) != 0 || (d & 3) != 0)
        return handle_fail(LEV_EINVAL, "tensor-core final pass needs A 16-byte aligned, lda and d multiples of 4");
    if (d > 256 || k > 256)
        return handle_fail(LEV_EINVAL, "tensor-core final pass needs d <= 256 and k <= 256");
    int32_t* status = handle_status(h);
    switch (prec) {
        case LEV_BF16: return run_final_tc<kBF16>(h, A, n, d, lda, Mfull, k, theta, status, st);
        case LEV_BF16X3: return run_final_tc<kBF16X3>(h, A, n, d, lda, Mfull, k, theta, status, st);
        case LEV_TF32: return run_final_tc<kTF32>(h, A, n, d, lda, Mfull, k, theta, status, st);
        default: return handle_fail(LEV_EINVAL, "unknown tensor-core precision");
    }
}

}  // namespace lev
