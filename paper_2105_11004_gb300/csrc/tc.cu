// Tensor-core (tcgen05, sm_103a) form of the fused final pass (Alg. 8 step 5):
// theta~_i = ||A_i Mfull||^2 with the product accumulated in TMEM and squared
// in the epilogue, so the n x k product never reaches memory.
//
// One persistent CTA per SM (BF16) or per SM of a 2-CTA cluster (BF16X3, TF32).
// Shared memory holds the CTA's part of the packed operand image of Mfull^T and
// a ring of slots; a slot holds one K block of the CTA's 128 rows of A.
//   * warp 17 (producer): 2-D tensor TMA of a slot's FP32 boxes (32 columns x
//     128 rows each, 128-byte swizzle);
//   * warps 4..15 (converters, three groups of four): round the slot IN PLACE to
//     the operand type; the groups take the slots in turn, so three are rounded
//     at once.
//     With 64-column K blocks the two FP32 boxes of row r occupy exactly the
//     bytes that the BF16 hi row r and lo row r take in the 128-byte swizzled
//     K-major operand layout (same row, same swizzle phase), so a warp that owns
//     whole rows reads them, syncs, and writes them back; TF32 rounds each
//     16-byte chunk where it lies;
//   * warp 16 (MMA): allocates TMEM (two accumulators of 256 columns), loads the
//     image once with bulk copies, and one thread issues tcgen05.mma (N = the
//     width of Mfull, 32 bytes of K per instruction); the MMA completion frees
//     the slot;
//   * warps 0..3 (epilogue): tcgen05.ld of the accumulator (TMEM lane = row),
//     sum of squares over the N columns, one store per row.
// N: Mfull's columns up to its last nonzero one, rounded up to 16 (k_mfull_width
// finds it on the device). Trailing zero columns add nothing to theta~; the
// r-column factor of lev_omega_factor's reduced form leaves k - r of them.
// BF16: M = 128 per CTA; the 128 KB image of Mfull^T (256 x 256 BF16) fits one
// CTA. BF16X3 (hi*hi + lo*hi + hi*lo) and TF32 need 256 KB for the image, so
// they run as CTA pairs with cta_group::2: one thread of the even CTA issues an
// M = 256 MMA for the pair; each CTA holds its own 128 rows of A and half of
// the image (128 columns of Mfull), and each CTA's TMEM receives its own rows
// with all 256 columns. Nothing is loaded twice and no operand crosses between
// the CTAs except through the MMA itself. The odd CTA reports "slot converted"
// and "accumulator drained" to the even CTA's mbarriers; MMA completions are
// multicast to both. Every wait is bounded (2 s of %globaltimer); on expiry the
// CTA records the failure in the status word and leaves its loops.
#include <atomic>
#include <cuda.h>
#include <cuda_bf16.h>

#include "lev_common.cuh"
#include "lev_tc.cuh"
#include "tc_common.cuh"

namespace lev {

namespace {

using namespace tcx;

enum Form { kBF16 = 0, kBF16X3 = 1, kTF32 = 2 };

// kKbe: operand elements per K block (128 bytes of a row); kNt: rows of the Mfull^T image one CTA
// holds; kPair: CTAs per MMA; kSlots: slots in the ring.
template <int F>
struct FormTraits;
template <>
struct FormTraits<kBF16> {
    static constexpr bool kTf32 = false, kSplit = false;
    static constexpr int kElem = 2, kKbe = 64, kNt = 256, kPair = 1, kSlots = 3;
};
template <>
struct FormTraits<kBF16X3> {
    static constexpr bool kTf32 = false, kSplit = true;
    static constexpr int kElem = 2, kKbe = 64, kNt = 128, kPair = 2, kSlots = 3;
};
template <>
struct FormTraits<kTF32> {
    static constexpr bool kTf32 = true, kSplit = false;
    static constexpr int kElem = 4, kKbe = 32, kNt = 128, kPair = 2, kSlots = 6;
};

constexpr int kTileRows = 128;                    // rows of A per CTA per tile (TMEM lanes)
constexpr int kBoxBytes = kTileRows * 128;        // one FP32 box: 128 rows x 32 columns = one 16 KB K block
constexpr int kNOut = 256;                        // accumulator columns per row (the widest MMA N)
// Converters: kCvtGroups groups of four warps; group g rounds the slot fills u with u mod
// kCvtGroups = g, so each slot belongs to one group (the slot counts are multiples of it) and its
// fills are taken in order, while the groups' slots are rounded at the same time.
constexpr int kEpiWarps = 4, kCvtGroups = 3, kCvtWarpsPerGroup = 4;
constexpr int kCvtWarps = kCvtGroups * kCvtWarpsPerGroup;
constexpr int kMmaWarp = kEpiWarps + kCvtWarps;   // warp 16
constexpr int kTmaWarp = kMmaWarp + 1;            // warp 17
constexpr int kThreads = (kTmaWarp + 1) * 32;     // 576
constexpr int kMaxSlots = 6;
constexpr uint64_t kWaitNs = 2000000000ull;       // 2 s
constexpr uint64_t kExitWaitNs = 5000000000ull;   // 5 s: a peer that timed out reaches the exit within one kWaitNs
constexpr int32_t kStatusTcTimeout = 2;

struct TcSmemCtl {
    uint64_t sfull[kMaxSlots], cfull[kMaxSlots], sempty[kMaxSlots], tfull[2], tempty[2], mfull, ipeer, mdone, xbar;
    uint32_t tmem_base;
    int32_t abort;
};

// Bounded wait on an mbarrier phase (acquire at cluster scope); false if this CTA gave up.
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, TcSmemCtl* ctl, int32_t* status) {
    if (mbar_try_wait_cluster(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait_cluster(bar, parity)) return true;
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

// Bounded wait that an abort does not cut short: used to drain copies, MMAs and peer
// arrivals still in flight before TMEM is freed and the CTA exits.
__device__ __forceinline__ bool drain_bar(uint32_t bar, uint32_t parity, uint64_t limit_ns, int32_t* status) {
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait_cluster(bar, parity)) {
        if (global_ns() - t0 > limit_ns) {
            atomicExch(status, kStatusTcTimeout);
            return false;
        }
    }
    return true;
}

// Arrive on the mbarrier at `bar` in the even CTA of the pair (this CTA when unpaired).
template <int PAIR>
__device__ __forceinline__ void arrive_leader(uint32_t bar, uint32_t me) {
    if constexpr (PAIR == 2) {
        if (me == 0)
            mbar_arrive_cluster(bar);
        else
            mbar_arrive_cluster(mapa_shared(bar, 0));
    } else {
        mbar_arrive(bar);
    }
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b, float* ra, float* rb) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 f = __bfloat1622float2(h);
    *ra = a - f.x;
    *rb = b - f.y;
    return *reinterpret_cast<const uint32_t*>(&h);
}

// MMA width for an Mfull whose columns from `width` on are zero: a multiple of 16 in [16, 256]
// (a multiple of 8 rows of the image in each CTA of a pair).
__device__ __forceinline__ int mma_width(const int* width) {
    int w = *width;
    w = w < 16 ? 16 : (w > kNOut ? kNOut : w);
    return (w + 15) & ~15;
}

// *width = 1 + the last column of Mfull (d x k) holding a nonzero (or NaN) entry; 0 if none.
__global__ void k_mfull_width(const float* __restrict__ M, int d, int k, int* width) {
    int w = 0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)d * k;
         e += (int64_t)gridDim.x * blockDim.x)
        if (M[e] != 0.f) w = max(w, (int)(e % k) + 1);
    w = (int)__reduce_max_sync(0xffffffffu, (unsigned)w);
    if ((threadIdx.x & 31) == 0 && w > 0) atomicMax(width, w);
}

// Round rows 16 cw .. 16 cw + 15 of one slot in place.
template <int F>
__device__ __forceinline__ void convert_slot(uint8_t* slot, int cw, int lane) {
    using T = FormTraits<F>;
    if constexpr (T::kTf32) {
        // one box; each 16-byte chunk is rounded where it lies
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t task = (uint32_t)(q * 32 + lane);           // 16 rows x 8 chunks
            const uint32_t row = (uint32_t)cw * 16u + (task >> 3), c = task & 7u;
            uint4* p = reinterpret_cast<uint4*>(slot + sw128_offset(row, c * 16u));
            const float4 x = *reinterpret_cast<const float4*>(p);
            *p = make_uint4(f32_to_tf32(x.x), f32_to_tf32(x.y), f32_to_tf32(x.z), f32_to_tf32(x.w));
        }
    } else {
        // two boxes (columns 0..31 and 32..63) -> BF16 hi K block in box 0's bytes, lo in box 1's
        float4 x[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const uint32_t task = (uint32_t)(q * 32 + lane);           // 16 rows x 16 chunks
            const uint32_t row = (uint32_t)cw * 16u + (task >> 4), ch = task & 15u;
            x[q] = *reinterpret_cast<const float4*>(slot + (ch >> 3) * kBoxBytes + sw128_offset(row, (ch & 7u) * 16u));
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const uint32_t task = (uint32_t)(q * 32 + lane);
            const uint32_t row = (uint32_t)cw * 16u + (task >> 4), ch = task & 15u;
            const uint32_t off = sw128_offset(row, ch * 8u);
            float r0, r1, r2, r3;
            const uint2 hi = make_uint2(pack_bf16x2(x[q].x, x[q].y, &r0, &r1), pack_bf16x2(x[q].z, x[q].w, &r2, &r3));
            *reinterpret_cast<uint2*>(slot + off) = hi;
            if constexpr (T::kSplit) {
                float u0, u1;
                const uint2 lo = make_uint2(pack_bf16x2(r0, r1, &u0, &u1), pack_bf16x2(r2, r3, &u0, &u1));
                *reinterpret_cast<uint2*>(slot + kBoxBytes + off) = lo;
            }
        }
    }
}

template <int F>
__global__ void __launch_bounds__(kThreads, 1) k_final_tc(const __grid_constant__ CUtensorMap tmA, int64_t n,
                                                          int nkb, const uint8_t* __restrict__ image,
                                                          uint32_t image_bytes, const int* __restrict__ width,
                                                          float* __restrict__ theta, int32_t* status) {
    using T = FormTraits<F>;
    constexpr int PAIR = T::kPair;
    constexpr int NS = T::kSlots;
    constexpr int BOXES = T::kKbe / 32;                       // FP32 boxes per K block
    constexpr int SLOT_BYTES = BOXES * kBoxBytes;
    static_assert(T::kNt * PAIR == kNOut, "the image holds up to 256 columns of Mfull");
    const int ne = mma_width(width);                          // MMA N
    const uint32_t kb_img_bytes = (uint32_t)(ne / PAIR) * 128u;   // one K block of this CTA's image
    const uint32_t img_used = (uint32_t)nkb * kb_img_bytes * (T::kSplit ? 2u : 1u);
    const uint32_t IDESC = make_idesc(T::kTf32, kTileRows * PAIR, ne);
    static_assert(NS <= kMaxSlots, "slot barriers");
    static_assert(NS % kCvtGroups == 0, "each slot belongs to one converter group");
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
    uint8_t* img = smem_raw + pad;                            // image_bytes (multiple of 1024)
    uint8_t* slots = img + image_bytes;                       // NS x SLOT_BYTES
    TcSmemCtl* ctl = reinterpret_cast<TcSmemCtl*>(slots + NS * SLOT_BYTES);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t me = PAIR == 2 ? cluster_ctarank() : 0u;
    const bool leader = me == 0;
    const int64_t group = blockIdx.x / PAIR, ngroups = gridDim.x / PAIR;
    constexpr int64_t kGroupRows = (int64_t)kTileRows * PAIR;
    const int64_t ntiles = (n + kGroupRows - 1) / kGroupRows;
    const int64_t my_tiles = ntiles > group ? (ntiles - group + ngroups - 1) / ngroups : 0;
    const int64_t uses = my_tiles * nkb;                      // slot fills (one K block each)

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(smem_u32(&ctl->sfull[s]), 1);
            mbar_init(smem_u32(&ctl->cfull[s]), kCvtWarpsPerGroup * PAIR);
            mbar_init(smem_u32(&ctl->sempty[s]), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(smem_u32(&ctl->tfull[a]), 1);
            mbar_init(smem_u32(&ctl->tempty[a]), kEpiWarps * PAIR);
        }
        mbar_init(smem_u32(&ctl->mfull), 1);
        mbar_init(smem_u32(&ctl->ipeer), 1);
        mbar_init(smem_u32(&ctl->mdone), 1);
        mbar_init(smem_u32(&ctl->xbar), PAIR);
        ctl->abort = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (PAIR == 2) asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    if (warp == kMmaWarp) {
        tmem_alloc_cg<PAIR>(smem_u32(&ctl->tmem_base), 2 * kNOut);
        tmem_relinquish_cg<PAIR>();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = ctl->tmem_base;

    if (warp == kTmaWarp) {
        // ---------------- producer: this CTA's 128 rows of one K block per slot
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            int64_t issued = 0;
            for (int64_t u = 0; u < uses; ++u) {
                if (!wait_bar(smem_u32(&ctl->sempty[s]), ph ^ 1u, ctl, status)) break;
                const int64_t t = group + (u / nkb) * ngroups;
                const int32_t x = (int32_t)(u % nkb) * T::kKbe;
                const int32_t y = (int32_t)(t * kGroupRows + (int64_t)me * kTileRows);
                const uint32_t bar = smem_u32(&ctl->sfull[s]);
                mbar_arrive_expect_tx(bar, (uint32_t)SLOT_BYTES);
                const uint32_t dst = smem_u32(slots + s * SLOT_BYTES);
#pragma unroll
                for (int b = 0; b < BOXES; ++b) tma_load_2d(dst + b * kBoxBytes, &tmA, x + b * 32, y, bar);
                ++issued;
                if (++s == NS) { s = 0; ph ^= 1u; }
            }
            // no copy may still be landing in this CTA's shared memory when it exits, and the
            // last "slot free" signals of the MMA (multicast in a pair) have landed here
            for (int64_t j = issued > NS ? issued - NS : 0; j < issued; ++j)
                drain_bar(smem_u32(&ctl->sfull[j % NS]), (uint32_t)((j / NS) & 1), kWaitNs, status);
            if (issued == uses && !*(volatile int32_t*)&ctl->abort) {
                for (int q = 0; q < NS; ++q) {
                    const int64_t k_uses = uses / NS + (q < uses % NS ? 1 : 0);
                    if (k_uses > 0) drain_bar(smem_u32(&ctl->sempty[q]), (uint32_t)((k_uses - 1) & 1), kWaitNs, status);
                }
            }
        }
        __syncwarp();
    } else if (warp == kMmaWarp) {
        if (lane == 0) {
            const uint8_t* src = image + (size_t)me * image_bytes;
            const uint32_t mbar = smem_u32(&ctl->mfull);
            mbar_arrive_expect_tx(mbar, img_used);
            for (uint32_t off = 0; off < img_used; off += 16384u) {
                const uint32_t len = min(16384u, img_used - off);
                bulk_g2s(smem_u32(img + off), src + off, len, mbar);
            }
            bool ok = wait_bar(mbar, 0, ctl, status);
            if (PAIR == 2 && !leader) {
                // the even CTA's MMAs read this CTA's half of the image
                if (ok) mbar_arrive_cluster(mapa_shared(smem_u32(&ctl->ipeer), 0));
            } else {
                if (PAIR == 2) ok = ok && wait_bar(smem_u32(&ctl->ipeer), 0, ctl, status);
                int s = 0;
                uint32_t sph = 0;
                int acc = 0;
                uint32_t acc_phase = 0;
                const uint32_t img_addr = smem_u32(img);
                const uint32_t slot_addr = smem_u32(slots);
                const uint16_t both = (uint16_t)(PAIR == 2 ? 0x3 : 0x1);
                for (int64_t tt = 0; ok && tt < my_tiles; ++tt) {
                    if (!wait_bar(smem_u32(&ctl->tempty[acc]), acc_phase ^ 1u, ctl, status)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t d_tmem = tmem + (uint32_t)(acc * kNOut);
                    for (int kb = 0; kb < nkb; ++kb) {
                        if (!wait_bar(smem_u32(&ctl->cfull[s]), sph, ctl, status)) { ok = false; break; }
                        tc_fence_after();
                        const uint32_t a_hi = slot_addr + (uint32_t)s * SLOT_BYTES;
                        const uint32_t m_hi = img_addr + (uint32_t)kb * kb_img_bytes;
#pragma unroll
                        for (int ks = 0; ks < 4; ++ks) {
                            const uint32_t koff = (uint32_t)ks * 32u;
                            const uint32_t accum = (kb | ks) != 0 ? 1u : 0u;
                            tc_mma_cg<PAIR, T::kTf32>(d_tmem, sw128_desc(a_hi + koff), sw128_desc(m_hi + koff),
                                                      IDESC, accum);
                            if constexpr (T::kSplit) {
                                const uint32_t a_lo = a_hi + kBoxBytes;
                                const uint32_t m_lo = m_hi + (uint32_t)nkb * kb_img_bytes;
                                tc_mma_cg<PAIR, false>(d_tmem, sw128_desc(a_lo + koff), sw128_desc(m_hi + koff),
                                                       IDESC, 1u);
                                tc_mma_cg<PAIR, false>(d_tmem, sw128_desc(a_hi + koff), sw128_desc(m_lo + koff),
                                                       IDESC, 1u);
                            }
                        }
                        // slot s is free again in both CTAs once these MMAs finish
                        tc_commit_mc<PAIR>(smem_u32(&ctl->sempty[s]), both);
                        if (++s == NS) { s = 0; sph ^= 1u; }
                    }
                    if (!ok) break;
                    tc_commit_mc<PAIR>(smem_u32(&ctl->tfull[acc]), both);
                    acc ^= 1;
                    if (acc == 0) acc_phase ^= 1u;
                }
                // every MMA has finished before TMEM is freed
                tc_commit_mc<PAIR>(smem_u32(&ctl->mdone), (uint16_t)0x1);
                drain_bar(smem_u32(&ctl->mdone), 0, kWaitNs, status);
            }
        }
        __syncwarp();
    } else if (warp >= kEpiWarps) {
        // ---------------- converters: each slot rounded in place by its group, 32 rows a warp
        const int cw = warp - kEpiWarps;
        const int grp = cw / kCvtWarpsPerGroup, wq = cw % kCvtWarpsPerGroup;
        for (int64_t u = grp; u < uses; u += kCvtGroups) {
            const int s = (int)(u % NS);
            if (!wait_bar(smem_u32(&ctl->sfull[s]), (uint32_t)((u / NS) & 1), ctl, status)) break;
            convert_slot<F>(slots + s * SLOT_BYTES, 2 * wq, lane);
            convert_slot<F>(slots + s * SLOT_BYTES, 2 * wq + 1, lane);
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) arrive_leader<PAIR>(smem_u32(&ctl->cfull[s]), me);
        }
    } else {
        // ---------------- epilogue: TMEM lane = row of this CTA's 128
        int acc = 0;
        uint32_t acc_phase = 0;
        for (int64_t tt = 0; tt < my_tiles; ++tt) {
            const int64_t t = group + tt * ngroups;
            if (!wait_bar(smem_u32(&ctl->tfull[acc]), acc_phase, ctl, status)) break;
            tc_fence_after();
            float sum = 0.f;
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(acc * kNOut);
            for (int c = 0; c < ne; c += 32) {
                if (c + 32 <= ne) {
                    uint32_t r[32];
                    tmem_ld32(taddr + (uint32_t)c, r);
                    tmem_ld_wait();
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const float y = __uint_as_float(r[j]);
                        sum = fmaf(y, y, sum);
                    }
                } else {
                    uint32_t r[16];
                    tmem_ld16(taddr + (uint32_t)c, r);
                    tmem_ld_wait();
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float y = __uint_as_float(r[j]);
                        sum = fmaf(y, y, sum);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) arrive_leader<PAIR>(smem_u32(&ctl->tempty[acc]), me);
            const int64_t row = t * kGroupRows + (int64_t)me * kTileRows + warp * 32 + lane;
            if (row < n) theta[row] = sum;
            acc ^= 1;
            if (acc == 0) acc_phase ^= 1u;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc_fence_after();
        tmem_dealloc_cg<PAIR>(tmem, 2 * kNOut);
    }
    if (PAIR == 2) {
        // neither CTA leaves while its peer may still signal its mbarriers (bounded)
        if (threadIdx.x == 0) {
            const uint32_t xb = smem_u32(&ctl->xbar);
            mbar_arrive_cluster(xb);
            mbar_arrive_cluster(mapa_shared(xb, me ^ 1u));
            drain_bar(xb, 0, kExitWaitNs, status);
        }
        __syncthreads();
    }
}

// Pack Mfull (d x k FP32, row-major) into the operand image of Mfull^T for an MMA of width N
// (mma_width): per column half h, per K block kb, NT = N / pairs rows (columns q = h NT + row of
// Mfull) of 128 bytes, 128-byte swizzled; split forms store the hi image then the lo image.
template <int F>
__global__ void k_pack_image(const float* __restrict__ M, int d, int k, int nkb, uint8_t* __restrict__ image,
                             uint32_t half_bytes, const int* __restrict__ width) {
    using T = FormTraits<F>;
    const int NT = mma_width(width) / T::kPair;
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
    int rc = handle_scratch(h, 0, (size_t)half_bytes * T::kPair + 16, &ws);
    if (rc != LEV_OK) return rc;
    uint8_t* image = static_cast<uint8_t*>(ws);
    int* width = reinterpret_cast<int*>(image + (size_t)half_bytes * T::kPair);
    cudaError_t e = cudaMemsetAsync(width, 0, sizeof(int), st);
    if (e != cudaSuccess) return handle_fail(LEV_ECUDA, cudaGetErrorString(e));
    k_mfull_width<<<32, 256, 0, st>>>(Mfull, (int)d, (int)k, width);
    k_pack_image<F><<<64, 256, 0, st>>>(Mfull, (int)d, (int)k, nkb, image, half_bytes, width);
    e = cudaGetLastError();
    if (e != cudaSuccess) return handle_fail(LEV_ECUDA, cudaGetErrorString(e));
    CUtensorMap tmA;
    if (!make_map_2d(&tmA, A, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, n, d, lda, 32, kTileRows))
        return handle_fail(LEV_ECUDA, "cuTensorMapEncodeTiled failed for the final pass");
    const size_t smem = 1024 + (size_t)half_bytes + (size_t)T::kSlots * (T::kKbe / 32) * kBoxBytes +
                        sizeof(TcSmemCtl) + 64;
    e = cudaFuncSetAttribute(k_final_tc<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return handle_fail(LEV_ECUDA, cudaGetErrorString(e));
    const int64_t ntiles = (n + (int64_t)kTileRows * T::kPair - 1) / ((int64_t)kTileRows * T::kPair);
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)T::kPair;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = T::kPair == 2 ? 1 : 0;
    // persistent grid: as many CTAs (pairs) as can be resident at once, so that the static tile
    // split never leaves a group waiting for a free SM (or SM pair) behind the others
    int64_t groups = handle_num_sms(h);
    if (T::kPair == 2) {
        static std::atomic<int> cached[64] = {};         // resident clusters per device (host threads share it)
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return handle_fail(LEV_ECUDA, "no current CUDA device");
        int clusters = dev >= 0 && dev < 64 ? cached[dev].load(std::memory_order_relaxed) : 0;
        if (clusters == 0) {
            cfg.gridDim = dim3((unsigned)(groups & ~1));
            e = cudaOccupancyMaxActiveClusters(&clusters, k_final_tc<F>, &cfg);
            if (e != cudaSuccess || clusters < 1)
                return handle_fail(LEV_ECUDA, "no resident 2-CTA cluster for the final pass");
            if (dev >= 0 && dev < 64) cached[dev].store(clusters, std::memory_order_relaxed);
        }
        groups = clusters;
    }
    if (groups > ntiles) groups = ntiles;
    if (groups < 1) groups = 1;
    cfg.gridDim = dim3((unsigned)(groups * T::kPair));
    e = cudaLaunchKernelEx(&cfg, k_final_tc<F>, tmA, n, nkb, (const uint8_t*)image, half_bytes, (const int*)width,
                           theta, status);
    if (e != cudaSuccess) return handle_fail(LEV_ECUDA, cudaGetErrorString(e));
    return LEV_OK;
}

// out (n x ldo) = A (n x d, lda); the columns d..ldo-1 of out are never read (TMA clips at d).
__global__ void k_copy_rows(const float* __restrict__ A, int64_t lda, int64_t n, int d, float* __restrict__ out,
                            int64_t ldo) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * d; e += (int64_t)gridDim.x * blockDim.x)
        out[(e / d) * ldo + (e % d)] = A[(e / d) * lda + (e % d)];
}

}  // namespace

int tc_final_dense(lev_handle* h, const float* A, int64_t n, int64_t d, int64_t lda, const float* Mfull, int64_t k,
                   int32_t prec, float* theta, cudaStream_t st) {
    if (d > 256 || k > 256)
        return handle_fail(LEV_EINVAL, "tensor-core final pass needs d <= 256 and k <= 256");
    if (n == 0) return LEV_OK;
    // TMA reads rows at a 16-byte aligned base with a row stride that is a multiple of 16 bytes;
    // any other A is first copied to a padded buffer of the handle
    if ((reinterpret_cast<uintptr_t>(A) & 15u) != 0 || (lda & 3) != 0) {
        const int64_t ldo = (d + 3) & ~int64_t(3);
        void* buf = nullptr;
        int rc = handle_scratch(h, 3, sizeof(float) * (size_t)n * ldo, &buf);
        if (rc != LEV_OK) return rc;
        int grid = (int)((n * d + 255) / 256);
        if (grid > 152 * 16) grid = 152 * 16;
        k_copy_rows<<<grid, 256, 0, st>>>(A, lda, n, (int)d, static_cast<float*>(buf), ldo);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return handle_fail(LEV_ECUDA, cudaGetErrorString(e));
        A = static_cast<const float*>(buf);
        lda = ldo;
    }
    int32_t* status = handle_status(h);
    switch (prec) {
        case LEV_BF16: return run_final_tc<kBF16>(h, A, n, d, lda, Mfull, k, theta, status, st);
        case LEV_BF16X3: return run_final_tc<kBF16X3>(h, A, n, d, lda, Mfull, k, theta, status, st);
        case LEV_TF32: return run_final_tc<kTF32>(h, A, n, d, lda, Mfull, k, theta, status, st);
        default: return handle_fail(LEV_EINVAL, "unknown tensor-core precision");
    }
}

}  // namespace lev
