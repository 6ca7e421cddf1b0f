// Tensor-core (tcgen05, sm_103a) form of the fused final pass (Alg. 8 step 5):
// theta~_i = ||A_i Mfull||^2 with the product accumulated in TMEM and squared
// in the epilogue, so the n x k product never reaches memory.
//
// One persistent CTA per SM (BF16) or per SM of a 2-CTA cluster (BF16X3, TF32).
// Shared memory holds the CTA's part of the packed operand image of Mfull^T (the
// B operand) and a ring of landing slots; a slot holds one K block of the CTA's
// 128 rows of A in FP32. Tensor memory holds one accumulator (256 columns) and
// a ring of A buffers: K blocks of the rows of A rounded to the operand type,
// the MMAs' A operand.
//   * warp 17 (producer): 2-D tensor TMA of a slot's FP32 boxes (32 columns x
//     128 rows each, 128-byte swizzle);
//   * warps 8..15 (converters, two per TMEM lane quarter, each half of a K
//     block), lane = row: read the row's FP32 values, free the slot (its bytes
//     are in registers), round them (BF16 hi, BF16 lo, or TF32) and store them
//     into the fill's A buffer with tcgen05.st once the MMAs of the buffer's
//     previous fill have finished. A slot is busy only from its copy to its
//     read; the A buffers (4 for the split form, 8 otherwise) decouple the
//     converters from the MMAs;
//   * warp 16 (MMA): allocates TMEM, loads the image once with bulk copies, and
//     one thread issues tcgen05.mma with A from TMEM and B from shared memory
//     (N = the width of Mfull, 32 bytes of K per instruction); the MMA
//     completion frees the A buffer;
//   * warps 0..7 (epilogue, two per TMEM lane quarter, each half of the
//     columns): tcgen05.ld of the accumulator (TMEM lane = row), sums of squares,
//     one store per row; then the MMAs of the next tile may overwrite it.
// N: Mfull's columns up to its last nonzero one, rounded up to 16 (k_mfull_width
// finds it on the device). Trailing zero columns add nothing to theta~; the
// r-column factor of lev_omega_factor's reduced form leaves k - r of them.
// BF16: M = 128 per CTA; the 128 KB image of Mfull^T (256 x 256 BF16) fits one
// CTA. BF16X3 (hi*hi + lo*hi + hi*lo) and TF32 need 256 KB for the image, so
// they run as CTA pairs with cta_group::2: one thread of the even CTA issues an
// M = 256 MMA for the pair; each CTA holds its own 128 rows of A (in its TMEM)
// and half of the image (half of Mfull's columns), and each CTA's TMEM receives
// its own rows with all N columns. Nothing is loaded twice and no operand
// crosses between the CTAs except through the MMA itself. The odd CTA reports
// "A buffer written" and "accumulator drained" to the even CTA's mbarriers; MMA
// completions are multicast to both. Every wait is bounded (2 s of
// %globaltimer); on expiry the CTA records the failure in the status word and
// leaves its loops.
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
// Epilogue and converters: eight warps each, two per TMEM lane quarter (warp mod 4). An epilogue
// warp reads half of the accumulator columns of its quarter's 32 rows; a converter warp rounds half
// of each K block of them, and takes every slot fill in order.
constexpr int kEpiWarps = 8, kCvtWarps = 8;
constexpr int kMmaWarp = kEpiWarps + kCvtWarps;   // warp 16
constexpr int kTmaWarp = kMmaWarp + 1;            // warp 17
constexpr int kThreads = (kTmaWarp + 1) * 32;     // 576
constexpr int kMaxSlots = 6;
constexpr int kMaxAbufs = 8;
constexpr uint64_t kWaitNs = 2000000000ull;       // 2 s
constexpr uint64_t kExitWaitNs = 5000000000ull;   // 5 s: a peer that timed out reaches the exit within one kWaitNs
constexpr int32_t kStatusTcTimeout = 2;

struct TcSmemCtl {
    uint64_t sfull[kMaxSlots], sempty[kMaxSlots], afull[kMaxAbufs], aempty[kMaxAbufs], tfull, tempty, mfull, ipeer,
        mdone, xbar;
    uint64_t pfull[2], pempty[2];
    float part[2][kTileRows];   // the second column half's sums of squares, by tile parity
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

// Relaxed arrival on the mbarrier at `bar` in the even CTA of the pair (this CTA when unpaired):
// hands over tensor-memory data (written, or read, and fenced by the caller).
template <int PAIR>
__device__ __forceinline__ void arrive_leader_tmem(uint32_t bar, uint32_t me) {
    if (PAIR == 2 && me != 0)
        mbar_arrive_relaxed_cluster(mapa_shared(bar, 0));
    else
        mbar_arrive_relaxed(bar);
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

// *width = 1 + the last column of Mfull (d x k, k <= 256) holding a nonzero (or NaN) entry; 0 if
// none (*width zeroed before). Block y covers rows y, y + gridDim.y, ...; thread x column x.
__global__ void k_mfull_width(const float* __restrict__ M, int d, int k, int* width) {
    __shared__ int wmax;
    if (threadIdx.x == 0) wmax = 0;
    __syncthreads();
    int w = 0;
    const int q = threadIdx.x;
    if (q < k)
        for (int i = blockIdx.y; i < d; i += gridDim.y)
            if (M[(int64_t)i * k + q] != 0.f) w = q + 1;
    w = (int)__reduce_max_sync(0xffffffffu, (unsigned)w);
    if ((threadIdx.x & 31) == 0 && w > 0) atomicMax(&wmax, w);
    __syncthreads();
    if (threadIdx.x == 0 && wmax > 0) atomicMax(width, wmax);
}

// Half a K block of this lane's row of A (columns 32 h .. 32 h + 31 of a BF16 K block, 16 h .. 16 h
// + 15 of a TF32 one): its FP32 values from the slot, then rounded to operand words, two BF16 or
// one TF32 a word, lower K first: hi[0..16) and, for the split form, lo[0..16).
template <int F>
struct HalfRow {
    static constexpr int kVec = FormTraits<F>::kKbe / 8;         // float4 per half row
    float4 x[kVec];
};
template <int F>
__device__ __forceinline__ void load_half_row(const uint8_t* slot, uint32_t row, int h, HalfRow<F>& v) {
#pragma unroll
    for (int q = 0; q < HalfRow<F>::kVec; ++q) {
        const int g = h * HalfRow<F>::kVec + q;                   // 16-byte chunk of the row's K block
        v.x[q] = *reinterpret_cast<const float4*>(slot + (g >> 3) * kBoxBytes + sw128_offset(row, (uint32_t)(g & 7) * 16u));
    }
}
template <int F>
struct HalfWords {
    uint32_t hi[16];
    uint32_t lo[FormTraits<F>::kSplit ? 16 : 1];
};
template <int F>
__device__ __forceinline__ void round_half_row(const HalfRow<F>& v, HalfWords<F>& w) {
    using T = FormTraits<F>;
#pragma unroll
    for (int q = 0; q < HalfRow<F>::kVec; ++q) {
        const float4 x = v.x[q];
        if constexpr (T::kTf32) {
            w.hi[4 * q + 0] = f32_to_tf32(x.x);
            w.hi[4 * q + 1] = f32_to_tf32(x.y);
            w.hi[4 * q + 2] = f32_to_tf32(x.z);
            w.hi[4 * q + 3] = f32_to_tf32(x.w);
        } else {
            float r0, r1, r2, r3;
            w.hi[2 * q] = pack_bf16x2(x.x, x.y, &r0, &r1);
            w.hi[2 * q + 1] = pack_bf16x2(x.z, x.w, &r2, &r3);
            if constexpr (T::kSplit) {
                float u0, u1;
                w.lo[2 * q] = pack_bf16x2(r0, r1, &u0, &u1);
                w.lo[2 * q + 1] = pack_bf16x2(r2, r3, &u0, &u1);
            }
        }
    }
}

// Sum of the squares of `cols` (a multiple of 16) consecutive accumulator columns of this thread's
// TMEM lane from taddr on: two 32-column loads in flight per wait, then the 32- and 16-column rest,
// summed in four independent chains (combined as (s0 + s1) + (s2 + s3)). release() runs once, right
// after the last load has completed, so that the accumulator is handed back before the last sums.
template <class Release>
__device__ __forceinline__ float tmem_sum_squares(uint32_t taddr, int cols, Release&& release) {
    if (cols <= 0) {
        release();
        return 0.f;
    }
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    int c = 0;
    for (; c + 64 <= cols; c += 64) {
        uint32_t r[32], q[32];
        tmem_ld32(taddr + (uint32_t)c, r);
        tmem_ld32(taddr + (uint32_t)c + 32u, q);
        tmem_ld_wait();
        if (c + 64 == cols) release();
#pragma unroll
        for (int j = 0; j < 32; j += 2) {
            const float y0 = __uint_as_float(r[j]), y1 = __uint_as_float(r[j + 1]);
            const float z0 = __uint_as_float(q[j]), z1 = __uint_as_float(q[j + 1]);
            s0 = fmaf(y0, y0, s0);
            s1 = fmaf(y1, y1, s1);
            s2 = fmaf(z0, z0, s2);
            s3 = fmaf(z1, z1, s3);
        }
    }
    for (; c + 32 <= cols; c += 32) {
        uint32_t r[32];
        tmem_ld32(taddr + (uint32_t)c, r);
        tmem_ld_wait();
        if (c + 32 == cols) release();
#pragma unroll
        for (int j = 0; j < 32; j += 4) {
            s0 = fmaf(__uint_as_float(r[j]), __uint_as_float(r[j]), s0);
            s1 = fmaf(__uint_as_float(r[j + 1]), __uint_as_float(r[j + 1]), s1);
            s2 = fmaf(__uint_as_float(r[j + 2]), __uint_as_float(r[j + 2]), s2);
            s3 = fmaf(__uint_as_float(r[j + 3]), __uint_as_float(r[j + 3]), s3);
        }
    }
    if (c < cols) {                                               // the last 16 columns
        uint32_t r[16];
        tmem_ld16(taddr + (uint32_t)c, r);
        tmem_ld_wait();
        release();
#pragma unroll
        for (int j = 0; j < 16; j += 4) {
            s0 = fmaf(__uint_as_float(r[j]), __uint_as_float(r[j]), s0);
            s1 = fmaf(__uint_as_float(r[j + 1]), __uint_as_float(r[j + 1]), s1);
            s2 = fmaf(__uint_as_float(r[j + 2]), __uint_as_float(r[j + 2]), s2);
            s3 = fmaf(__uint_as_float(r[j + 3]), __uint_as_float(r[j + 3]), s3);
        }
    }
    return (s0 + s1) + (s2 + s3);
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
    constexpr uint32_t kAcols = T::kSplit ? 64u : 32u;        // TMEM columns of one K block of A
    constexpr uint32_t kAbase = kNOut;                        // A buffers after the accumulator
    constexpr int NA = (int)((512u - kAbase) / kAcols);       // A buffers: 4 (split form) or 8
    constexpr uint32_t kKstepCols = 8u;                       // TMEM columns of A per MMA (32 bytes of K)
    static_assert(T::kNt * PAIR == kNOut, "the image holds up to 256 columns of Mfull");
    static_assert(NS <= kMaxSlots && NA <= kMaxAbufs, "slot and A-buffer barriers");
    const int ne = mma_width(width);                          // MMA N
    const uint32_t IDESC = make_idesc(T::kTf32, kTileRows * PAIR, ne);
    const uint32_t kb_img_bytes = (uint32_t)(ne / PAIR) * 128u;   // one K block of this CTA's image
    const uint32_t img_used = (uint32_t)nkb * kb_img_bytes * (T::kSplit ? 2u : 1u);
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
            mbar_init(smem_u32(&ctl->sempty[s]), kCvtWarps);
        }
        for (int b = 0; b < NA; ++b) {
            mbar_init(smem_u32(&ctl->afull[b]), kCvtWarps * PAIR);
            mbar_init(smem_u32(&ctl->aempty[b]), 1);
        }
        mbar_init(smem_u32(&ctl->tfull), 1);
        mbar_init(smem_u32(&ctl->tempty), kEpiWarps * PAIR);
        for (int a = 0; a < 2; ++a) {
            mbar_init(smem_u32(&ctl->pfull[a]), kEpiWarps / 2);
            mbar_init(smem_u32(&ctl->pempty[a]), kEpiWarps / 2);
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
        tmem_alloc_cg<PAIR>(smem_u32(&ctl->tmem_base), 512);
        tmem_relinquish_cg<PAIR>();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = ctl->tmem_base;

    if (warp == kTmaWarp) {
        // ---------------- producer: this CTA's 128 rows of one K block per slot
        if (lane == 0) {
            int64_t issued = 0;
            for (int64_t u = 0; u < uses; ++u) {
                const int s = (int)(u % NS);
                if (!wait_bar(smem_u32(&ctl->sempty[s]), (uint32_t)((u / NS) & 1) ^ 1u, ctl, status)) break;
                const int64_t t = group + (u / nkb) * ngroups;
                const int32_t x = (int32_t)(u % nkb) * T::kKbe;
                const int32_t y = (int32_t)(t * kGroupRows + (int64_t)me * kTileRows);
                const uint32_t bar = smem_u32(&ctl->sfull[s]);
                mbar_arrive_expect_tx(bar, (uint32_t)SLOT_BYTES);
                const uint32_t dst = smem_u32(slots + s * SLOT_BYTES);
#pragma unroll
                for (int b = 0; b < BOXES; ++b) tma_load_2d(dst + b * kBoxBytes, &tmA, x + b * 32, y, bar);
                ++issued;
            }
            // no copy may still be landing in this CTA's shared memory when it exits
            for (int64_t j = issued > NS ? issued - NS : 0; j < issued; ++j)
                drain_bar(smem_u32(&ctl->sfull[j % NS]), (uint32_t)((j / NS) & 1), kWaitNs, status);
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
                const uint32_t img_addr = smem_u32(img);
                const uint16_t both = (uint16_t)(PAIR == 2 ? 0x3 : 0x1);
                for (int64_t tt = 0; ok && tt < my_tiles; ++tt) {
                    // the epilogue has read the previous tile's accumulator
                    if (!wait_bar(smem_u32(&ctl->tempty), (uint32_t)(tt & 1) ^ 1u, ctl, status)) { ok = false; break; }
                    tc_fence_after();
                    for (int kb = 0; kb < nkb; ++kb) {
                        const int64_t u = tt * nkb + kb;
                        const int b = (int)(u % NA);
                        if (!wait_bar(smem_u32(&ctl->afull[b]), (uint32_t)((u / NA) & 1), ctl, status)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t a_hi = tmem + kAbase + (uint32_t)b * kAcols;
                        const uint32_t m_hi = img_addr + (uint32_t)kb * kb_img_bytes;
#pragma unroll
                        for (int ks = 0; ks < 4; ++ks) {
                            const uint32_t acol = (uint32_t)ks * kKstepCols, koff = (uint32_t)ks * 32u;
                            const uint32_t accum = (kb | ks) != 0 ? 1u : 0u;
                            tc_mma_ts<PAIR, T::kTf32>(tmem, a_hi + acol, sw128_desc(m_hi + koff), IDESC, accum);
                            if constexpr (T::kSplit) {
                                const uint32_t a_lo = a_hi + 32u;
                                const uint32_t m_lo = m_hi + (uint32_t)nkb * kb_img_bytes;
                                tc_mma_ts<PAIR, false>(tmem, a_lo + acol, sw128_desc(m_hi + koff), IDESC, 1u);
                                tc_mma_ts<PAIR, false>(tmem, a_hi + acol, sw128_desc(m_lo + koff), IDESC, 1u);
                            }
                        }
                        // A buffer b is free again in both CTAs once these MMAs finish
                        tc_commit_mc<PAIR>(smem_u32(&ctl->aempty[b]), both);
                    }
                    if (!ok) break;
                    tc_commit_mc<PAIR>(smem_u32(&ctl->tfull), both);
                }
                // every MMA has finished before TMEM is freed
                tc_commit_mc<PAIR>(smem_u32(&ctl->mdone), (uint16_t)0x1);
                drain_bar(smem_u32(&ctl->mdone), 0, kWaitNs, status);
            }
        }
        __syncwarp();
    } else if (warp >= kEpiWarps) {
        // ---------------- converters: lane = row of the warp's lane quarter, half h of each K block
        const int cw = warp - kEpiWarps;                      // kEpiWarps is a multiple of 4
        const int wq = cw & 3, h = cw >> 2;                   // wq = warp mod 4: the TMEM lanes it may access
        const uint32_t row = (uint32_t)(wq * 32 + lane);
        const uint32_t lane_addr = tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)h * 16u;
        for (int64_t u = 0; u < uses; ++u) {
            const int s = (int)(u % NS), b = (int)(u % NA);
            if (!wait_bar(smem_u32(&ctl->sfull[s]), (uint32_t)((u / NS) & 1), ctl, status)) break;
            HalfRow<F> v;
            load_half_row<F>(slots + s * SLOT_BYTES, row, h, v);
            HalfWords<F> w;
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&ctl->sempty[s]));      // the slot's bytes are in registers
            round_half_row<F>(v, w);
            // the MMAs that read A buffer b for fill u - NA have finished (both CTAs)
            if (!wait_bar(smem_u32(&ctl->aempty[b]), (uint32_t)((u / NA) & 1) ^ 1u, ctl, status)) break;
            tc_fence_after();
            const uint32_t a = lane_addr + kAbase + (uint32_t)b * kAcols;
            tmem_st16(a, w.hi);
            if constexpr (T::kSplit) tmem_st16(a + 32u, w.lo);
            tmem_st_wait();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) arrive_leader_tmem<PAIR>(smem_u32(&ctl->afull[b]), me);
        }
        // the MMA completions multicast to this CTA's A-buffer barriers have all landed
        if (cw == 0 && lane == 0 && !*(volatile int32_t*)&ctl->abort) {
            for (int q = 0; q < NA; ++q) {
                const int64_t k_uses = uses / NA + (q < uses % NA ? 1 : 0);
                if (k_uses > 0) drain_bar(smem_u32(&ctl->aempty[q]), (uint32_t)((k_uses - 1) & 1), kWaitNs, status);
            }
        }
    } else {
        // ---------------- epilogue: TMEM lane = row of this CTA's 128; warp w reads columns
        // [0, split) (w < 4) or [split, ne) (w >= 4) of rows 32 (w mod 4) .. + 31
        const int wq = warp & 3, eh = warp >> 2;
        const int split = min(ne, 64 * ((ne + 127) / 128));   // a multiple of 64 (or all of ne)
        const uint32_t lanes = tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)(eh ? split : 0);
        const int cols = eh ? ne - split : split;
        for (int64_t tt = 0; tt < my_tiles; ++tt) {
            const int64_t t = group + tt * ngroups;
            if (!wait_bar(smem_u32(&ctl->tfull), (uint32_t)(tt & 1), ctl, status)) break;
            tc_fence_after();
            // the accumulator goes back to the MMA warp as soon as its last columns are read
            const float sum = tmem_sum_squares(lanes, cols, [&] {
                tc_fence_before();
                __syncwarp();
                if (lane == 0) arrive_leader_tmem<PAIR>(smem_u32(&ctl->tempty), me);
            });
            // the second column half's warps hand their sums to the first's through part[tt & 1]
            // (two buffers; each is refilled once the first half has read it)
            const int pb = (int)(tt & 1);
            const uint32_t pph = (uint32_t)((tt >> 1) & 1);
            float* part = ctl->part[pb];
            if (eh) {
                if (!wait_bar(smem_u32(&ctl->pempty[pb]), pph ^ 1u, ctl, status)) break;
                part[wq * 32 + lane] = sum;
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&ctl->pfull[pb]));
            } else {
                if (!wait_bar(smem_u32(&ctl->pfull[pb]), pph, ctl, status)) break;
                const float other = part[wq * 32 + lane];
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&ctl->pempty[pb]));
                const int64_t row = t * kGroupRows + (int64_t)me * kTileRows + wq * 32 + lane;
                if (row < n) theta[row] = sum + other;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc_fence_after();
        tmem_dealloc_cg<PAIR>(tmem, 512);
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
    const int per_half = nkb * NT * T::kKbe;                   // at most 2^16 entries (d, k <= 256)
    const int total = per_half * T::kPair;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int h = e / per_half;
        int rem = e - h * per_half;
        const int kb = rem / (NT * T::kKbe);
        rem -= kb * (NT * T::kKbe);
        const int nl = rem / T::kKbe, el = rem % T::kKbe;
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
    k_mfull_width<<<dim3(1, 64), 256, 0, st>>>(Mfull, (int)d, (int)k, width);
    k_pack_image<F><<<256, 256, 0, st>>>(Mfull, (int)d, (int)k, nkb, image, half_bytes, width);
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
    const cudaEvent_t* marks = handle_final_marks(h);
    if (marks && (e = cudaEventRecord(marks[0], st)) != cudaSuccess) return handle_fail(LEV_ECUDA, cudaGetErrorString(e));
    e = cudaLaunchKernelEx(&cfg, k_final_tc<F>, tmA, n, nkb, (const uint8_t*)image, half_bytes, (const int*)width,
                           theta, status);
    if (e != cudaSuccess) return handle_fail(LEV_ECUDA, cudaGetErrorString(e));
    if (marks && (e = cudaEventRecord(marks[1], st)) != cudaSuccess) return handle_fail(LEV_ECUDA, cudaGetErrorString(e));
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
