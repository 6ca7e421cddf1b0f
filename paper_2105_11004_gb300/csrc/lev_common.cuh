// Common device helpers of the leverage-score library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lev.h"

namespace lev {

// ---------------------------------------------------------------------------
// Counter-based random streams (definitions in lev.h).
// splitmix64 (Steele, Lea and Flood 2014) evaluated as a pure function of
// (key, counter): state = key + (c+1) * golden, then the 64-bit finaliser.
// ---------------------------------------------------------------------------
constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kStreamMul = 0xD1B54A32D192ED03ull;
constexpr int kStreamHash = 1, kStreamG = 2, kStreamOmega = 3, kStreamSrhtSign = 4, kStreamSrhtRows = 5;

__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t key, uint64_t c) {
    uint64_t z = key + (c + 1ull) * kGolden;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t stream_key(uint64_t seed, int t) {
    return seed ^ ((uint64_t)t * kStreamMul);
}

// CountSketch hash of row i (Sec. 3.4.3): bucket by multiply-shift of the high
// word, sign from bit 0.
__device__ __forceinline__ uint32_t bucket_of(uint64_t x, uint32_t s) {
    return (uint32_t)(((x >> 32) * (uint64_t)s) >> 32);
}
__device__ __forceinline__ float sign_of(uint64_t x) { return (x & 1ull) ? -1.0f : 1.0f; }

// Box-Muller standard normal, cosine branch, FP64 (CUDA's log/sqrt/cospi).
__device__ __forceinline__ double box_muller(uint64_t key, uint64_t c) {
    uint64_t x1 = splitmix64(key, 2ull * c);
    uint64_t x2 = splitmix64(key, 2ull * c + 1ull);
    double u1 = (double)((x1 >> 11) + 1ull) * 0x1.0p-53;
    double u2 = (double)(x2 >> 11) * 0x1.0p-53;
    return sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}

// The same draw in FP32 arithmetic, within a few FP32 ulp of the FP64 draw (the entries of G:
// 1e9 of them at the largest sketch, where FP64's 1/64 rate would dominate the generation).
// The 53-bit integers behind u1 and u2 are kept exact until one final conversion each:
//  * ln u1: logf(u1) for u1 <= 1/2; log1pf(-t) with t = 1 - u1 = (2^53 - 1 - a) 2^-53 above, so
//    that ln u1 keeps its relative accuracy as u1 -> 1 (a = x1 >> 11, u1 = (a + 1) 2^-53);
//  * cos(2 pi u2) = cos(2 pi v), v = min(u2, 1 - u2) = b' 2^-53 in [0, 1/2]: cospi(2 v) for
//    v < 1/8, else sinpi(1/2 - 2 v) with 1/2 - 2 v = (2^51 - b') 2^-52 formed in integers, so
//    that the result keeps its relative accuracy near the zero at v = 1/4.
__device__ __forceinline__ float box_muller_f32(uint64_t key, uint64_t c) {
    const uint64_t a = splitmix64(key, 2ull * c) >> 11;
    const uint64_t b = splitmix64(key, 2ull * c + 1ull) >> 11;
    const uint64_t top = 1ull << 53;
    float L;
    if (a + 1ull <= (top >> 1))
        L = logf((float)(a + 1ull) * 0x1.0p-53f);
    else
        L = log1pf(-(float)(top - 1ull - a) * 0x1.0p-53f);
    const float r = sqrtf(-2.0f * L);
    const uint64_t bp = b <= (top >> 1) ? b : top - b;                     // v = bp 2^-53
    float cs;
    if (bp < (1ull << 50))
        cs = cospif((float)bp * 0x1.0p-52f);
    else
        cs = sinpif((float)((int64_t)(1ull << 51) - (int64_t)bp) * 0x1.0p-52f);
    return r * cs;
}

// ---------------------------------------------------------------------------
// Device status word: bounded waits record why they gave up, then return.
// ---------------------------------------------------------------------------
constexpr int32_t kStatusTimeoutBarrier = 1;
constexpr long long kSpinLimit = 1ll << 22;     // x >= 256 ns sleep: about 1-2 s at most

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_volatile(const int32_t* p) {
    return *(const volatile int32_t*)p;
}

// Grid-wide barrier for a cooperatively launched grid (all CTAs co-resident).
// `count` is zeroed before the launch and only grows; `epoch` is the number
// of barriers this CTA has passed (same in every CTA). The wait is bounded:
// on timeout the status word is set and false is returned everywhere after.
__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned& epoch, int32_t* status) {
    __syncthreads();
    if (threadIdx.x == 0) {
        epoch += 1;
        const unsigned target = epoch * gridDim.x;
        __threadfence();
        atomicAdd(count, 1u);
        long long spins = 0;
        while (ld_acquire_gpu(count) < target) {
            if (ld_volatile(status) != 0) break;
            if (++spins > kSpinLimit) { atomicExch(status, kStatusTimeoutBarrier); break; }
            __nanosleep(256);
        }
        __threadfence();
    } else {
        epoch += 1;
    }
    __syncthreads();
    return ld_volatile(status) == 0;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace lev
