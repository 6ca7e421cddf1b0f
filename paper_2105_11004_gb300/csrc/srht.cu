// Subsampled randomized Hadamard transform after the CountSketch (Sec. 3.4.2 and Sec. 4.1):
// C = F B with F = sqrt(s/t) P H D (t x s), applied to B = S A (s x d, FP32, row-major) before the
// Gaussian stage, which then multiplies an m x t Gaussian matrix instead of an m x s one.
//   D: signs from bit 0 of stream 4 at row b;
//   H: the Walsh-Hadamard matrix in Sylvester order scaled by 1/sqrt(s), applied in place as
//      butterflies (x_i, x_{i+h}) -> (x_i + x_{i+h}, x_i - x_{i+h}), h = 1, 2, 4, ..., s/2;
//   P: t independent uniform draws of rows (multiply-shift of the high word of stream 5 at q).
// The butterflies run in passes of at most 9 stages: a CTA holds one group of 2^L rows that the
// pass's stages couple (consecutive rows in the first pass, rows 2^9 apart in the second, ...)
// for 32 columns in shared memory, so each pass reads and writes B once. A gather then scales the
// t drawn rows by 1/sqrt(t) (= sqrt(s/t) / sqrt(s)).
#include <algorithm>

#include "lev_common.cuh"
#include "lev_kernels.cuh"

namespace lev {

namespace {

constexpr int kSrhtMaxStages = 9;          // 2^9 rows x 32 columns x 4 bytes = 64 KB per CTA
constexpr int kSrhtCols = 32;

// Stages h = 2^h0 .. 2^(h0+L-1). Group g couples the rows base + q 2^h0 (q < 2^L) with
// base = (g mod 2^h0) + (g / 2^h0) 2^(h0+L). blockIdx.x is the 32-column tile and blockIdx.y the
// group, so the CTAs that read the same rows run together; a thread moves 4 columns (float4).
// The first pass multiplies row b by its sign, hashed once per row.
__global__ void __launch_bounds__(256) k_fwht_pass(float* __restrict__ B, int64_t s, int d, int L, int h0,
                                                   uint64_t sign_key, int apply_sign, int vec) {
    extern __shared__ float4 sm4[];                                // 2^L rows x 8 float4 (32 columns)
    __shared__ float sgn[1 << kSrhtMaxStages];
    const int c0 = blockIdx.x * kSrhtCols;
    const int64_t g = blockIdx.y;
    const int G = 1 << L;
    const int64_t lo = g & ((int64_t(1) << h0) - 1);
    const int64_t base = lo + ((g >> h0) << (h0 + L));
    const int t = threadIdx.x;
    constexpr int V = kSrhtCols / 4;                               // float4 per row segment
    for (int q = t; q < G; q += blockDim.x)
        sgn[q] = apply_sign ? sign_of(splitmix64(sign_key, (uint64_t)(base + ((int64_t)q << h0)))) : 1.f;
    __syncthreads();
    // every load of the thread is issued before the first is used (the CTA's 64 KB in flight)
    constexpr int IT = (1 << kSrhtMaxStages) * V / 256;
    float4 r[IT];
#pragma unroll
    for (int i = 0; i < IT; ++i) {
        const int e = t + i * 256;
        r[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (e < G * V) {
            const int q = e / V, c = (e % V) * 4;
            const float* src = B + (base + ((int64_t)q << h0)) * d + c0 + c;
            if (vec && c0 + c + 3 < d) {
                r[i] = *reinterpret_cast<const float4*>(src);
            } else {
                r[i].x = c0 + c < d ? src[0] : 0.f;
                r[i].y = c0 + c + 1 < d ? src[1] : 0.f;
                r[i].z = c0 + c + 2 < d ? src[2] : 0.f;
                r[i].w = c0 + c + 3 < d ? src[3] : 0.f;
            }
        }
    }
#pragma unroll
    for (int i = 0; i < IT; ++i) {
        const int e = t + i * 256;
        if (e < G * V) {
            const float sg = sgn[e / V];
            sm4[e] = make_float4(r[i].x * sg, r[i].y * sg, r[i].z * sg, r[i].w * sg);
        }
    }
    __syncthreads();
    for (int j = 0; j < L; ++j) {
        for (int e = t; e < (G / 2) * V; e += blockDim.x) {
            const int pi = e / V, c = e % V;
            const int q0 = ((pi >> j) << (j + 1)) + (pi & ((1 << j) - 1));
            const int q1 = q0 + (1 << j);
            const float4 a = sm4[q0 * V + c], b = sm4[q1 * V + c];
            sm4[q0 * V + c] = make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
            sm4[q1 * V + c] = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
        }
        __syncthreads();
    }
    for (int e = t; e < G * V; e += blockDim.x) {
        const int q = e / V, c = (e % V) * 4;
        float* dst = B + (base + ((int64_t)q << h0)) * d + c0 + c;
        const float4 v = sm4[e];
        if (vec && c0 + c + 3 < d) {
            *reinterpret_cast<float4*>(dst) = v;
        } else {
            if (c0 + c < d) dst[0] = v.x;
            if (c0 + c + 1 < d) dst[1] = v.y;
            if (c0 + c + 2 < d) dst[2] = v.z;
            if (c0 + c + 3 < d) dst[3] = v.w;
        }
    }
}

// Row b of B times its sign D_b (the adjoint applies D after the butterflies).
__global__ void k_row_signs(float* __restrict__ B, int64_t s, int d, uint64_t sign_key) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < s * d; e += (int64_t)gridDim.x * blockDim.x)
        B[e] *= sign_of(splitmix64(sign_key, (uint64_t)(e / d)));
}

// Adjoint scatter, deterministic: count the draws per row of s, order each row's draws by q (counting
// sort, then a rank sort within each row's segment), and sum them in that order.
__global__ void k_srht_hist(int64_t t, uint32_t s, uint64_t rows_key, int* count) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < t; q += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&count[bucket_of(splitmix64(rows_key, (uint64_t)q), s)], 1);
}
__global__ void k_srht_scatter_q(int64_t t, uint32_t s, uint64_t rows_key, const int* off, int* cursor, uint32_t* out) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < t; q += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t b = bucket_of(splitmix64(rows_key, (uint64_t)q), s);
        out[off[b] + atomicAdd(&cursor[b], 1)] = (uint32_t)q;
    }
}
// X[b, :] = sum over the draws q of row b, in increasing q, of Y[q, :] / sqrt(t)
__global__ void k_srht_gather_adj(const float* __restrict__ Y, const int* __restrict__ off,
                                  const uint32_t* __restrict__ ord, int64_t s, int d, float inv_sqrt_t,
                                  float* __restrict__ X) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < s * d; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = e / d;
        const int c = (int)(e % d);
        float acc = 0.f;
        for (int f = off[b]; f < off[b + 1]; ++f) acc += Y[(int64_t)ord[f] * d + c];
        X[e] = acc * inv_sqrt_t;
    }
}

// C[q, :] = B[pi(q), :] / sqrt(t), pi(q) the q-th row draw.
__global__ void k_srht_gather(const float* __restrict__ B, int64_t s, int d, int64_t t, uint64_t rows_key,
                              float inv_sqrt_t, float* __restrict__ C) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < t * d; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = e / d;
        const int c = (int)(e % d);
        const int64_t row = bucket_of(splitmix64(rows_key, (uint64_t)q), (uint32_t)s);
        C[e] = B[row * d + c] * inv_sqrt_t;
    }
}

}  // namespace

// H' B in place (the unnormalised Walsh-Hadamard transform of the columns), with B first multiplied
// by the signs D when sign_key is nonzero.
static cudaError_t launch_fwht(float* B, int64_t s, int64_t d, uint64_t sign_key, bool apply_sign, cudaStream_t st) {
    int p = 0;
    while ((int64_t(1) << p) < s) ++p;
    if ((int64_t(1) << p) != s || p > 24) return cudaErrorInvalidValue;   // groups fit grid.y
    const size_t smem = sizeof(float) * ((size_t)1 << kSrhtMaxStages) * kSrhtCols;
    cudaError_t e = cudaFuncSetAttribute(k_fwht_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned tiles = (unsigned)((d + kSrhtCols - 1) / kSrhtCols);
    const int vec = ((reinterpret_cast<uintptr_t>(B) & 15u) == 0 && (d & 3) == 0) ? 1 : 0;
    int h0 = 0;
    do {                                                           // s = 1 still takes one pass (the sign)
        const int L = p - h0 < kSrhtMaxStages ? p - h0 : kSrhtMaxStages;
        const int64_t groups = s >> L;
        k_fwht_pass<<<dim3(tiles, (unsigned)groups), 256, sizeof(float) * ((size_t)1 << L) * kSrhtCols, st>>>(
            B, s, (int)d, L, h0, sign_key, (h0 == 0 && apply_sign) ? 1 : 0, vec);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        h0 += L;
    } while (h0 < p);
    return cudaSuccess;
}

cudaError_t launch_srht(float* B, int64_t s, int64_t d, int64_t t, uint64_t seed, float* C, cudaStream_t st) {
    if (t < 1 || t > s) return cudaErrorInvalidValue;
    const uint64_t sign_key = stream_key(seed, kStreamSrhtSign), rows_key = stream_key(seed, kStreamSrhtRows);
    cudaError_t e = launch_fwht(B, s, d, sign_key, true, st);
    if (e != cudaSuccess) return e;
    int grid = (int)((t * d + 255) / 256);
    if (grid > 152 * 16) grid = 152 * 16;
    k_srht_gather<<<grid, 256, 0, st>>>(B, s, (int)d, t, rows_key, (float)(1.0 / sqrt((double)t)), C);
    return cudaGetLastError();
}

cudaError_t launch_srht_adjoint(const float* Y, int64_t s, int64_t d, int64_t t, uint64_t seed, int* count, int* off,
                                uint32_t* tmp, uint32_t* ord, float* X, cudaStream_t st) {
    if (t < 1 || t > s || t > (int64_t(1) << 31)) return cudaErrorInvalidValue;
    const uint64_t sign_key = stream_key(seed, kStreamSrhtSign), rows_key = stream_key(seed, kStreamSrhtRows);
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int) * (size_t)(s + 1), st);
    if (e != cudaSuccess) return e;
    const int gq = (int)std::min<int64_t>((t + 255) / 256, 152 * 8);
    k_srht_hist<<<gq, 256, 0, st>>>(t, (uint32_t)s, rows_key, count);
    if ((e = launch_scan_offsets(count, off, s, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(count, 0, sizeof(int) * (size_t)(s + 1), st)) != cudaSuccess) return e;
    k_srht_scatter_q<<<gq, 256, 0, st>>>(t, (uint32_t)s, rows_key, off, count, tmp);
    if ((e = launch_segment_sort(off, s, tmp, ord, st)) != cudaSuccess) return e;
    const int gx = (int)std::min<int64_t>((s * d + 255) / 256, 152 * 16);
    k_srht_gather_adj<<<gx, 256, 0, st>>>(Y, off, ord, s, (int)d, (float)(1.0 / sqrt((double)t)), X);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_fwht(X, s, d, 0, false, st)) != cudaSuccess) return e;
    k_row_signs<<<gx, 256, 0, st>>>(X, s, (int)d, sign_key);
    return cudaGetLastError();
}

}  // namespace lev
