// Rank-revealing QR of the sketch through its Gram matrix (FP64), sm_103a.
//
// The pivoted QR of Alg. 4 (xGEQP3-style greatest-trailing-norm pivoting, Sec. 6)
// and the pivoted Cholesky factorisation of G = A~^T A~ produce the same
// permutation, rank and R in exact arithmetic: the squared trailing column
// norms of the QR are the diagonal of the Schur complement of G, and the rows
// of R are the scaled pivot rows of that Schur complement. On a GPU whose FP64
// rate is low, this moves the m d^2 FP64 work into one embarrassingly parallel
// product and leaves only d^3/3 of sequential work on a d x d matrix:
//
//   k_gram_fp64 / k_gram_reduce: G = A~^T A~, FP64 products of the FP32 sketch
//     entries (exact) accumulated in FP64, upper 32 x 32 tiles split over rows,
//     split partials reduced in a fixed order and mirrored;
//   k_pchol: one thread-block cluster of CL CTAs holds the Schur complement in
//     distributed shared memory (CTA c owns the columns l = c mod CL). Every CTA
//     keeps a replicated copy of the Schur diagonal, updated with the same FMAs
//     as the owners' columns, so every CTA takes the same pivot p_j (largest
//     diagonal, ties to the lowest column) and the same rank decision
//     S_pp <= tau^2 S_00 without exchanging them. Step j: wait (bounded) until
//     the owner of column p_j has published it, copy it (DSMEM), write row j of
//     R for the own columns, update the own columns; the owner of the next
//     pivot updates that column first and publishes its progress, so the chain
//     of dependent steps costs one DSMEM round trip, not a cluster barrier.
//
// The Gram route resolves |R_jj| / |R_00| down to about sqrt(m u) ~ 1e-7; the
// caller uses the Householder kernel when tau is below 1e-6 or d > 512.
#include <climits>

#include "lev_common.cuh"
#include "lev_kernels.cuh"

namespace lev {

namespace {

constexpr int GT = 32;                 // Gram tile
constexpr uint64_t kClusterWaitNs = 2000000000ull;
constexpr int32_t kStatusClusterTimeout = 3;
constexpr int64_t kClusterMaxD = 512;   // larger Gram matrices do not fit one cluster's shared memory

__host__ __device__ inline int gram_tiles(int d) {
    const int nt = (d + GT - 1) / GT;
    return nt * (nt + 1) / 2;
}

__device__ inline void tile_coords(int t, int nt, int& bi, int& bj) {
    bi = 0;
    while (t >= nt - bi) { t -= nt - bi; ++bi; }
    bj = bi + t;
}

__global__ void __launch_bounds__(256) k_gram_fp64(const float* __restrict__ At, int m, int d, int rows_per_split,
                                                   double* __restrict__ Gp) {
    // 16 rows of the two column panels per stage, converted to FP64 once when staged
    __shared__ double As[16][GT];
    __shared__ double Bs[16][GT];
    const int nt = (d + GT - 1) / GT;
    const int T = nt * (nt + 1) / 2;
    int bi, bj;
    tile_coords(blockIdx.x, nt, bi, bj);
    const int split = blockIdx.y;
    const int r_begin = split * rows_per_split, r_end = min(m, r_begin + rows_per_split);
    const int t = threadIdx.x;
    const int ty = t >> 3, tx = t & 7;           // 32 x 8 threads -> outputs (ty, tx*4 .. tx*4+3)
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int r0 = r_begin; r0 < r_end; r0 += 16) {
        for (int e = t; e < 16 * GT; e += 256) {
            const int r = e / GT, c = e % GT;
            const int row = r0 + r;
            const bool rok = row < r_end;
            As[r][c] = (rok && bi * GT + c < d) ? (double)At[(int64_t)row * d + bi * GT + c] : 0.0;
            Bs[r][c] = (rok && bj * GT + c < d) ? (double)At[(int64_t)row * d + bj * GT + c] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const double a = As[r][ty];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = fma(a, Bs[r][tx * 4 + q], acc[q]);
        }
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

// ---------------------------------------------------------------- cluster helpers

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t mapa_u32(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
__device__ __forceinline__ double ld_dsmem_f64(uint32_t addr) {
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ int ld_dsmem_s32(uint32_t addr) {
    int v;
    asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ void cluster_hw_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

struct PcholCtl {
    unsigned progress;   // step t whose pivot column (owned here) is final; read by peers
    int abort;
    uint64_t mbar;       // final cluster barrier
};

__device__ __forceinline__ unsigned ld_acquire_dsmem_u32(uint32_t addr) {
    unsigned v;
    asm volatile("ld.acquire.cluster.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_cta_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.cluster.shared::cta.u32 [%0], %1;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(p))),
                 "r"(v)
                 : "memory");
}

// Bounded final cluster barrier (no CTA leaves while a peer may still read its
// shared memory): thread 0 arrives on every CTA's barrier and waits on its own.
__device__ void cluster_exit_barrier(PcholCtl* ctl, int CL, int32_t* status) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t local = static_cast<uint32_t>(__cvta_generic_to_shared(&ctl->mbar));
        for (int c = 0; c < CL; ++c) {
            const uint32_t ra = mapa_u32(local, (uint32_t)c);
            asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(ra) : "memory");
        }
        const uint64_t t0 = gtimer();
        for (uint32_t it = 0;; ++it) {
            uint32_t ok;
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
                "selp.u32 %0, 1, 0, p;\n\t}"
                : "=r"(ok)
                : "r"(local), "r"(0u)
                : "memory");
            if (ok) break;
            if ((it & 31u) == 31u && gtimer() - t0 > kClusterWaitNs) {
                atomicExch(status, kStatusClusterTimeout);
                break;
            }
        }
    }
    __syncthreads();
}

// Pivoted Cholesky of G (d x d FP64, symmetric) on one cluster of CL CTAs.
// Every CTA keeps a replicated copy of the Schur diagonal, updated with the
// same FMAs as the owners' columns, so all CTAs take the same pivots without
// exchanging them. The owner of the next pivot updates that column first and
// then publishes its progress; readers wait (bounded) only for that owner.
template <int CL>
__global__ void __launch_bounds__(256, 1) k_pchol(const double* __restrict__ G, int d, int m, double tau,
                                                  const int32_t* __restrict__ forced, int forced_rank,
                                                  double* __restrict__ Rorig, int32_t* __restrict__ piv,
                                                  int64_t* __restrict__ rank_out, int32_t* status) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int ncl = (d + CL - 1) / CL;
    double* S = reinterpret_cast<double*>(smem);                  // ncl x d, column l = lc*CL + me
    double* rbuf = S + (size_t)ncl * d;                           // d: scaled pivot column
    double* diag = rbuf + d;                                      // d: replicated Schur diagonal
    int* active = reinterpret_cast<int*>(diag + d);               // d
    PcholCtl* ctl = reinterpret_cast<PcholCtl*>(active + ((d + 3) & ~3));
    __shared__ int red_i[8];
    __shared__ int s_next;
    __shared__ double s_inv, s_rjj;
    __shared__ int s_stop;
    const int me = (int)cluster_rank();
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;

    for (int lc = 0; lc < ncl; ++lc) {
        const int c = lc * CL + me;
        for (int i = tid; i < d; i += 256) S[(size_t)lc * d + i] = (c < d) ? G[(int64_t)c * d + i] : 0.0;
    }
    for (int i = tid; i < d; i += 256) {
        active[i] = 1;
        diag[i] = G[(int64_t)i * d + i];
    }
    if (tid == 0) {
        ctl->progress = 0;
        ctl->abort = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(
                         static_cast<uint32_t>(__cvta_generic_to_shared(&ctl->mbar))),
                     "r"(CL)
                     : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    cluster_hw_sync();               // columns, counters and barrier initialised everywhere

    // argmax of the replicated diagonal over active columns (ties: lowest column).
    // Non-negative doubles order like their bit patterns read as int64, so the
    // search runs on the integer pipes (FP64 instructions are scarce here);
    // a negative diagonal (rounding of a vanished column) never wins against
    // a positive one, and if none is positive the rank test stops anyway.
    __shared__ long long red_b[8];
    auto pick = [&]() -> int {
        long long bb = LLONG_MIN;
        int bi = 0x7fffffff;
        for (int i = tid; i < d; i += 256)
            if (active[i]) {
                const long long v = __double_as_longlong(diag[i]);
                if (v > bb || (v == bb && i < bi)) { bb = v; bi = i; }
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const long long ov = __shfl_xor_sync(0xffffffffu, bb, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > bb || (ov == bb && oi < bi)) { bb = ov; bi = oi; }
        }
        if (lane == 0) { red_b[wid] = bb; red_i[wid] = bi; }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < 8; ++w)
                if (red_b[w] > bb || (red_b[w] == bb && red_i[w] < bi)) { bb = red_b[w]; bi = red_i[w]; }
            s_next = bi;
        }
        __syncthreads();
        return s_next;
    };

    const int steps = forced ? min(forced_rank, min(m, d)) : min(m, d);
    double s00 = 0.0;
    int j = 0;
    bool ok = true;
    int p = forced ? (steps > 0 ? forced[0] : -1) : pick();
    for (; j < steps; ++j) {
        // 1. rank test on the squared trailing norm of the pivot (replicated, identical in
        //    every CTA), sqrt and reciprocal once per step on thread 0
        if (p < 0 || p >= d || !active[p]) break;
        if (tid == 0) {
            const double bv = diag[p];
            if (j == 0) s00 = bv;
            int stop = !(bv > 0.0);
            if (!forced && bv <= tau * tau * s00) stop = 1;
            s_stop = stop;
            if (!stop) {
                s_rjj = sqrt(bv);
                s_inv = 1.0 / s_rjj;
            }
        }
        __syncthreads();
        if (s_stop) break;
        const double rjj = s_rjj, inv = s_inv;
        const int own = p % CL, lp = p / CL;
        // 2. wait until the owner has finished column p (bounded), then copy it
        if (tid == 0) {
            const uint32_t a =
                mapa_u32(static_cast<uint32_t>(__cvta_generic_to_shared(&ctl->progress)), (uint32_t)own);
            const uint64_t t0 = gtimer();
            for (uint32_t it = 0;; ++it) {
                if (ld_acquire_dsmem_u32(a) >= (unsigned)j) break;
                if ((it & 31u) == 31u && gtimer() - t0 > kClusterWaitNs) {
                    atomicExch(status, kStatusClusterTimeout);
                    ctl->abort = 1;
                    break;
                }
            }
        }
        __syncthreads();
        if (ctl->abort) { ok = false; break; }
        {
            const uint32_t a = mapa_u32(static_cast<uint32_t>(__cvta_generic_to_shared(S + (size_t)lp * d)),
                                        (uint32_t)own);
            for (int i = tid; i < d; i += 256) rbuf[i] = active[i] ? ld_dsmem_f64(a + 8u * (uint32_t)i) * inv : 0.0;
        }
        __syncthreads();
        if (tid == 0) {
            active[p] = 0;
            if (me == 0) {
                piv[j] = p;
                Rorig[(int64_t)j * d + p] = rjj;
            }
        }
        __syncthreads();
        // 3. replicated diagonal update and the next pivot
        for (int i = tid; i < d; i += 256)
            if (active[i]) diag[i] = fma(-rbuf[i], rbuf[i], diag[i]);
        __syncthreads();
        const int pn = forced ? (j + 1 < steps ? forced[j + 1] : -1) : pick();
        // 4. own columns: the next pivot's column first, then publish, then the rest
        const bool own_next = pn >= 0 && pn < d && (pn % CL) == me && active[pn];
        if (own_next) {
            double* col = S + (size_t)(pn / CL) * d;
            const double rc = rbuf[pn];
            for (int i = tid; i < d; i += 256)
                if (active[i]) col[i] = fma(-rbuf[i], rc, col[i]);
            if (tid == 0) Rorig[(int64_t)j * d + pn] = rc;
        }
        __syncthreads();
        if (tid == 0 && own_next) st_release_cta_u32(&ctl->progress, (unsigned)(j + 1));
        for (int lc = 0; lc < ncl; ++lc) {
            const int c = lc * CL + me;
            if (c >= d || c == pn || !active[c]) continue;
            const double rc = rbuf[c];
            if (tid == 0) Rorig[(int64_t)j * d + c] = rc;
            double* col = S + (size_t)lc * d;
            for (int i = tid; i < d; i += 256)
                if (active[i]) col[i] = fma(-rbuf[i], rc, col[i]);
        }
        __syncthreads();
        p = pn;
    }
    if (me == 0 && tid == 0) *rank_out = j;
    if (ok) cluster_exit_barrier(ctl, CL, status);
}

// Pivoted Cholesky of G for larger d: one cooperative grid (one CTA per SM), the
// Schur complement updated in place in global memory (L2 resident), CTA c owning
// the columns l = c mod gridDim. As in the cluster kernel every CTA keeps a
// replicated diagonal and takes the same pivots; the owner of the next pivot
// updates that column first and publishes its progress in a global flag, which
// readers poll (bounded) before copying the column from L2.
__device__ __forceinline__ unsigned ld_acquire_gpu_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__global__ void __launch_bounds__(256, 1) k_pchol_grid(double* __restrict__ S, int d, int m, double tau,
                                                       const int32_t* __restrict__ forced, int forced_rank,
                                                       double* __restrict__ Rorig, int32_t* __restrict__ piv,
                                                       int64_t* __restrict__ rank_out, unsigned* progress,
                                                       int32_t* status) {
    extern __shared__ __align__(16) uint8_t smem[];
    double* rbuf = reinterpret_cast<double*>(smem);               // d
    double* diag = rbuf + d;                                      // d
    int* active = reinterpret_cast<int*>(diag + d);               // d
    __shared__ long long red_b[8];
    __shared__ int red_i[8];
    __shared__ int s_next, s_stop, s_abort;
    __shared__ double s_inv, s_rjj;
    const int G = gridDim.x, me = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int i = tid; i < d; i += 256) {
        active[i] = 1;
        diag[i] = __ldcg(S + (int64_t)i * d + i);
    }
    if (tid == 0) s_abort = 0;
    __syncthreads();
    auto pick = [&]() -> int {
        long long bb = LLONG_MIN;
        int bi = 0x7fffffff;
        for (int i = tid; i < d; i += 256)
            if (active[i]) {
                const long long v = __double_as_longlong(diag[i]);
                if (v > bb || (v == bb && i < bi)) { bb = v; bi = i; }
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const long long ov = __shfl_xor_sync(0xffffffffu, bb, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > bb || (ov == bb && oi < bi)) { bb = ov; bi = oi; }
        }
        if (lane == 0) { red_b[wid] = bb; red_i[wid] = bi; }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < 8; ++w)
                if (red_b[w] > bb || (red_b[w] == bb && red_i[w] < bi)) { bb = red_b[w]; bi = red_i[w]; }
            s_next = bi;
        }
        __syncthreads();
        return s_next;
    };
    const int steps = forced ? min(forced_rank, min(m, d)) : min(m, d);
    double s00 = 0.0;
    int j = 0;
    int p = forced ? (steps > 0 ? forced[0] : -1) : pick();
    for (; j < steps; ++j) {
        if (p < 0 || p >= d || !active[p]) break;
        if (tid == 0) {
            const double bv = diag[p];
            if (j == 0) s00 = bv;
            int stop = !(bv > 0.0);
            if (!forced && bv <= tau * tau * s00) stop = 1;
            s_stop = stop;
            if (!stop) {
                s_rjj = sqrt(bv);
                s_inv = 1.0 / s_rjj;
            }
        }
        __syncthreads();
        if (s_stop) break;
        const double rjj = s_rjj, inv = s_inv;
        const int own = p % G;
        if (tid == 0) {
            const uint64_t t0 = gtimer();
            for (uint32_t it = 0;; ++it) {
                if (ld_acquire_gpu_u32(progress + own) >= (unsigned)j) break;
                if ((it & 31u) == 31u && gtimer() - t0 > kClusterWaitNs) {
                    atomicExch(status, kStatusClusterTimeout);
                    s_abort = 1;
                    break;
                }
            }
        }
        __syncthreads();
        if (s_abort) break;
        const double* colp = S + (int64_t)p * d;
        for (int i = tid; i < d; i += 256) rbuf[i] = active[i] ? __ldcg(colp + i) * inv : 0.0;
        __syncthreads();
        if (tid == 0) {
            active[p] = 0;
            if (me == 0) {
                piv[j] = p;
                Rorig[(int64_t)j * d + p] = rjj;
            }
        }
        __syncthreads();
        for (int i = tid; i < d; i += 256)
            if (active[i]) diag[i] = fma(-rbuf[i], rbuf[i], diag[i]);
        __syncthreads();
        const int pn = forced ? (j + 1 < steps ? forced[j + 1] : -1) : pick();
        const bool own_next = pn >= 0 && pn < d && (pn % G) == me && active[pn];
        if (own_next) {
            double* col = S + (int64_t)pn * d;
            const double rc = rbuf[pn];
            for (int i = tid; i < d; i += 256)
                if (active[i]) __stcg(col + i, fma(-rbuf[i], rc, __ldcg(col + i)));
            if (tid == 0) Rorig[(int64_t)j * d + pn] = rc;
            __syncthreads();
            if (tid == 0) {
                __threadfence();
                st_release_gpu_u32(progress + me, (unsigned)(j + 1));
            }
        }
        for (int c = me; c < d; c += G) {
            if (c == pn || !active[c]) continue;
            const double rc = rbuf[c];
            if (tid == 0) Rorig[(int64_t)j * d + c] = rc;
            double* col = S + (int64_t)c * d;
            for (int i = tid; i < d; i += 256)
                if (active[i]) __stcg(col + i, fma(-rbuf[i], rc, __ldcg(col + i)));
        }
        __syncthreads();
        p = pn;
    }
    if (me == 0 && tid == 0) *rank_out = j;
}

}  // namespace

int gram_splits(int64_t m, int64_t d) {
    const int T = gram_tiles((int)d);
    const int64_t blocks = (m + GT - 1) / GT;
    int64_t s = (2 * 152 + T - 1) / T;
    if (s > blocks) s = blocks;
    if (s < 1) s = 1;
    return (int)s;
}

size_t gram_partial_doubles(int64_t m, int64_t d) {
    return (size_t)gram_splits(m, d) * gram_tiles((int)d) * GT * GT;
}

cudaError_t launch_gram_pivoted_cholesky(const float* Atilde, int64_t m, int64_t d, double tau,
                                         const int32_t* forced, int64_t forced_rank, const QrScratch& q,
                                         int32_t* status, cudaStream_t st) {
    const int splits = gram_splits(m, d);
    int64_t blocks_rows = (m + GT - 1) / GT;
    const int rows_per_split = (int)(((blocks_rows + splits - 1) / splits) * GT);
    dim3 grid((unsigned)gram_tiles((int)d), (unsigned)splits);
    k_gram_fp64<<<grid, 256, 0, st>>>(Atilde, (int)m, (int)d, rows_per_split, q.Gp);
    k_gram_reduce<<<152 * 4, 256, 0, st>>>(q.Gp, (int)d, splits, q.G);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;

    auto launch = [&](auto kern, int CL) -> cudaError_t {
        const int ncl = (int)((d + CL - 1) / CL);
        const size_t smem = sizeof(double) * (size_t)ncl * d + 2 * sizeof(double) * (size_t)d +
                            sizeof(int) * (size_t)((d + 3) & ~3) + sizeof(PcholCtl) + 64;
        cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        if (CL > 8) {
            err = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            if (err != cudaSuccess) return err;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)CL);
        cfg.blockDim = dim3(256);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)CL;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nclusters = 0;
        err = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg);
        if (err != cudaSuccess || nclusters < 1) {
            cudaGetLastError();
            return cudaErrorNotSupported;
        }
        return cudaLaunchKernelEx(&cfg, kern, (const double*)q.G, (int)d, (int)m, tau, forced, (int)forced_rank,
                                  q.Rorig, q.piv, q.rank, status);
    };
    if (d <= kClusterMaxD) {
        e = launch(k_pchol<16>, 16);
        if (e == cudaErrorNotSupported) e = launch(k_pchol<8>, 8);
        return e;
    }
    // larger d: cooperative grid over the SMs, Schur complement in place in G
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = 2 * sizeof(double) * (size_t)d + sizeof(int) * (size_t)d + 64;
    if ((e = cudaFuncSetAttribute(k_pchol_grid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
    const int pgrid = sms < (int)d ? sms : (int)d;
    if ((e = cudaMemsetAsync(q.flags, 0, sizeof(unsigned) * (size_t)pgrid, st)) != cudaSuccess) return e;
    double* S = q.G;
    const int32_t* fp = forced;
    int fr = (int)forced_rank, di = (int)d, mi = (int)m;
    void* kargs[] = {&S, &di, &mi, &tau, &fp, &fr, (void*)&q.Rorig, (void*)&q.piv, (void*)&q.rank, (void*)&q.flags,
                     &status};
    e = cudaLaunchCooperativeKernel((const void*)k_pchol_grid, dim3((unsigned)pgrid), dim3(256), kargs, smem, st);
    return e;
}

}  // namespace lev
