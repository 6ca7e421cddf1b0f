// Rank decisions beyond the diagonal test of the pivoted QR, on sm_103a (FP64).
//
//  * singular values of the sketch: one-sided (Hestenes) Jacobi on the rows of R, the triangular
//    factor of A~ P (sigma(R) = sigma(A~)): plane rotations of row pairs (Y <- J Y) until every
//    pair is orthogonal, after which the row norms are the singular values and the normalised rows
//    the right singular vectors of R. One cooperative grid; the pairs of a round are disjoint
//    (round-robin order), a bounded grid barrier separates the rounds. The rank is then the count
//    of sigma_j > tau sigma_1 (Alg. 11 step 3; Sec. 7.2: the singular values see a gap that the
//    diagonal of R can miss);
//  * strong-RRQR measures at a fixed k (Alg. 2 after Gu and Eisenstat): from R in pivot order,
//    Z = R11^{-1} [I | R12], the row norms of R11^{-1}, gamma_j^2 = G_jj - ||R[:k, j]||^2 (the
//    Schur complement's diagonal, G = A~^T A~), and the largest
//    rho_ij^2 = (R11^{-1} R12)_ij^2 + gamma_j^2 ||e_i^T R11^{-1}||^2 with its (i, j).
#include "lev_common.cuh"
#include "lev_kernels.cuh"

namespace lev {

namespace {

constexpr double kJacobiTol = 1e-12;   // a pair counts as orthogonal when |y_p.y_q| <= tol ||y_p|| ||y_q||

__device__ __forceinline__ void round_pair(int n, int t, int i, int& p, int& q) {
    if (i == 0) {
        p = t;
        q = n - 1;
    } else {
        p = (t + i) % (n - 1);
        q = (t - i + n - 1) % (n - 1);
    }
}

__device__ __forceinline__ void st_release_gpu(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

// Double-float arithmetic (a value is hi + lo, two FP32 numbers, about 48 significant bits): FP64
// runs at 1/64 of the FP32 rate on this GPU, and the Jacobi's dot products and rotations are its
// bulk. Every step uses the round-to-nearest intrinsics, so nothing is contracted into an FMA that
// would break the error-free transformations (Knuth's TwoSum, the fma-based TwoProduct).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void df_add(float ah, float al, float bh, float bl, float& sh, float& sl) {
    float s, e;
    two_sum(ah, bh, s, e);
    e = __fadd_rn(e, __fadd_rn(al, bl));
    two_sum(s, e, sh, sl);
}

// (ah + al)(bh + bl), the al bl term dropped (below 2^-48 of the product)
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float& ph, float& pl) {
    const float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    two_sum(p, e, ph, pl);
}

// (s, c) += (xh + xl)(yh + yl): the exact product xh yh = p + e, the cross terms into e, p added
// error-free to s, the errors collected in c
__device__ __forceinline__ void df_dot_acc(float xh, float xl, float yh, float yl, float& s, float& c) {
    const float p = __fmul_rn(xh, yh);
    float e = __fmaf_rn(xh, yh, -p);
    e = __fmaf_rn(xh, yl, e);
    e = __fmaf_rn(xl, yh, e);
    float s1, q;
    two_sum(s, p, s1, q);
    s = s1;
    c = __fadd_rn(c, __fadd_rn(q, e));
}

// the same pair on every lane (df_add is symmetric in its two arguments)
__device__ __forceinline__ void df_warp_sum(float& h, float& l) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
        df_add(h, l, oh, ol, h, l);
    }
}

// Yh, Yl = the double-float split of R (hi = fl32(x), lo = fl32(x - hi)); Y = Yh + Yl back in FP64.
__global__ void k_split_rows(const double* __restrict__ R, int64_t count, float* __restrict__ Yh,
                             float* __restrict__ Yl) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
        const double x = R[e];
        const float h = (float)x;
        Yh[e] = h;
        Yl[e] = (float)(x - (double)h);
    }
}

__global__ void k_join_rows(const float* __restrict__ Yh, const float* __restrict__ Yl, int64_t count,
                            double* __restrict__ Y) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
        Y[e] = (double)Yh[e] + (double)Yl[e];
}

// One-sided Jacobi on rows 0..r-1 (r read from *d_rows, at most d) of Y = Yh + Yl (double-float,
// row-major, ld = d), one CTA a pair: thread t holds elements t + 256 j (j < PER, d <= 256 PER) of
// both rows; the three dot products are compensated sums reduced over the warps in double-float
// and over the CTA in FP64 by one thread, which also takes the rotation (in FP64) and splits it;
// the rotation itself runs in double-float. Rounds are ordered by rows, not by a grid barrier:
// version[p] (zeroed by the caller) counts the rounds applied to row p, and the CTA that holds pair
// (p, q) in global round T waits (bounded) until both rows reached version T, rotates them and
// publishes T + 1. Every CTA takes its pairs in round order and all CTAs are resident (cooperative
// launch), so the earliest unfinished pair always has its rows ready. A grid barrier ends each
// sweep; rotated[s] counts the rotations of sweep s (zeroed by the caller) and the sweeps stop
// after one without any. *sweeps_out = sweeps run (max_sweeps + 1 when the last sweep still
// rotated).
template <int PER>
__global__ void __launch_bounds__(256) k_jacobi_rows(float* __restrict__ Yh, float* __restrict__ Yl,
                                                     const int64_t* __restrict__ d_rows, int d, int max_sweeps,
                                                     unsigned* __restrict__ rotated, unsigned* __restrict__ barrier,
                                                     unsigned* __restrict__ version, int32_t* __restrict__ status,
                                                     int32_t* __restrict__ sweeps_out) {
    __shared__ float part[6][8];
    __shared__ float rot[4];
    __shared__ int do_rot;
    const int r = (int)min(max(*d_rows, (int64_t)0), (int64_t)d);
    const int n = r + (r & 1);
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    unsigned epoch = 0;
    if (n < 2) {
        if (blockIdx.x == 0 && tid == 0) *sweeps_out = 0;
        return;
    }
    for (int s = 0; s < max_sweeps; ++s) {
        for (int t = 0; t < n - 1; ++t) {
            const unsigned T = (unsigned)s * (unsigned)(n - 1) + (unsigned)t;
            for (int i = blockIdx.x; i < n / 2; i += gridDim.x) {
                int p, q;
                round_pair(n, t, i, p, q);
                const bool pv = p < r, qv = q < r;                       // q may be the padding row
                if (tid == 0) {
                    long long spins = 0;
                    while ((pv && ld_acquire_gpu(version + p) < T) || (qv && ld_acquire_gpu(version + q) < T)) {
                        if (ld_volatile(status) != 0) break;
                        if (++spins > kSpinLimit) {
                            atomicExch(status, kStatusTimeoutBarrier);
                            break;
                        }
                        __nanosleep(32);
                    }
                }
                __syncthreads();
                if (ld_volatile(status) != 0) return;
                if (pv && qv) {
                    float xh[PER], xl[PER], yh[PER], yl[PER];
                    const int64_t op = (int64_t)p * d, oq = (int64_t)q * d;
#pragma unroll
                    for (int j = 0; j < PER; ++j) {
                        const int e = tid + 256 * j;
                        const bool ok = e < d;
                        xh[j] = ok ? Yh[op + e] : 0.f;
                        xl[j] = ok ? Yl[op + e] : 0.f;
                        yh[j] = ok ? Yh[oq + e] : 0.f;
                        yl[j] = ok ? Yl[oq + e] : 0.f;
                    }
                    float ah = 0.f, al = 0.f, bh = 0.f, bl = 0.f, ch = 0.f, cl = 0.f;
#pragma unroll
                    for (int j = 0; j < PER; ++j) {
                        df_dot_acc(xh[j], xl[j], xh[j], xl[j], ah, al);
                        df_dot_acc(yh[j], yl[j], yh[j], yl[j], bh, bl);
                        df_dot_acc(xh[j], xl[j], yh[j], yl[j], ch, cl);
                    }
                    df_warp_sum(ah, al);
                    df_warp_sum(bh, bl);
                    df_warp_sum(ch, cl);
                    if (lane == 0) {
                        part[0][w] = ah; part[1][w] = al;
                        part[2][w] = bh; part[3][w] = bl;
                        part[4][w] = ch; part[5][w] = cl;
                    }
                    __syncthreads();
                    if (tid == 0) {
                        double a = 0.0, b = 0.0, c = 0.0;
                        for (int u = 0; u < 8; ++u) {
                            a += (double)part[0][u] + (double)part[1][u];
                            b += (double)part[2][u] + (double)part[3][u];
                            c += (double)part[4][u] + (double)part[5][u];
                        }
                        int go = 0;
                        if (a > 0.0 && b > 0.0 && fabs(c) > kJacobiTol * sqrt(a) * sqrt(b)) {
                            const double zeta = (b - a) / (2.0 * c);
                            const double tr = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                            const double cs = 1.0 / sqrt(1.0 + tr * tr), sn = cs * tr;
                            const float csh = (float)cs, snh = (float)sn;
                            rot[0] = csh;
                            rot[1] = (float)(cs - (double)csh);
                            rot[2] = snh;
                            rot[3] = (float)(sn - (double)snh);
                            go = 1;
                            atomicAdd(&rotated[s], 1u);
                        }
                        do_rot = go;
                    }
                    __syncthreads();
                    if (do_rot) {
                        const float csh = rot[0], csl = rot[1], snh = rot[2], snl = rot[3];
#pragma unroll
                        for (int j = 0; j < PER; ++j) {
                            const int e = tid + 256 * j;
                            if (e >= d) continue;
                            float t1h, t1l, t2h, t2l, nh, nl;
                            df_mul(csh, csl, xh[j], xl[j], t1h, t1l);             // x' = cs x - sn y
                            df_mul(snh, snl, yh[j], yl[j], t2h, t2l);
                            df_add(t1h, t1l, -t2h, -t2l, nh, nl);
                            Yh[op + e] = nh;
                            Yl[op + e] = nl;
                            df_mul(snh, snl, xh[j], xl[j], t1h, t1l);             // y' = sn x + cs y
                            df_mul(csh, csl, yh[j], yl[j], t2h, t2l);
                            df_add(t1h, t1l, t2h, t2l, nh, nl);
                            Yh[oq + e] = nh;
                            Yl[oq + e] = nl;
                        }
                    }
                }
                __syncthreads();                                             // rows written, rot read
                if (tid == 0) {
                    __threadfence();
                    if (pv) st_release_gpu(version + p, T + 1);
                    if (qv) st_release_gpu(version + q, T + 1);
                }
            }
        }
        if (!grid_barrier(barrier, epoch, status)) return;
        if (*(volatile unsigned*)&rotated[s] == 0u) {
            if (blockIdx.x == 0 && tid == 0) *sweeps_out = s + 1;
            return;
        }
    }
    if (blockIdx.x == 0 && tid == 0) *sweeps_out = max_sweeps + 1;
}

// sigma (d, descending; zeros past the r rows) and order (the row of Y that holds each) from the
// row norms of Y; *rank_out = #{sigma_j > tau sigma_1}. One CTA of 1024 threads, bitonic sort of
// (sigma, row) pairs, ties to the lower row.
__global__ void __launch_bounds__(1024) k_sigma_rank(const double* __restrict__ Y, const int64_t* __restrict__ d_rows,
                                                     int d, double tau, double* __restrict__ sigma,
                                                     int32_t* __restrict__ order, int64_t* __restrict__ rank_out) {
    __shared__ double sv[1024];
    __shared__ int si[1024];
    __shared__ int cnt;
    const int r = (int)min(max(*d_rows, (int64_t)0), (int64_t)d);
    const int t = threadIdx.x;
    if (t == 0) cnt = 0;
    for (int i = t; i < 1024; i += blockDim.x) {
        double v = -1.0;
        if (i < r) {
            const double* y = Y + (int64_t)i * d;
            double s2 = 0.0;
            for (int j = 0; j < d; ++j) s2 = fma(y[j], y[j], s2);
            v = sqrt(s2);
        }
        sv[i] = v;
        si[i] = i;
    }
    __syncthreads();
    for (int size = 2; size <= 1024; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const int j = t ^ stride;
            if (j > t) {
                const bool desc = (t & size) == 0;
                const bool t_first = sv[t] > sv[j] || (sv[t] == sv[j] && si[t] < si[j]);
                if (t_first != desc) {
                    const double v = sv[t];
                    sv[t] = sv[j];
                    sv[j] = v;
                    const int x = si[t];
                    si[t] = si[j];
                    si[j] = x;
                }
            }
            __syncthreads();
        }
    }
    const double top = sv[0];
    if (t < d) {
        sigma[t] = t < r ? sv[t] : 0.0;
        order[t] = t < r ? si[t] : -1;
        if (t < r && top > 0.0 && sv[t] > tau * top) atomicAdd(&cnt, 1);
    }
    __syncthreads();
    if (t == 0) *rank_out = cnt;
}

// Z[:, c] = R11^{-1} b_c (k x d, row-major, ld = d): b_c = e_c for c < k, R[:k, c] for c >= k.
// One CTA per column, one thread per row, the unit-diagonal substitution of the Omega solve
// (Rs: R11's strictly upper part scaled by its diagonal and transposed).
__global__ void __launch_bounds__(1024) k_srrqr_solve(const double* __restrict__ R, const double* __restrict__ Rs,
                                                      int d, int k, double* __restrict__ Z) {
    __shared__ double xs[2];
    const int c = blockIdx.x, i = threadIdx.x;
    double x = 0.0;
    if (i < k) {
        const double b = c < k ? (i == c ? 1.0 : 0.0) : R[(int64_t)i * d + c];
        x = b / R[(int64_t)i * d + i];
    }
    const int top = c < k ? c : k - 1;               // e_c has no entries below row c
    for (int j = top; j >= 0; --j) {
        if (i == j) xs[j & 1] = x;
        __syncthreads();
        if (i < j) x = fma(-Rs[(int64_t)j * d + i], xs[j & 1], x);
    }
    if (i < k) Z[(int64_t)i * d + c] = x;
}

// wn[i] = ||e_i^T R11^{-1}||^2 (i < k); g2[j] = max(G[P_j][P_j] - ||R[:k, j]||^2, 0) (k <= j < d).
__global__ void k_srrqr_norms(const double* __restrict__ Z, const double* __restrict__ R,
                              const double* __restrict__ G, const int32_t* __restrict__ perm, int d, int k,
                              double* __restrict__ wn, double* __restrict__ g2) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < k) {
        double s = 0.0;
        for (int c = t; c < k; ++c) s = fma(Z[(int64_t)t * d + c], Z[(int64_t)t * d + c], s);
        wn[t] = s;
    } else if (t < d) {
        const int pc = perm[t];
        double s = G[(int64_t)pc * d + pc];
        for (int i = 0; i < k; ++i) s = fma(-R[(int64_t)i * d + t], R[(int64_t)i * d + t], s);
        g2[t] = s > 0.0 ? s : 0.0;
    }
}

// Largest rho^2 over i < k, k <= j < d (ties to the lower row-major index i (d - k) + (j - k)):
// per-CTA winners into part, then one CTA picks among them. out: {rho^2, i, j}.
__device__ __forceinline__ bool better(double v, long long e, double bv, long long be) {
    return v > bv || (v == bv && e < be);
}

__global__ void __launch_bounds__(256) k_srrqr_argmax(const double* __restrict__ Z, const double* __restrict__ wn,
                                                      const double* __restrict__ g2, int d, int k,
                                                      double* __restrict__ part_v, long long* __restrict__ part_e) {
    __shared__ double bv_s[256];
    __shared__ long long be_s[256];
    const long long total = (long long)k * (d - k);
    double bv = -1.0;
    long long be = total;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / (d - k)), j = k + (int)(e % (d - k));
        const double x = Z[(int64_t)i * d + j];
        const double v = fma(x, x, g2[j] * wn[i]);
        if (better(v, e, bv, be)) {
            bv = v;
            be = e;
        }
    }
    bv_s[threadIdx.x] = bv;
    be_s[threadIdx.x] = be;
    __syncthreads();
    for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
        if (threadIdx.x < o && better(bv_s[threadIdx.x + o], be_s[threadIdx.x + o], bv_s[threadIdx.x], be_s[threadIdx.x])) {
            bv_s[threadIdx.x] = bv_s[threadIdx.x + o];
            be_s[threadIdx.x] = be_s[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part_v[blockIdx.x] = bv_s[0];
        part_e[blockIdx.x] = be_s[0];
    }
}

__global__ void __launch_bounds__(256) k_srrqr_pick(const double* __restrict__ part_v, const long long* __restrict__ part_e,
                                                    int parts, int d, int k, double* __restrict__ out) {
    __shared__ double bv_s[256];
    __shared__ long long be_s[256];
    double bv = -1.0;
    long long be = 1ll << 62;
    for (int u = threadIdx.x; u < parts; u += blockDim.x)
        if (better(part_v[u], part_e[u], bv, be)) {
            bv = part_v[u];
            be = part_e[u];
        }
    bv_s[threadIdx.x] = bv;
    be_s[threadIdx.x] = be;
    __syncthreads();
    for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
        if (threadIdx.x < o && better(bv_s[threadIdx.x + o], be_s[threadIdx.x + o], bv_s[threadIdx.x], be_s[threadIdx.x])) {
            bv_s[threadIdx.x] = bv_s[threadIdx.x + o];
            be_s[threadIdx.x] = be_s[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = bv_s[0];
        out[1] = (double)(be_s[0] / (d - k));
        out[2] = (double)(k + be_s[0] % (d - k));
    }
}

// perm[i] <-> perm[j] when rho^2 > phi^2 (out = {rho^2, i, j} of k_srrqr_pick).
__global__ void k_srrqr_swap(const double* __restrict__ out, double phi2, int32_t* __restrict__ perm) {
    if (threadIdx.x == 0 && out[0] > phi2) {
        const int i = (int)out[1], j = (int)out[2];
        const int32_t x = perm[i];
        perm[i] = perm[j];
        perm[j] = x;
    }
}

}  // namespace

// Y or Z (d x d), sigma, wn, g2 (d each), out (16), argmax partials (1024 values + 1024 indices),
// then 64 uint32 of barrier and rotation counts, order (d int32), the sweep count, the row versions
// of the Jacobi (d uint32, from the sweep count + 2), and the double-float rows (2 d^2 FP32).
size_t rank_scratch_doubles(int64_t d) { return (size_t)(d * d + 3 * d + 16 + 2 * 1024 + 32 + d + 8 + d + d * d + 8); }

cudaError_t launch_svd_rank(const double* R, const int64_t* d_rows, int64_t d, double tau, double* Y, float* Yhl,
                            unsigned* work, double* sigma, int32_t* order, int64_t* rank_out, int32_t* sweeps_out,
                            unsigned* version, int32_t* status, int num_sms, cudaStream_t st) {
    cudaError_t e;
    constexpr int kMaxSweeps = 40;
    if (d > 1024) return cudaErrorInvalidValue;
    float* Yh = Yhl;
    float* Yl = Yhl + d * d;
    int cg = (int)((d * d + 255) / 256);
    if (cg > 152 * 8) cg = 152 * 8;
    k_split_rows<<<cg, 256, 0, st>>>(R, d * d, Yh, Yl);
    unsigned* barrier = work;
    unsigned* rotated = work + 1;
    if ((e = cudaMemsetAsync(work, 0, sizeof(unsigned) * (1 + kMaxSweeps), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(version, 0, sizeof(unsigned) * (size_t)d, st)) != cudaSuccess) return e;
    int di = (int)d, ms = kMaxSweeps;
    void* kargs[] = {&Yh, &Yl, (void*)&d_rows, &di, &ms, &rotated, &barrier, &version, &status, &sweeps_out};
    const void* fn = d <= 256 ? (const void*)k_jacobi_rows<1>
                   : d <= 512 ? (const void*)k_jacobi_rows<2> : (const void*)k_jacobi_rows<4>;
    int occ = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 256, 0)) != cudaSuccess) return e;
    int grid = (int)((d + 1) / 2);                      // one CTA a pair where they fit
    const int cap = num_sms * (occ < 1 ? 1 : occ);
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    if ((e = cudaLaunchCooperativeKernel(fn, dim3((unsigned)grid), dim3(256), kargs, 0, st)) != cudaSuccess) return e;
    k_join_rows<<<cg, 256, 0, st>>>(Yh, Yl, d * d, Y);
    k_sigma_rank<<<1, 1024, 0, st>>>(Y, d_rows, (int)d, tau, sigma, order, rank_out);
    return cudaGetLastError();
}

cudaError_t launch_srrqr_step(const double* R, const double* Rs, const double* G, int32_t* perm, int64_t d, int64_t k,
                              double phi, double* Z, double* wn, double* g2, double* part_v, long long* part_e,
                              double* out, cudaStream_t st) {
    if (k < 1 || k >= d || d > 1024) return cudaErrorInvalidValue;
    k_srrqr_solve<<<(unsigned)d, (unsigned)((k + 31) / 32 * 32), 0, st>>>(R, Rs, (int)d, (int)k, Z);
    k_srrqr_norms<<<(unsigned)((d + 255) / 256), 256, 0, st>>>(Z, R, G, perm, (int)d, (int)k, wn, g2);
    const long long total = k * (d - k);
    int parts = (int)((total + 255) / 256);
    if (parts > 1024) parts = 1024;
    k_srrqr_argmax<<<(unsigned)parts, 256, 0, st>>>(Z, wn, g2, (int)d, (int)k, part_v, part_e);
    k_srrqr_pick<<<1, 256, 0, st>>>(part_v, part_e, parts, (int)d, (int)k, out);
    k_srrqr_swap<<<1, 32, 0, st>>>(out, phi * phi, perm);
    return cudaGetLastError();
}

}  // namespace lev
