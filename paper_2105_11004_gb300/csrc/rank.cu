// Rank decisions beyond the diagonal test of the pivoted QR, on sm_103a (FP64).
//
//  * singular values of the sketch: one-sided (Hestenes) Jacobi on the rows of R, the triangular
//    factor of A~ P (sigma(R) = sigma(A~)): plane rotations of row pairs (Y <- J Y) until every
//    pair is orthogonal, after which the row norms are the singular values and the normalised rows
//    the right singular vectors of R. One cooperative grid; the pairs of a round are disjoint
//    (round-robin order), a bounded grid barrier separates the rounds. The rank is then the count
//    of sigma_j > tau sigma_1 (Alg. 11 step 3; Sec. 6.2: the singular values see a gap that the
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

// Y: rows 0..r-1 (r read from *d_rows, at most d), row-major, ld = d. Rounds are ordered by rows,
// not by a grid barrier: version[p] (zeroed by the caller) counts the rounds applied to row p, and
// the CTA that holds pair (p, q) in global round T waits (bounded) until both rows reached version
// T, rotates them and publishes T + 1. Every CTA takes its pairs in round order and all CTAs are
// resident (cooperative launch), so the earliest unfinished pair always has its rows ready. A grid
// barrier ends each sweep; rotated[s] counts the rotations of sweep s (zeroed by the caller) and
// the sweeps stop after one without any. *sweeps_out = sweeps run (max_sweeps + 1 when the last
// sweep still rotated).
__global__ void __launch_bounds__(256) k_jacobi_rows(double* __restrict__ Y, const int64_t* __restrict__ d_rows,
                                                     int d, int max_sweeps, unsigned* __restrict__ rotated,
                                                     unsigned* __restrict__ barrier, unsigned* __restrict__ version,
                                                     int32_t* __restrict__ status, int32_t* __restrict__ sweeps_out) {
    __shared__ double part[3][8];
    __shared__ double tot[3];
    const int r = (int)min(max(*d_rows, (int64_t)0), (int64_t)d);
    const int n = r + (r & 1);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned epoch = 0;
    if (n < 2) {
        if (blockIdx.x == 0 && threadIdx.x == 0) *sweeps_out = 0;
        return;
    }
    for (int s = 0; s < max_sweeps; ++s) {
        for (int t = 0; t < n - 1; ++t) {
            const unsigned T = (unsigned)s * (unsigned)(n - 1) + (unsigned)t;
            for (int i = blockIdx.x; i < n / 2; i += gridDim.x) {
                int p, q;
                round_pair(n, t, i, p, q);
                const bool pv = p < r, qv = q < r;                       // q may be the padding row
                if (threadIdx.x == 0) {
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
                    double* yp = Y + (int64_t)p * d;
                    double* yq = Y + (int64_t)q * d;
                    double a = 0.0, b = 0.0, c = 0.0;
                    for (int j = threadIdx.x; j < d; j += blockDim.x) {
                        const double x = yp[j], y = yq[j];
                        a = fma(x, x, a);
                        b = fma(y, y, b);
                        c = fma(x, y, c);
                    }
                    a = warp_sum(a);
                    b = warp_sum(b);
                    c = warp_sum(c);
                    if (lane == 0) {
                        part[0][w] = a;
                        part[1][w] = b;
                        part[2][w] = c;
                    }
                    __syncthreads();
                    if (threadIdx.x < 3) {
                        double v = 0.0;
                        for (int u = 0; u < (int)(blockDim.x >> 5); ++u) v += part[threadIdx.x][u];
                        tot[threadIdx.x] = v;
                    }
                    __syncthreads();
                    a = tot[0];
                    b = tot[1];
                    c = tot[2];
                    if (a > 0.0 && b > 0.0 && fabs(c) > kJacobiTol * sqrt(a) * sqrt(b)) {
                        const double zeta = (b - a) / (2.0 * c);
                        const double tr = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                        const double cs = 1.0 / sqrt(1.0 + tr * tr), sn = cs * tr;
                        for (int j = threadIdx.x; j < d; j += blockDim.x) {
                            const double x = yp[j], y = yq[j];
                            yp[j] = cs * x - sn * y;
                            yq[j] = sn * x + cs * y;
                        }
                        if (threadIdx.x == 0) atomicAdd(&rotated[s], 1u);
                    }
                }
                __syncthreads();                                             // rows written, tot read
                if (threadIdx.x == 0) {
                    __threadfence();
                    if (pv) st_release_gpu(version + p, T + 1);
                    if (qv) st_release_gpu(version + q, T + 1);
                }
            }
        }
        if (!grid_barrier(barrier, epoch, status)) return;
        if (*(volatile unsigned*)&rotated[s] == 0u) {
            if (blockIdx.x == 0 && threadIdx.x == 0) *sweeps_out = s + 1;
            return;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *sweeps_out = max_sweeps + 1;
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
// of the Jacobi (d uint32, from the sweep count + 2).
size_t rank_scratch_doubles(int64_t d) { return (size_t)(d * d + 3 * d + 16 + 2 * 1024 + 32 + d + 8 + d); }

cudaError_t launch_svd_rank(const double* R, const int64_t* d_rows, int64_t d, double tau, double* Y,
                            unsigned* work, double* sigma, int32_t* order, int64_t* rank_out, int32_t* sweeps_out,
                            unsigned* version, int32_t* status, int num_sms, cudaStream_t st) {
    cudaError_t e;
    constexpr int kMaxSweeps = 40;
    if (d > 1024) return cudaErrorInvalidValue;
    if ((e = cudaMemcpyAsync(Y, R, sizeof(double) * (size_t)(d * d), cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return e;
    unsigned* barrier = work;
    unsigned* rotated = work + 1;
    if ((e = cudaMemsetAsync(work, 0, sizeof(unsigned) * (1 + kMaxSweeps), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(version, 0, sizeof(unsigned) * (size_t)d, st)) != cudaSuccess) return e;
    int grid = (int)((d + 1) / 2);
    if (grid > num_sms) grid = num_sms;
    if (grid < 1) grid = 1;
    int di = (int)d, ms = kMaxSweeps;
    void* kargs[] = {&Y, (void*)&d_rows, &di, &ms, &rotated, &barrier, &version, &status, &sweeps_out};
    if ((e = cudaLaunchCooperativeKernel((const void*)k_jacobi_rows, dim3((unsigned)grid), dim3(256), kargs, 0, st)) !=
        cudaSuccess)
        return e;
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
