// CountGauss preconditioning (Alg. 11) and LSQR on the preconditioned least-squares problem, on
// sm_103a.
//
//  * N = V_k Sigma_k^{-1} from the row Jacobi of R (rank.cu): with A~ P = Q R and Y = J R (rows
//    orthogonal), A~ = (Q J^T) diag(sigma) (W P^T) with W = diag(sigma)^{-1} Y, so the i-th right
//    singular vector of A~ is P w_i and N[P_j][i] = Y[order_i][j] / sigma_i^2;
//  * LSQR (Paige and Saunders) on B = A N. The Golub-Kahan step needs u' = A (N v) - alpha u and
//    then A^T u'; both come from ONE pass over A, because A^T u' is linear in u': each row r gives
//    x_r = A_r . t + gamma u_r (t = N v, gamma = -alpha / beta_prev on the stored, unnormalised u)
//    and adds A_r^T x_r to the CTA's partial of z = A^T u'. A warp takes a row (128-bit loads, the
//    row kept in registers for both products); the lanes sum A_r^T x_r in FP32 over 32 rows, then
//    fold into FP64 shared-memory partials, reduced over CTAs in a fixed order (deterministic). The
//    small steps (z, v = N^T z - beta v, the plane rotations, y and w, t = N v) are FP64 kernels
//    on the device; the host reads the convergence flag every few iterations.
#include "lev_common.cuh"
#include "lev_kernels.cuh"

namespace lev {

namespace {

// LSQR state (FP64 words of the state array).
enum : int {
    S_ALPHA = 0, S_BETA, S_RHOBAR, S_PHIBAR, S_SU, S_GAMMA, S_BNORM2, S_DONE, S_ITERS, S_ATOL, S_BSTOP,
    S_RNORM, S_ARNORM, S_COUNT
};

__global__ void k_precond_n(const double* __restrict__ Y, const int32_t* __restrict__ order,
                            const double* __restrict__ sigma, const int32_t* __restrict__ perm,
                            const int64_t* __restrict__ d_rank, int d, double* __restrict__ N) {
    const int k = (int)min(max(*d_rank, (int64_t)0), (int64_t)d);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)d * d;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / d), j = (int)(e % d);          // column i of N, pivot position j
        double v = 0.0;
        if (i < k) {
            const double s = sigma[i];
            v = Y[(int64_t)order[i] * d + j] / (s * s);
        }
        N[(int64_t)perm[j] * d + i] = v;
    }
}

// Nt[i][j] = N[j][i] for i < k (d x d, row-major).
__global__ void k_transpose_n(const double* __restrict__ N, int d, int k, double* __restrict__ Nt) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)k * d;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / d), j = (int)(e % d);
        Nt[e] = N[(int64_t)j * d + i];
    }
}

__device__ __forceinline__ float4 ld_stream4(const float* p) {
    float4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
    return v;
}

constexpr int kPassWarps = 8;
constexpr int kFold = 32;

template <bool VEC>
__device__ __forceinline__ float4 load4(const float* p, int col, int d) {
    if (VEC && col + 3 < d) return ld_stream4(p + col);
    return make_float4(col < d ? p[col] : 0.f, col + 1 < d ? p[col + 1] : 0.f, col + 2 < d ? p[col + 2] : 0.f,
                       col + 3 < d ? p[col + 3] : 0.f);
}

__device__ __forceinline__ void fold4(double* z, int col, int d, float4& a) {
    if (col < d) z[col] += a.x;
    if (col + 1 < d) z[col + 1] += a.y;
    if (col + 2 < d) z[col + 2] += a.z;
    if (col + 3 < d) z[col + 3] += a.w;
    a = make_float4(0.f, 0.f, 0.f, 0.f);
}

// One fused pass (see the header). zpart: gridDim.x x d FP64; npart: gridDim.x FP64 (sum x_r^2).
// Lane l holds columns c*128 + 4l .. +3 for c < NC; a warp takes U rows at a time, all their loads
// (and the U values of u, one per lane) issued before any is used. VEC: A 16-byte aligned with
// lda % 4 == 0.
template <int NC, int U, bool VEC>
__global__ void __launch_bounds__(32 * kPassWarps, (NC <= 2 ? 3 : 1)) k_lsqr_pass(const float* __restrict__ A, int64_t lda, int64_t n,
                                                               int d, const float* __restrict__ t,
                                                               const double* __restrict__ state,
                                                               float* __restrict__ u, double* __restrict__ zpart,
                                                               double* __restrict__ npart) {
    extern __shared__ double zs[];                      // kPassWarps x d
    __shared__ double ns[kPassWarps];
    if (state[S_DONE] != 0.0) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const float gamma = (float)state[S_GAMMA];
    for (int j = threadIdx.x; j < kPassWarps * d; j += blockDim.x) zs[j] = 0.0;
    float4 tr[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) tr[c] = load4<false>(t, c * 128 + lane * 4, d);
    __syncthreads();
    float4 acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    double nrm = 0.0;
    int since = 0;
    double* zw = zs + w * d;
    const int64_t wid = (int64_t)blockIdx.x * kPassWarps + w, nw = (int64_t)gridDim.x * kPassWarps;
    for (int64_t r0 = wid * U; r0 < n; r0 += nw * U) {
        float4 a[U][NC];
        const int64_t rq = r0 + (lane < U ? lane : 0);
        const float uq = (lane < U && rq < n) ? u[rq] : 0.f;
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const bool ok = r0 + q < n;
            const float* row = A + (r0 + q) * lda;
#pragma unroll
            for (int c = 0; c < NC; ++c)
                a[q][c] = ok ? load4<VEC>(row, c * 128 + lane * 4, d) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float dot[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            float s = 0.f;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                s = fmaf(a[q][c].x, tr[c].x, s);
                s = fmaf(a[q][c].y, tr[c].y, s);
                s = fmaf(a[q][c].z, tr[c].z, s);
                s = fmaf(a[q][c].w, tr[c].w, s);
            }
            dot[q] = s;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int q = 0; q < U; ++q) dot[q] += __shfl_xor_sync(0xffffffffu, dot[q], o);
        float mine = 0.f;                                   // lane q < U: x of row r0 + q
#pragma unroll
        for (int q = 0; q < U; ++q)
            if (lane == q) mine = fmaf(gamma, uq, dot[q]);
        if (lane < U && rq < n && r0 + lane < n) {
            u[rq] = mine;
            nrm = fma((double)mine, (double)mine, nrm);
        }
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const float x = __shfl_sync(0xffffffffu, mine, q);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                acc[c].x = fmaf(a[q][c].x, x, acc[c].x);
                acc[c].y = fmaf(a[q][c].y, x, acc[c].y);
                acc[c].z = fmaf(a[q][c].z, x, acc[c].z);
                acc[c].w = fmaf(a[q][c].w, x, acc[c].w);
            }
        }
        since += U;
        if (since >= kFold) {
            since = 0;
#pragma unroll
            for (int c = 0; c < NC; ++c) fold4(zw, c * 128 + lane * 4, d, acc[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) fold4(zw, c * 128 + lane * 4, d, acc[c]);
    nrm = warp_sum(nrm);
    if (lane == 0) ns[w] = nrm;
    __syncthreads();
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        double s = 0.0;
        for (int q = 0; q < kPassWarps; ++q) s += zs[q * d + j];
        zpart[(int64_t)blockIdx.x * d + j] = s;
    }
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < kPassWarps; ++q) s += ns[q];
        npart[blockIdx.x] = s;
    }
}

// The same pass for CSR A. Each warp keeps z = A^T x of its rows in its own FP32 shared-memory
// array (native shared-memory float atomics; a column of a sparse row gets few terms per warp, so
// FP32 adds about u_32 sqrt(terms) to a sum that LSQR uses at the 1e-6 level), summed over the
// warps in FP64 into the CTA's partial; t = N v sits in shared memory. k_lsqr_csr_short takes the rows of at most 8 entries, 8
// lanes a row and four rows a warp (a row is a chain of dependent loads: bounds, entries, t);
// k_lsqr_csr_long the others, a whole warp a row, found by scanning 32 row lengths at a time.
// Columns outside [0, d) count as zero.
__device__ __forceinline__ void csr_pass_finish(const float* zs, const double* ns, int d, double* zrow,
                                                double* nout) {
    __syncthreads();
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        double s = 0.0;
        for (int q = 0; q < kPassWarps; ++q) s += (double)zs[q * d + j];
        zrow[j] = s;
    }
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < kPassWarps; ++q) s += ns[q];
        *nout = s;
    }
}

__global__ void __launch_bounds__(32 * kPassWarps) k_lsqr_csr_short(const int64_t* __restrict__ row_ptr,
                                                                    const int32_t* __restrict__ col,
                                                                    const float* __restrict__ val, int64_t n, int d,
                                                                    const float* __restrict__ t,
                                                                    const double* __restrict__ state,
                                                                    float* __restrict__ u, double* __restrict__ zpart,
                                                                    double* __restrict__ npart) {
    extern __shared__ float zsf[];                      // kPassWarps x d, then t (d floats)
    __shared__ double ns[kPassWarps];
    if (state[S_DONE] != 0.0) return;
    float* zs = zsf;
    float* ts = zsf + kPassWarps * d;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, seg = lane >> 3, sl = lane & 7;
    const float gamma = (float)state[S_GAMMA];
    for (int j = threadIdx.x; j < kPassWarps * d; j += blockDim.x) zs[j] = 0.f;
    for (int j = threadIdx.x; j < d; j += blockDim.x) ts[j] = t[j];
    __syncthreads();
    float* zw = zs + w * d;
    double nrm = 0.0;
    const int64_t wid = (int64_t)blockIdx.x * kPassWarps + w, nw = (int64_t)gridDim.x * kPassWarps;
    // one-deep pipeline: the bounds and u of the next four rows load while this four runs
    int64_t rn = wid * 4 + seg;
    int64_t np0 = rn < n ? row_ptr[rn] : 0, np1 = rn < n ? row_ptr[rn + 1] : 0;
    float nu = (rn < n && sl == 0) ? u[rn] : 0.f;
    for (int64_t r0 = wid * 4; r0 < n; r0 += nw * 4) {
        const int64_t r = r0 + seg;
        const bool rok = r < n;
        const int64_t p0 = np0, p1 = np1;
        const float ur = nu;
        const int len = (int)(p1 - p0);
        const bool mine = rok && len <= 8;
        int c = -1;
        float a = 0.f;
        if (mine && sl < len) {
            c = col[p0 + sl];
            a = val[p0 + sl];
        }
        rn = r + nw * 4;
        np0 = rn < n ? row_ptr[rn] : 0;
        np1 = rn < n ? row_ptr[rn + 1] : 0;
        nu = (rn < n && sl == 0) ? u[rn] : 0.f;
        if ((unsigned)c >= (unsigned)d) { c = -1; a = 0.f; }
        float dot = c >= 0 ? a * ts[c] : 0.f;
        dot += __shfl_xor_sync(0xffffffffu, dot, 4);
        dot += __shfl_xor_sync(0xffffffffu, dot, 2);
        dot += __shfl_xor_sync(0xffffffffu, dot, 1);
        float x = 0.f;
        if (mine && sl == 0) {
            x = fmaf(gamma, ur, dot);
            u[r] = x;
            nrm = fma((double)x, (double)x, nrm);
        }
        x = __shfl_sync(0xffffffffu, x, seg * 8);
        if (c >= 0) atomicAdd(zw + c, a * x);
    }
    nrm = warp_sum(nrm);
    if (lane == 0) ns[w] = nrm;
    csr_pass_finish(zs, ns, d, zpart + (int64_t)blockIdx.x * d, npart + blockIdx.x);
}

__global__ void __launch_bounds__(32 * kPassWarps) k_lsqr_csr_long(const int64_t* __restrict__ row_ptr,
                                                                   const int32_t* __restrict__ col,
                                                                   const float* __restrict__ val, int64_t n, int d,
                                                                   const float* __restrict__ t,
                                                                   const double* __restrict__ state,
                                                                   float* __restrict__ u, double* __restrict__ zpart,
                                                                   double* __restrict__ npart) {
    extern __shared__ float zsf[];
    __shared__ double ns[kPassWarps];
    if (state[S_DONE] != 0.0) return;
    float* zs = zsf;
    float* ts = zsf + kPassWarps * d;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const float gamma = (float)state[S_GAMMA];
    for (int j = threadIdx.x; j < kPassWarps * d; j += blockDim.x) zs[j] = 0.f;
    for (int j = threadIdx.x; j < d; j += blockDim.x) ts[j] = t[j];
    __syncthreads();
    float* zw = zs + w * d;
    double nrm = 0.0;
    const int64_t wid = (int64_t)blockIdx.x * kPassWarps + w, nw = (int64_t)gridDim.x * kPassWarps;
    for (int64_t r0 = wid * 32; r0 < n; r0 += nw * 32) {
        const int64_t rl = r0 + lane;
        const int64_t lenl = rl < n ? row_ptr[rl + 1] - row_ptr[rl] : 0;
        unsigned todo = __ballot_sync(0xffffffffu, lenl > 8);
        while (todo) {
            const int b = __ffs(todo) - 1;
            todo &= todo - 1;
            const int64_t i = r0 + b;
            const int64_t p0 = row_ptr[i], p1 = row_ptr[i + 1];
            float dot = 0.f;
            for (int64_t e = p0 + lane; e < p1; e += 32) {
                const int c = col[e];
                if ((unsigned)c < (unsigned)d) dot = fmaf(val[e], ts[c], dot);
            }
            dot = warp_sum(dot);
            float x = 0.f;
            if (lane == 0) {
                x = fmaf(gamma, u[i], dot);
                u[i] = x;
                nrm = fma((double)x, (double)x, nrm);
            }
            x = __shfl_sync(0xffffffffu, x, 0);
            for (int64_t e = p0 + lane; e < p1; e += 32) {
                const int c = col[e];
                if ((unsigned)c < (unsigned)d) atomicAdd(zw + c, val[e] * x);
            }
        }
    }
    nrm = warp_sum(nrm);
    if (lane == 0) ns[w] = nrm;
    csr_pass_finish(zs, ns, d, zpart + (int64_t)blockIdx.x * d, npart + blockIdx.x);
}

// z[j] = sum over CTAs of zpart and beta = sqrt(sum of npart), in a fixed order: block b < gridDim.x
// - 1 takes columns 32b .. 32b + 31 (lane = column), warp w the partials w, w + 8, ..., then the
// warps' sums are added in warp order; the last block does the same for npart.
__global__ void __launch_bounds__(256) k_lsqr_reduce(const double* __restrict__ zpart, const double* __restrict__ npart,
                                                     int parts, int d, double* __restrict__ z,
                                                     double* __restrict__ state) {
    __shared__ double ws[8][32];
    if (state[S_DONE] != 0.0) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const bool last = blockIdx.x == gridDim.x - 1;
    const int j = blockIdx.x * 32 + lane;
    double s = 0.0;
    if (last) {
        for (int c = w * 32 + lane; c < parts; c += 256) s += npart[c];
        s = warp_sum(s);
    } else if (j < d) {
        for (int c = w; c < parts; c += 8) s += zpart[(int64_t)c * d + j];
    }
    ws[w][lane] = s;
    __syncthreads();
    if (w == 0) {
        double t = 0.0;
        for (int q = 0; q < 8; ++q) t += ws[q][lane];
        if (last) {
            if (lane == 0) state[S_BETA] = sqrt(t);
        } else if (j < d) {
            z[j] = t;
        }
    }
}

// vp[i] = (N^T z)[i] / beta - beta v[i]  (z = A^T u_unnormalised): one warp per i, lanes over j.
__global__ void k_lsqr_nt(const double* __restrict__ Nt, const double* __restrict__ z, const double* __restrict__ v,
                          int d, int k, const double* __restrict__ state, double* __restrict__ vp) {
    if (state[S_DONE] != 0.0) return;
    const int lane = threadIdx.x & 31;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= k) return;
    double s = 0.0;
    for (int j = lane; j < d; j += 32) s = fma(Nt[(int64_t)i * d + j], z[j], s);
    s = warp_sum(s);
    if (lane == 0) {
        const double beta = state[S_BETA];
        vp[i] = beta > 0.0 ? s / beta - beta * v[i] : 0.0;
    }
}

// The scalar part of an LSQR step, one CTA of 1024 threads (k <= 1024). init: the first step
// (alpha_1 v_1 = B^T u_1; w = v; phibar = beta_1; rhobar = alpha_1).
__global__ void __launch_bounds__(1024) k_lsqr_scalar(const double* __restrict__ vp, int k, int init,
                                                      double* __restrict__ v, double* __restrict__ w,
                                                      double* __restrict__ y, double* __restrict__ state) {
    __shared__ double red[32];
    __shared__ double coef[3];
    if (state[S_DONE] != 0.0) return;
    const int i = threadIdx.x, lane = i & 31, wq = i >> 5;
    const double x = i < k ? vp[i] : 0.0;
    double s = warp_sum(x * x);
    if (lane == 0) red[wq] = s;
    __syncthreads();
    if (wq == 0) {
        s = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        s = warp_sum(s);
        if (lane == 0) red[0] = s;
    }
    __syncthreads();
    const double alpha = sqrt(red[0]);
    const double beta = state[S_BETA];
    if (i == 0) {
        double phi_rho = 0.0, theta_rho = 0.0;
        if (init) {
            state[S_PHIBAR] = beta;
            state[S_RHOBAR] = alpha;
            state[S_BNORM2] = alpha * alpha;
            state[S_ITERS] = 0.0;
            state[S_BSTOP] = state[S_BSTOP] * beta;     // btol ||b||
            if (beta == 0.0 || alpha == 0.0) state[S_DONE] = 1.0;
        } else {
            const double rhobar = state[S_RHOBAR], phibar = state[S_PHIBAR];
            const double rho = hypot(rhobar, beta);
            const double c = rhobar / rho, sn = beta / rho;
            const double theta = sn * alpha;
            state[S_RHOBAR] = -c * alpha;
            const double phi = c * phibar;
            const double phibar2 = sn * phibar;
            state[S_PHIBAR] = phibar2;
            phi_rho = phi / rho;
            theta_rho = theta / rho;
            const double bn2 = state[S_BNORM2] + alpha * alpha + beta * beta;
            state[S_BNORM2] = bn2;
            state[S_ITERS] += 1.0;
            state[S_RNORM] = phibar2;
            state[S_ARNORM] = phibar2 * alpha * fabs(c);
            if (state[S_ARNORM] <= state[S_ATOL] * sqrt(bn2) * phibar2 || phibar2 <= state[S_BSTOP] || alpha == 0.0)
                state[S_DONE] = 1.0;
        }
        state[S_ALPHA] = alpha;
        state[S_SU] = beta > 0.0 ? 1.0 / beta : 0.0;
        state[S_GAMMA] = beta > 0.0 ? -alpha / beta : 0.0;     // next pass: A t - alpha u, u = stored / beta
        coef[0] = alpha;
        coef[1] = phi_rho;
        coef[2] = theta_rho;
    }
    __syncthreads();
    if (i < k) {
        const double vn = coef[0] > 0.0 ? x / coef[0] : 0.0;
        if (init) {
            v[i] = vn;
            w[i] = vn;
            y[i] = 0.0;
        } else {
            y[i] = fma(coef[1], w[i], y[i]);
            w[i] = fma(-coef[2], w[i], vn);
            v[i] = vn;
        }
    }
}

// t[j] = (N v)[j] as FP32 (next pass) or x[j] = (N y)[j] as FP64: one warp per j, lanes over i.
__global__ void k_lsqr_nv(const double* __restrict__ N, const double* __restrict__ v, int d, int k,
                          const double* __restrict__ state, int check_done, float* __restrict__ t32,
                          double* __restrict__ x64) {
    if (check_done && state[S_DONE] != 0.0) return;
    const int lane = threadIdx.x & 31;
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (j >= d) return;
    double s = 0.0;
    for (int i = lane; i < k; i += 32) s = fma(N[(int64_t)j * d + i], v[i], s);
    s = warp_sum(s);
    if (lane == 0) {
        if (t32) t32[j] = (float)s;
        if (x64) x64[j] = s;
    }
}

__global__ void k_lsqr_init_state(double* state, double atol, double btol) {
    if (threadIdx.x == 0) {
        for (int q = 0; q < S_COUNT; ++q) state[q] = 0.0;
        state[S_GAMMA] = 1.0;                           // first pass: x_r = 0 + 1 * b_r
        state[S_ATOL] = atol;
        state[S_BSTOP] = btol;
    }
}

}  // namespace

// ws layout: state (S_COUNT, padded to +8), v, w, y, vp, z (d each), t (d FP32), zpart (parts x d),
// npart (parts), Nt (d x d).
size_t lsqr_scratch_doubles(int64_t d, int parts) {
    return (size_t)(S_COUNT + 8 + 5 * d + d / 2 + 2 + (size_t)parts * (d + 1) + (size_t)d * d);
}

// Partial rows of z: the CSR pass uses 8 per SM (6 for the short rows: many warps hide the chain of
// dependent loads of a row), the dense pass 3 per SM; the workspace holds the larger count.
int lsqr_parts(int num_sms) { return num_sms * 8; }

int lsqr_state_doubles() { return S_COUNT; }

cudaError_t launch_precond_n(const double* Y, const int32_t* order, const double* sigma, const int32_t* perm,
                             const int64_t* d_rank, int64_t d, double* N, cudaStream_t st) {
    int grid = (int)((d * d + 255) / 256);
    if (grid > 152 * 8) grid = 152 * 8;
    k_precond_n<<<grid, 256, 0, st>>>(Y, order, sigma, perm, d_rank, (int)d, N);
    return cudaGetLastError();
}

template <int NC, int U>
static cudaError_t lsqr_pass(bool vec, int parts, size_t smem, cudaStream_t st, const float* A, int64_t lda, int64_t n,
                             int d, const float* t, const double* state, float* u, double* zpart, double* npart) {
    cudaError_t e;
    const int mx = (int)(sizeof(double) * kPassWarps * 1024);
    if (vec) {
        if ((e = cudaFuncSetAttribute(k_lsqr_pass<NC, U, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx)) !=
            cudaSuccess)
            return e;
        k_lsqr_pass<NC, U, true><<<parts, 32 * kPassWarps, smem, st>>>(A, lda, n, d, t, state, u, zpart, npart);
    } else {
        if ((e = cudaFuncSetAttribute(k_lsqr_pass<NC, U, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx)) !=
            cudaSuccess)
            return e;
        k_lsqr_pass<NC, U, false><<<parts, 32 * kPassWarps, smem, st>>>(A, lda, n, d, t, state, u, zpart, npart);
    }
    return cudaGetLastError();
}

cudaError_t launch_lsqr(const float* A, int64_t lda, const int64_t* row_ptr, const int32_t* col, const float* val,
                        int64_t n, int64_t d, const double* N, int64_t k, float* u,
                        double* x, int max_iter, double atol, double btol, double* ws, int parts, double* host_state,
                        int* iters_out, double* rnorm_out, cudaStream_t st) {
    cudaError_t e;
    if (d > 1024 || k < 1 || k > d) return cudaErrorInvalidValue;
    double* state = ws;
    double* v = ws + S_COUNT + 8;
    double* w = v + d;
    double* y = w + d;
    double* vp = y + d;
    double* z = vp + d;
    float* t = reinterpret_cast<float*>(z + d);
    double* zpart = z + d + d / 2 + 2;
    double* npart = zpart + (size_t)parts * d;
    double* Nt = npart + parts;
    const int nc = (int)((d + 127) / 128);
    const bool vec = A && (reinterpret_cast<uintptr_t>(A) % 16 == 0) && (lda % 4 == 0);
    const size_t smem = sizeof(double) * (size_t)kPassWarps * d;
    const bool csr = row_ptr != nullptr;
    const int parts_s = parts * 3 / 4, parts_l = parts - parts_s;
    if (!csr) parts = parts * 3 / 8;                    // dense: 3 CTAs a SM
    const size_t smem_csr = sizeof(float) * (size_t)(kPassWarps + 1) * d;
    if (csr) {
        const int mx = (int)(sizeof(float) * (kPassWarps + 1) * 1024);
        if ((e = cudaFuncSetAttribute(k_lsqr_csr_short, cudaFuncAttributeMaxDynamicSharedMemorySize, mx)) != cudaSuccess)
            return e;
        if ((e = cudaFuncSetAttribute(k_lsqr_csr_long, cudaFuncAttributeMaxDynamicSharedMemorySize, mx)) != cudaSuccess)
            return e;
    }
    auto pass = [&]() -> cudaError_t {
        if (csr) {
            k_lsqr_csr_short<<<parts_s, 32 * kPassWarps, smem_csr, st>>>(row_ptr, col, val, n, (int)d, t, state, u,
                                                                         zpart, npart);
            k_lsqr_csr_long<<<parts_l, 32 * kPassWarps, smem_csr, st>>>(row_ptr, col, val, n, (int)d, t, state, u,
                                                                        zpart + (size_t)parts_s * d, npart + parts_s);
            return cudaGetLastError();
        }
        if (nc == 1) return lsqr_pass<1, 8>(vec, parts, smem, st, A, lda, n, (int)d, t, state, u, zpart, npart);
        if (nc == 2) return lsqr_pass<2, 4>(vec, parts, smem, st, A, lda, n, (int)d, t, state, u, zpart, npart);
        if (nc <= 4) return lsqr_pass<4, 2>(vec, parts, smem, st, A, lda, n, (int)d, t, state, u, zpart, npart);
        return lsqr_pass<8, 1>(vec, parts, smem, st, A, lda, n, (int)d, t, state, u, zpart, npart);
    };
    int tg = (int)((k * d + 255) / 256);
    if (tg > 152 * 8) tg = 152 * 8;
    k_transpose_n<<<tg, 256, 0, st>>>(N, (int)d, (int)k, Nt);
    const int warps_k = (int)((k * 32 + 255) / 256), warps_d = (int)((d * 32 + 255) / 256);
    const int red_grid = (int)((d + 31) / 32) + 1;
    k_lsqr_init_state<<<1, 32, 0, st>>>(state, atol, btol);
    if ((e = cudaMemsetAsync(t, 0, sizeof(float) * (size_t)d, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(v, 0, sizeof(double) * (size_t)d, st)) != cudaSuccess) return e;
    // beta_1 u_1 = b (u holds b), alpha_1 v_1 = N^T A^T u_1
    if ((e = pass()) != cudaSuccess) return e;
    k_lsqr_reduce<<<red_grid, 256, 0, st>>>(zpart, npart, parts, (int)d, z, state);
    k_lsqr_nt<<<warps_k, 256, 0, st>>>(Nt, z, v, (int)d, (int)k, state, vp);
    k_lsqr_scalar<<<1, 1024, 0, st>>>(vp, (int)k, 1, v, w, y, state);
    k_lsqr_nv<<<warps_d, 256, 0, st>>>(N, v, (int)d, (int)k, state, 1, t, nullptr);
    constexpr int kCheck = 16;
    int it = 0;
    while (it < max_iter) {
        const int batch = (max_iter - it) < kCheck ? (max_iter - it) : kCheck;
        for (int b = 0; b < batch; ++b) {
            if ((e = pass()) != cudaSuccess) return e;
            k_lsqr_reduce<<<red_grid, 256, 0, st>>>(zpart, npart, parts, (int)d, z, state);
            k_lsqr_nt<<<warps_k, 256, 0, st>>>(Nt, z, v, (int)d, (int)k, state, vp);
            k_lsqr_scalar<<<1, 1024, 0, st>>>(vp, (int)k, 0, v, w, y, state);
            k_lsqr_nv<<<warps_d, 256, 0, st>>>(N, v, (int)d, (int)k, state, 1, t, nullptr);
        }
        it += batch;
        if ((e = cudaMemcpyAsync(host_state, state, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return e;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
        if (host_state[S_DONE] != 0.0) break;
    }
    k_lsqr_nv<<<warps_d, 256, 0, st>>>(N, y, (int)d, (int)k, state, 0, nullptr, x);
    if ((e = cudaMemcpyAsync(host_state, state, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    if (iters_out) *iters_out = (int)host_state[S_ITERS];
    if (rnorm_out) *rnorm_out = host_state[S_RNORM];
    return cudaGetLastError();
}

}  // namespace lev
