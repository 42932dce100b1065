// Ground state of H_S by Lanczos on the device.
//
// The paper hands its matrix-free operator to external eigensolvers (ARPACK,
// PRIMME; Results and Methods "Matrix evaluation").  Here the solver runs on
// the GPU next to the product: per step, y = H v_j, then classical
// Gram-Schmidt against all previous vectors applied twice (FP64 dots), the
// norm, and the next vector; every `check_every` steps one CTA solves the
// tridiagonal problem (multisection on Sturm counts for the lowest
// eigenvalue, inverse iteration for its eigenvector) and the host reads the
// residual estimate beta_{j+1} |s_j| through pinned memory.
//
// Mixed precision: the Krylov basis and the products are FP32 (FP64 dots,
// FP64 tridiagonal); the Ritz vector is then formed in FP64 and refined by
// short FP64 Lanczos restarts from it until its FP64 residual meets `tol` or
// the Rayleigh quotient stops moving.
#include <algorithm>
#include <chrono>
#include <cmath>

#include "qsd_internal.cuh"

namespace qsd {

namespace {

constexpr int kRedThreads = 256;
constexpr int kMaxSteps = 700;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum; result valid in thread 0.
__device__ double block_sum(double v, double *sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (warp == 0) {
        r = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
        r = warp_sum(r);
    }
    __syncthreads();
    return r;
}

__device__ __forceinline__ double uniform_pm1(uint64_t seed, uint64_t i) {
    uint64_t z = (seed ^ i) + 0x9E3779B97F4A7C15ull;
    z = fmix64(z);
    return 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
}

template <typename TV>
__global__ void k_start(TV *v, int64_t D, uint64_t seed, const double *v0, double *w) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= D) return;
    const double x = v0 ? v0[i] : uniform_pm1(seed, (uint64_t)i);
    w[i] = x;
}

// partial[i * B + b] = sum over the block's rows of V[i][r] u[r], i < nvec
template <typename TV, typename TU>
__global__ void k_gemv_t(const TV *__restrict__ V, int64_t D, int nvec, const TU *__restrict__ u, double *partial) {
    __shared__ double sh[32];
    const int B = gridDim.x;
    const int64_t chunk = (D + B - 1) / B;
    const int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = min(D, r0 + chunk);
    for (int i = 0; i < nvec; ++i) {
        const TV *vi = V + (size_t)i * D;
        double s = 0.0;
        for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) s = fma((double)vi[r], (double)u[r], s);
        s = block_sum(s, sh);
        if (threadIdx.x == 0) partial[(size_t)i * B + blockIdx.x] = s;
    }
}

// h[i] = sum_b partial[i][b] (fixed order); optionally alpha += h[j]
__global__ void k_reduce_rows(const double *__restrict__ partial, int nvec, int B, double *h, double *alpha_j,
                              int j) {
    __shared__ double sh[32];
    const int i = blockIdx.x;
    if (i >= nvec) return;
    double s = 0.0;
    for (int b = threadIdx.x; b < B; b += blockDim.x) s += partial[(size_t)i * B + b];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
        h[i] = s;
        if (alpha_j && i == j) *alpha_j += s;
    }
}

// w[r] = u[r] - sum_i V[i][r] h[i]
template <typename TV, typename TU>
__global__ void k_gemv_sub(const TV *__restrict__ V, int64_t D, int nvec, const double *__restrict__ h,
                           const TU *u, double *w) {
    extern __shared__ double hs[];
    for (int i = threadIdx.x; i < nvec; i += blockDim.x) hs[i] = h[i];
    __syncthreads();
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= D) return;
    double acc = (double)u[r];
    for (int i = 0; i < nvec; ++i) acc = fma(-(double)V[(size_t)i * D + r], hs[i], acc);
    w[r] = acc;
}

__global__ void k_sq_partial(const double *__restrict__ w, int64_t D, double *partial) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < D; r += (int64_t)gridDim.x * blockDim.x)
        s = fma(w[r], w[r], s);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void k_sqrt_sum(const double *__restrict__ partial, int B, double *out) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int b = threadIdx.x; b < B; b += blockDim.x) s += partial[b];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) *out = sqrt(s);
}

template <typename TV>
__global__ void k_scale_to(const double *__restrict__ w, const double *__restrict__ nrm, int64_t D, TV *v) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= D) return;
    const double s = *nrm;
    v[r] = (TV)(s > 0.0 ? w[r] / s : 0.0);
}

__global__ void k_axpy_res(const double *__restrict__ hu, const double *__restrict__ u, const double *__restrict__ theta,
                           int64_t D, double *r) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= D) return;
    r[i] = hu[i] - (*theta) * u[i];
}

__global__ void k_dot_partial(const double *__restrict__ a, const double *__restrict__ b, int64_t D, double *partial) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < D; r += (int64_t)gridDim.x * blockDim.x)
        s = fma(a[r], b[r], s);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void k_sum(const double *__restrict__ partial, int B, double *out) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int b = threadIdx.x; b < B; b += blockDim.x) s += partial[b];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) *out = s;
}

// ------------------------------------------------------------- tridiagonal
// Number of eigenvalues of T (diagonal a[0..m), off-diagonal b[1..m)) below x.
__device__ int sturm(const double *a, const double *b, int m, double x) {
    int c = 0;
    double q = 1.0;
    for (int i = 0; i < m; ++i) {
        q = a[i] - x - (i ? b[i] * b[i] / q : 0.0);
        if (q == 0.0) q = -1e-300;
        c += q < 0.0;
    }
    return c;
}

// One CTA.  out[0] = theta (lowest eigenvalue), out[1] = |beta_m s_{m-1}|
// (residual estimate), out[2..2+m) = unit eigenvector s.
__global__ void k_tridiag(const double *__restrict__ alpha, const double *__restrict__ beta, int m, double *out) {
    extern __shared__ double sm[];
    double *a = sm, *b = sm + m, *s = sm + 2 * m;
    __shared__ double lo_hi[2];
    __shared__ int cnt[kRedThreads];
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        a[i] = alpha[i];
        b[i] = i ? beta[i] : 0.0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double lo = a[0], hi = a[0];
        for (int i = 0; i < m; ++i) {
            const double rad = (i ? fabs(b[i]) : 0.0) + (i + 1 < m ? fabs(b[i + 1]) : 0.0);
            lo = fmin(lo, a[i] - rad);
            hi = fmax(hi, a[i] + rad);
        }
        const double pad = 1e-12 * fmax(fabs(lo), fabs(hi)) + 1e-300;
        lo_hi[0] = lo - pad;
        lo_hi[1] = hi + pad;
    }
    __syncthreads();
    // multisection: each thread tests one of blockDim.x interior points
    for (int it = 0; it < 64; ++it) {
        const double lo = lo_hi[0], hi = lo_hi[1];
        const double x = lo + (hi - lo) * (double)(threadIdx.x + 1) / (double)(blockDim.x + 1);
        cnt[threadIdx.x] = sturm(a, b, m, x);
        __syncthreads();
        if (threadIdx.x == 0) {
            int k = 0;
            while (k < (int)blockDim.x && cnt[k] < 1) ++k;
            const double nlo = k == 0 ? lo : lo + (hi - lo) * (double)k / (double)(blockDim.x + 1);
            const double nhi = k == (int)blockDim.x ? hi : lo + (hi - lo) * (double)(k + 1) / (double)(blockDim.x + 1);
            lo_hi[0] = nlo;
            lo_hi[1] = nhi;
        }
        __syncthreads();
        if (lo_hi[1] - lo_hi[0] <= 4e-16 * fmax(fabs(lo_hi[0]), fabs(lo_hi[1])) + 1e-300) break;
    }
    if (threadIdx.x != 0) return;
    const double theta = 0.5 * (lo_hi[0] + lo_hi[1]);
    // Inverse iteration (T - theta I) s = rhs.  Gaussian elimination with
    // partial pivoting on the tridiagonal matrix gives an upper factor with
    // two super-diagonals (D_, U1, U2), multipliers Lm and swap flags piv.
    double scale = 0.0;
    for (int i = 0; i < m; ++i) scale = fmax(scale, fabs(a[i]) + fabs(b[i]));
    const double tiny = 1e-14 * fmax(scale, 1e-300);
    double *D_ = sm + 3 * m, *U1 = sm + 4 * m, *U2 = sm + 5 * m, *Lm = sm + 6 * m;
    int *piv = reinterpret_cast<int *>(sm + 7 * m);
    for (int i = 0; i < m; ++i) {
        D_[i] = a[i] - theta;
        U1[i] = i + 1 < m ? b[i + 1] : 0.0;
        U2[i] = 0.0;
    }
    for (int i = 0; i + 1 < m; ++i) {
        const double sub = b[i + 1];  // entry (i+1, i)
        if (fabs(sub) > fabs(D_[i])) {
            // row i+1 (still original: sub, D_[i+1], U1[i+1]) becomes the pivot row
            piv[i] = 1;
            const double mult = D_[i] / sub;
            Lm[i] = mult;
            const double u0 = U1[i], w0 = U2[i];
            D_[i] = sub;
            U1[i] = D_[i + 1];
            U2[i] = U1[i + 1];
            D_[i + 1] = u0 - mult * U1[i];
            U1[i + 1] = w0 - mult * U2[i];
        } else {
            piv[i] = 0;
            if (fabs(D_[i]) < tiny) D_[i] = D_[i] >= 0 ? tiny : -tiny;
            const double mult = sub / D_[i];
            Lm[i] = mult;
            D_[i + 1] -= mult * U1[i];
        }
    }
    if (fabs(D_[m - 1]) < tiny) D_[m - 1] = D_[m - 1] >= 0 ? tiny : -tiny;
    for (int i = 0; i < m; ++i) s[i] = 1.0;
    for (int iter = 0; iter < 3; ++iter) {
        for (int i = 0; i + 1 < m; ++i) {
            if (piv[i]) {
                const double t = s[i];
                s[i] = s[i + 1];
                s[i + 1] = t - Lm[i] * s[i];
            } else {
                s[i + 1] -= Lm[i] * s[i];
            }
        }
        for (int i = m - 1; i >= 0; --i) {
            double v = s[i];
            if (i + 1 < m) v -= U1[i] * s[i + 1];
            if (i + 2 < m) v -= U2[i] * s[i + 2];
            s[i] = v / D_[i];
        }
        double nrm = 0.0;
        for (int i = 0; i < m; ++i) nrm += s[i] * s[i];
        nrm = sqrt(nrm);
        for (int i = 0; i < m; ++i) s[i] /= nrm;
    }
    out[0] = theta;
    out[1] = fabs(beta[m] * s[m - 1]);
    for (int i = 0; i < m; ++i) out[2 + i] = s[i];
}

// u[r] = sum_i V[i][r] s[i]
template <typename TV>
__global__ void k_ritz(const TV *__restrict__ V, int64_t D, int nvec, const double *__restrict__ s, double *u) {
    extern __shared__ double ss[];
    for (int i = threadIdx.x; i < nvec; i += blockDim.x) ss[i] = s[i];
    __syncthreads();
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= D) return;
    double acc = 0.0;
    for (int i = 0; i < nvec; ++i) acc = fma((double)V[(size_t)i * D + r], ss[i], acc);
    u[r] = acc;
}

struct Krylov {
    int64_t D = 0;
    int m = 0;
    bool fp32 = false;
    int B = 0;
    DevBuf V, hv, w, h, partial, alpha, beta, tri, scal;
};

size_t tri_smem(int m) { return (size_t)8 * m * 8 + 64; }

// Runs up to p_steps Lanczos steps from start vector `start` (FP64 [D]) and
// returns the lowest Ritz value; the Ritz vector goes to u (FP64 [D]).
struct LanczosResult {
    double theta = 0.0, est = 0.0;
    int steps = 0;
    bool converged = false;
    bool timeout = false;
};

template <typename TV>
LanczosResult run_lanczos(qsd_ctx ctx, qsd_op op, qsd_sub sub, const double *diag, Krylov &K, const double *start,
                          uint64_t seed, int max_steps, double tol, int check_every, double *u,
                          std::chrono::steady_clock::time_point deadline, bool has_deadline, int *applies,
                          int prec32 = QSD_FP32_DOT2) {
    cudaStream_t s = ctx->stream;
    const int64_t D = K.D;
    const int m = std::min<int64_t>(max_steps, D);
    const int prec = std::is_same<TV, float>::value ? prec32 : QSD_FP64;
    TV *V = K.V.as<TV>();
    TV *hv = K.hv.as<TV>();
    double *w = K.w.as<double>(), *h = K.h.as<double>(), *part = K.partial.as<double>();
    double *alpha = K.alpha.as<double>(), *beta = K.beta.as<double>(), *tri = K.tri.as<double>();
    double *scal = K.scal.as<double>();
    const int nbD = blocks_for(D, 256);
    const int B = K.B;
    QSD_CUDA(cudaMemsetAsync(alpha, 0, (size_t)(K.m + 1) * 8, s));
    QSD_CUDA(cudaMemsetAsync(beta, 0, (size_t)(K.m + 2) * 8, s));
    // v_0 = start / |start|
    k_start<TV><<<nbD, 256, 0, s>>>(V, D, seed, start, w);
    k_sq_partial<<<B, kRedThreads, 0, s>>>(w, D, part);
    k_sqrt_sum<<<1, kRedThreads, 0, s>>>(part, B, scal);
    k_scale_to<TV><<<nbD, 256, 0, s>>>(w, scal, D, V);
    QSD_LAUNCH_CHECK();
    LanczosResult res;
    double *h_tri = nullptr;
    QSD_CUDA(cudaMallocHost(&h_tri, 32));
    int j = 0;
    try {
        for (j = 0; j < m; ++j) {
            const TV *vj = V + (size_t)j * D;
            apply_H(ctx, op, sub, diag, prec, 1, vj, hv, s);
            ++*applies;
            const int nvec = j + 1;
            const size_t hsm = (size_t)nvec * 8;
            // pass 1: h = V^T hv ; w = hv - V h ; alpha_j = h_j
            k_gemv_t<TV, TV><<<B, kRedThreads, 0, s>>>(V, D, nvec, hv, part);
            k_reduce_rows<<<nvec, 128, 0, s>>>(part, nvec, B, h, alpha + j, j);
            k_gemv_sub<TV, TV><<<nbD, 256, hsm, s>>>(V, D, nvec, h, hv, w);
            // pass 2: h = V^T w ; w -= V h ; alpha_j += h_j
            k_gemv_t<TV, double><<<B, kRedThreads, 0, s>>>(V, D, nvec, w, part);
            k_reduce_rows<<<nvec, 128, 0, s>>>(part, nvec, B, h, alpha + j, j);
            k_gemv_sub<TV, double><<<nbD, 256, hsm, s>>>(V, D, nvec, h, w, w);
            // beta_{j+1} = |w|, v_{j+1} = w / beta_{j+1}
            k_sq_partial<<<B, kRedThreads, 0, s>>>(w, D, part);
            k_sqrt_sum<<<1, kRedThreads, 0, s>>>(part, B, beta + j + 1);
            if (j + 1 < K.m + 1 && j + 1 < m) k_scale_to<TV><<<nbD, 256, 0, s>>>(w, beta + j + 1, D, V + (size_t)(j + 1) * D);
            QSD_LAUNCH_CHECK();
            const bool last = (j + 1 == m);
            if ((j + 1) % check_every == 0 || last) {
                k_tridiag<<<1, kRedThreads, tri_smem(nvec), s>>>(alpha, beta, nvec, tri);
                QSD_LAUNCH_CHECK();
                QSD_CUDA(cudaMemcpyAsync(h_tri, tri, 16, cudaMemcpyDeviceToHost, s));
                QSD_CUDA(cudaMemcpyAsync(h_tri + 2, beta + j + 1, 8, cudaMemcpyDeviceToHost, s));
                QSD_CUDA(cudaStreamSynchronize(s));
                const double hb = h_tri[2];
                res.theta = h_tri[0];
                res.est = h_tri[1];
                res.steps = j + 1;
                const double at = std::max(std::fabs(res.theta), 1e-300);
                if (res.est <= tol * at || hb <= 1e-13 * at) {
                    res.converged = true;
                    break;
                }
                if (has_deadline && std::chrono::steady_clock::now() > deadline) {
                    res.timeout = true;
                    break;
                }
            }
        }
        // Ritz vector u = V[0..n) s
        const int nvec = res.steps;
        k_ritz<TV><<<nbD, 256, (size_t)nvec * 8, s>>>(V, D, nvec, tri + 2, u);
        QSD_LAUNCH_CHECK();
        // normalise u in FP64
        k_sq_partial<<<B, kRedThreads, 0, s>>>(u, D, part);
        k_sqrt_sum<<<1, kRedThreads, 0, s>>>(part, B, scal);
        k_scale_to<double><<<nbD, 256, 0, s>>>(u, scal, D, u);
        QSD_LAUNCH_CHECK();
        QSD_CUDA(cudaStreamSynchronize(s));
    } catch (...) {
        cudaFreeHost(h_tri);
        throw;
    }
    cudaFreeHost(h_tri);
    return res;
}

void alloc_krylov(qsd_ctx ctx, Krylov &K, int64_t D, int m, bool fp32) {
    K.D = D;
    K.m = m;
    K.fp32 = fp32;
    K.B = std::max(1, std::min<int>(2 * ctx->num_sms, (int)((D + 255) / 256)));
    const size_t sv = fp32 ? 4 : 8;
    K.V.alloc((size_t)(m + 1) * D * sv);
    K.hv.alloc((size_t)D * sv);
    K.w.alloc((size_t)D * 8);
    K.h.alloc((size_t)(m + 2) * 8);
    K.partial.alloc((size_t)(m + 2) * K.B * 8);
    K.alpha.alloc((size_t)(m + 2) * 8);
    K.beta.alloc((size_t)(m + 3) * 8);
    K.tri.alloc((size_t)(m + 4) * 8);
    K.scal.alloc(32);
}

// FP64 residual and Rayleigh quotient of a unit vector u: returns (theta, |Hu - theta u|)
std::pair<double, double> fp64_residual(qsd_ctx ctx, qsd_op op, qsd_sub sub, const double *diag, const double *u,
                                        double *hu, double *r, double *part, int B, double *scal, int *applies) {
    cudaStream_t s = ctx->stream;
    const int64_t D = sub->D;
    apply_H(ctx, op, sub, diag, QSD_FP64, 1, u, hu, s);
    ++*applies;
    k_dot_partial<<<B, kRedThreads, 0, s>>>(u, hu, D, part);
    k_sum<<<1, kRedThreads, 0, s>>>(part, B, scal);
    k_axpy_res<<<blocks_for(D, 256), 256, 0, s>>>(hu, u, scal, D, r);
    k_sq_partial<<<B, kRedThreads, 0, s>>>(r, D, part);
    k_sqrt_sum<<<1, kRedThreads, 0, s>>>(part, B, scal + 1);
    QSD_LAUNCH_CHECK();
    double h[2];
    QSD_CUDA(cudaMemcpyAsync(h, scal, 16, cudaMemcpyDeviceToHost, s));
    QSD_CUDA(cudaStreamSynchronize(s));
    return {h[0], h[1]};
}

}  // namespace

void rayleigh_quotient(qsd_ctx ctx, qsd_op op, qsd_sub sub, const double *diag, const double *u, double *out) {
    cudaStream_t s = ctx->stream;
    const int64_t D = sub->D;
    const int B = std::max(1, std::min<int>(2 * ctx->num_sms, (int)((D + 255) / 256)));
    double *hu = static_cast<double *>(ctx->scratch[2].get((size_t)D * 8));
    double *part = static_cast<double *>(ctx->scratch[3].get((size_t)4 * 2048 * 8));
    double *scal = part + 3 * 2048;
    apply_H(ctx, op, sub, diag, QSD_FP64, 1, u, hu, s);
    k_dot_partial<<<B, kRedThreads, 0, s>>>(u, hu, D, part);
    k_sum<<<1, kRedThreads, 0, s>>>(part, B, scal);            // u^T H u
    k_dot_partial<<<B, kRedThreads, 0, s>>>(u, u, D, part + 2048);
    k_sum<<<1, kRedThreads, 0, s>>>(part + 2048, B, scal + 1); // u^T u
    QSD_LAUNCH_CHECK();
    double h[2];
    QSD_CUDA(cudaMemcpyAsync(h, scal, 16, cudaMemcpyDeviceToHost, s));
    QSD_CUDA(cudaStreamSynchronize(s));
    if (!(h[1] > 0.0)) fail(QSD_ERR_INVALID_ARG, "rayleigh_quotient: u is zero");
    const double theta = h[0] / h[1];
    QSD_CUDA(cudaMemcpyAsync(scal + 2, &theta, 8, cudaMemcpyHostToDevice, s));
    // r = H u - theta u, |r|^2
    k_axpy_res<<<blocks_for(D, 256), 256, 0, s>>>(hu, u, scal + 2, D, hu);
    k_sq_partial<<<B, kRedThreads, 0, s>>>(hu, D, part);
    k_sqrt_sum<<<1, kRedThreads, 0, s>>>(part, B, scal + 3);
    QSD_LAUNCH_CHECK();
    double rn = 0.0;
    QSD_CUDA(cudaMemcpyAsync(&rn, scal + 3, 8, cudaMemcpyDeviceToHost, s));
    QSD_CUDA(cudaStreamSynchronize(s));
    out[0] = theta;
    out[1] = rn / std::sqrt(h[1]);
    out[2] = h[1];
}

int lanczos_ground_state(qsd_ctx ctx, qsd_op op, qsd_sub sub, const qsd_lanczos_params &p, double *energy,
                         double *vec_out, qsd_lanczos_info *info) {
    const auto t0 = std::chrono::steady_clock::now();
    const bool has_deadline = p.time_limit_s > 0.0;
    const auto deadline = t0 + std::chrono::microseconds((int64_t)(p.time_limit_s * 1e6));
    Binding *bind = get_binding(ctx, op, sub);
    const double *diag = bind->diag.as<double>();
    const int64_t D = sub->D;
    const bool mixed = p.precision != QSD_FP64;
    // the tridiagonal CTA keeps 8 m doubles in shared memory (<= 48 KB)
    const int m = (int)std::min<int64_t>(std::min(p.max_steps, kMaxSteps), D);
    const double tol = p.tol > 0 ? p.tol : 1e-9;
    int applies = 0;
    DevBuf u((size_t)D * 8), hu((size_t)D * 8), r((size_t)D * 8);
    LanczosResult res;
    int total_steps = 0, restarts = 0;
    double e_unrefined = 0.0;
    Krylov K;
    {
        alloc_krylov(ctx, K, D, m, mixed);
        // the FP32 phase stops where FP32 round-off limits the estimate
        const double phase_tol = mixed ? std::max(tol, 1e-5) : tol;
        if (mixed)
            res = run_lanczos<float>(ctx, op, sub, diag, K, p.v0, p.seed, m, phase_tol, p.check_every, u.as<double>(),
                                     deadline, has_deadline, &applies, p.precision);
        else
            res = run_lanczos<double>(ctx, op, sub, diag, K, p.v0, p.seed, m, phase_tol, p.check_every,
                                      u.as<double>(), deadline, has_deadline, &applies);
        total_steps += res.steps;
    }
    e_unrefined = res.theta;
    auto rq = fp64_residual(ctx, op, sub, diag, u.as<double>(), hu.as<double>(), r.as<double>(), K.partial.as<double>(),
                            K.B, K.scal.as<double>(), &applies);
    double theta = mixed ? rq.first : res.theta;
    double resid = rq.second / std::max(std::fabs(rq.first), 1e-300);
    bool converged = resid <= tol || (res.converged && !mixed && res.est <= tol * std::fabs(res.theta));
    if (mixed) {
        // FP64 restarts from the current Ritz vector
        Krylov K64;
        const int ms = (int)std::min<int64_t>(std::min(std::max(p.refine_steps, 2), kMaxSteps), D);
        alloc_krylov(ctx, K64, D, ms, false);
        double prev = theta;
        const double rtol = p.refine_tol > 0 ? p.refine_tol : 1e-10;
        while (!converged && restarts < std::max(p.max_refine, 0)) {
            if (has_deadline && std::chrono::steady_clock::now() > deadline) { res.timeout = true; break; }
            QSD_CUDA(cudaMemcpyAsync(r.p, u.p, (size_t)D * 8, cudaMemcpyDeviceToDevice, ctx->stream));
            LanczosResult rr = run_lanczos<double>(ctx, op, sub, diag, K64, r.as<double>(), p.seed, ms, tol,
                                                   std::min(p.check_every, ms), u.as<double>(), deadline,
                                                   has_deadline, &applies);
            total_steps += rr.steps;
            ++restarts;
            rq = fp64_residual(ctx, op, sub, diag, u.as<double>(), hu.as<double>(), r.as<double>(),
                               K64.partial.as<double>(), K64.B, K64.scal.as<double>(), &applies);
            theta = rq.first;
            resid = rq.second / std::max(std::fabs(theta), 1e-300);
            const double change = std::fabs(theta - prev) / std::max(std::fabs(theta), 1e-300);
            prev = theta;
            if (resid <= tol || change <= rtol) converged = true;
        }
    } else if (!converged) {
        converged = res.converged;
    }
    *energy = theta;
    if (vec_out) QSD_CUDA(cudaMemcpyAsync(vec_out, u.p, (size_t)D * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    QSD_CUDA(cudaStreamSynchronize(ctx->stream));
    if (info) {
        info->steps = total_steps;
        info->refine_restarts = restarts;
        info->residual = resid;
        info->energy_unrefined = e_unrefined;
        info->applies = applies;
    }
    if (take_device_error(ctx)) fail(QSD_ERR_INTERNAL, "lanczos: hash probe exceeded the table size");
    if (res.timeout) return QSD_ERR_TIMEOUT;
    return converged ? QSD_OK : QSD_ERR_NOT_CONVERGED;
}

}  // namespace qsd
