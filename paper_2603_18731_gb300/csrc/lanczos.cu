// Ground state of H_S by Lanczos on the device.
//
// The paper hands its matrix-free operator to external eigensolvers (ARPACK,
// PRIMME; Results, and Methods "Matrix evaluation").  Here the solver runs on
// the GPU next to the product.  Per step: u = H q_j; the three-term
// recurrence, then one classical Gram-Schmidt pass against all previous
// vectors with FP64 dots (complete reorthogonalisation, below); alpha_j and
// beta_{j+1} = |w|; q_{j+1} = w / beta_{j+1}.
// Every `check_every` steps one CTA solves the tridiagonal problem
// (multisection on Sturm counts for the lowest eigenvalue, inverse iteration
// for its eigenvector) and the residual estimate beta_{j+1} |s_j| reaches the
// host through pinned memory.
//
// The step index lives in device memory and every kernel reads it, so one
// chunk of `check_every` steps is a fixed sequence of launches: it is captured
// once into a CUDA graph and replayed for every chunk.
//
// Mixed precision: the Krylov basis and the products are FP32 (FP64 dots and
// tridiagonal); the Ritz vector is formed in FP64 and refined by short FP64
// Lanczos restarts from it until its FP64 residual meets `tol` or the FP64
// Rayleigh quotient stops moving.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>

#include "factor_kernel.cuh"
#include "lanczos.cuh"
#include "tile_queue.cuh"

namespace qsd {

// Row blocks of the dot passes: about 1024 rows per block (four rows per
// thread per vector) for large subspaces, at most four blocks per SM; small
// subspaces keep at least min(D / 256, 2 per SM) blocks (measured on GB300:
// XXZ 300,000 rows 304 blocks, Ising 1 M rows 608, TFIM 4096 rows 16; 256-row
// blocks, up to eight per SM, made the XXZ pass slower, 31.9 against 27.2 us).
int dot_blocks(int64_t D, int num_sms) {
    const int64_t by_rows = (D + 1023) / 1024;
    const int64_t floor_blocks = std::min<int64_t>((D + 255) / 256, 2 * (int64_t)num_sms);
    return (int)std::max<int64_t>(1, std::min<int64_t>(4 * (int64_t)num_sms, std::max(by_rows, floor_blocks)));
}

namespace {

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

__global__ void k_start(int64_t D, uint64_t seed, const double *v0, double *w, int *jdev) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        jdev[0] = 0;  // the step
        jdev[2] = 0;  // the block count of k_sub1
    }
    if (i >= D) return;
    w[i] = v0 ? v0[i] : uniform_pm1(seed, (uint64_t)i);
}

// Kernel bodies take their block index `vb` and block count `vg` as
// arguments, so that a packed launch (below) can run the same arithmetic for
// several jobs in one grid.
//
// One step j (j = the step counter): u = H q_j (the product); alpha0 =
// q_j.u; the three-term recurrence w = u - alpha0 q_j - beta_j q_{j-1};
// then one classical Gram-Schmidt pass of w against q_0..q_j, c = Q^T w,
// w -= Q c; alpha_j = alpha0 + c_j, beta_{j+1} = |w|, q_{j+1} = w /
// beta_{j+1}.  This is complete reorthogonalisation in the form of Golub and
// Van Loan (Matrix Computations, the Lanczos chapter): the recurrence is
// the first pass for the two vectors whose large coefficients cancel, the
// full pass is their second, and w's coefficients on the older vectors are
// of the order of the rounding error already, so one pass leaves them at
// working precision.  2 D (j + 2) FP64 FMAs per step, half those of
// classical Gram-Schmidt applied twice to u: the GB300's FP64 pipe (2 FMAs
// per SM and cycle) bounds these passes.

// Rows [r0, r1) of row block vb of B.
__device__ __forceinline__ void row_chunk(int64_t D, int vb, int B, int64_t &r0, int64_t &r1) {
    const int64_t chunk = (D + B - 1) / B;
    r0 = (int64_t)vb * chunk;
    r1 = min(D, r0 + chunk);
}

// partial[vb] = sum over the block's rows of q[r] u[r] (block sum, fixed order)
template <typename TV>
__device__ void adot_body(const TV *__restrict__ q, const TV *__restrict__ u, int64_t D, double *partial, int vb,
                          int B, double *sh) {
    int64_t r0, r1;
    row_chunk(D, vb, B, r0, r1);
    const int64_t st = blockDim.x;
    double s0 = 0.0, s1 = 0.0;
    int64_t r = r0 + threadIdx.x;
    for (; r + st < r1; r += 2 * st) {
        s0 = fma((double)q[r], (double)u[r], s0);
        s1 = fma((double)q[r + st], (double)u[r + st], s1);
    }
    if (r < r1) s0 = fma((double)q[r], (double)u[r], s0);
    const double t = block_sum(s0 + s1, sh);
    if (threadIdx.x == 0) partial[vb] = t;
}

template <typename TV>
__global__ void k_adot(const TV *__restrict__ q, const TV *__restrict__ u, int64_t D, double *partial) {
    __shared__ double sh[32];
    adot_body<TV>(q, u, D, partial, blockIdx.x, gridDim.x, sh);
}

// partial[i * B + vb] = sum over the block's rows of V[i][r] w[r].
// Warp w of the block takes the vectors i = w, w + 8, ...: its lanes stride
// the block's rows (coalesced; the block's slice of w stays in L1), four rows
// per lane per round, and one warp reduction per vector -- no block barrier.
// The vectors go two at a time, then one (each round loads w once for both:
// 12 loads in flight per lane, no predicated loads); per vector the sum runs
// in the same fixed order whatever the grouping, so the result is
// deterministic.  w has no __restrict__: the same block wrote it (plain
// loads, coherent within the block after its barrier).
template <int G, typename TV>
__device__ __forceinline__ void dot_group(const TV *__restrict__ V, int64_t D, int i0, int nw, const double *w,
                                          int64_t r0, int64_t r1, double *partial, int vb, int B) {
    const int lane = threadIdx.x & 31;
    const TV *__restrict__ vi[G];
    double s0[G], s1[G], s2[G], s3[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        vi[g] = V + (size_t)(i0 + g * nw) * D;
        s0[g] = s1[g] = s2[g] = s3[g] = 0.0;
    }
    int64_t r = r0 + lane;
    for (; r + 96 < r1; r += 128) {
        const double u0 = w[r], u1 = w[r + 32], u2 = w[r + 64], u3 = w[r + 96];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            s0[g] = fma((double)vi[g][r], u0, s0[g]);
            s1[g] = fma((double)vi[g][r + 32], u1, s1[g]);
            s2[g] = fma((double)vi[g][r + 64], u2, s2[g]);
            s3[g] = fma((double)vi[g][r + 96], u3, s3[g]);
        }
    }
    for (; r < r1; r += 32) {
        const double u0 = w[r];
#pragma unroll
        for (int g = 0; g < G; ++g) s0[g] = fma((double)vi[g][r], u0, s0[g]);
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const double t = warp_sum((s0[g] + s1[g]) + (s2[g] + s3[g]));
        if (lane == 0) partial[(size_t)(i0 + g * nw) * B + vb] = t;
    }
}

// Row block vb of the step's dot pass.  Every block sums the B partials of
// q_j.u in fixed order into alpha0 (block 0 keeps it in sc[0]), writes its
// rows of w = u - alpha0 q_j - beta_j q_{j-1}, and after a barrier takes
// partial[i * B + vb] for i <= j.  a0s: a shared double of the caller.
template <typename TV>
__device__ void dot1_body(const TV *__restrict__ V, int64_t D, int j, const TV *__restrict__ u,
                          const double *__restrict__ pa, double bj, double *w, double *partial, double *sc, int vb,
                          int B, double *sh, double &a0s) {
    double t = 0.0;
    for (int b = threadIdx.x; b < B; b += blockDim.x) t += pa[b];
    t = block_sum(t, sh);
    if (threadIdx.x == 0) {
        a0s = t;
        if (vb == 0) sc[0] = t;
    }
    __syncthreads();
    const double a0 = a0s;
    int64_t r0, r1;
    row_chunk(D, vb, B, r0, r1);
    const TV *__restrict__ qj = V + (size_t)j * D;
    if (j > 0) {
        const TV *__restrict__ qp = V + (size_t)(j - 1) * D;
        for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x)
            w[r] = fma(-bj, (double)qp[r], fma(-a0, (double)qj[r], (double)u[r]));
    } else {
        for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) w[r] = fma(-a0, (double)qj[r], (double)u[r]);
    }
    __syncthreads();  // the block's rows of w, visible to all its threads
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5, nvec = j + 1;
    int i = warp;
    for (; i + nw < nvec; i += 2 * nw) dot_group<2, TV>(V, D, i, nw, w, r0, r1, partial, vb, B);
    if (i < nvec) dot_group<1, TV>(V, D, i, nw, w, r0, r1, partial, vb, B);
}

template <typename TV>
__global__ void k_dot1(const TV *__restrict__ V, int64_t D, const int *__restrict__ jdev, const TV *__restrict__ u,
                       const double *__restrict__ pa, const double *__restrict__ beta, double *w, double *partial,
                       double *sc) {
    __shared__ double sh[32];
    __shared__ double a0s;
    const int j = *jdev;
    dot1_body<TV>(V, D, j, u, pa, j > 0 ? beta[j] : 0.0, w, partial, sc, blockIdx.x, gridDim.x, sh, a0s);
}

// h[i] = sum_b partial[i][b] in fixed order (block i; blocks past j exit)
__device__ void reduce_body(const double *__restrict__ partial, int B, double *h, int i, double *sh) {
    double s = 0.0;
    for (int b = threadIdx.x; b < B; b += blockDim.x) s += partial[(size_t)i * B + b];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) h[i] = s;
}

__global__ void k_reduce(const double *__restrict__ partial, const int *__restrict__ jdev, int B, double *h) {
    __shared__ double sh[32];
    if ((int)blockIdx.x > *jdev) return;
    reduce_body(partial, B, h, blockIdx.x, sh);
}

// Row r of the subtraction pass: w[r] -= sum_{i<=j} V[i][r] c_i (c in
// shared memory); returns w[r]^2 (0 past the end).
template <typename TV>
__device__ __forceinline__ double sub_row(const TV *__restrict__ V, int64_t D, int nvec, const double *hs, double *w,
                                          int64_t r) {
    if (r >= D) return 0.0;
    double acc = w[r];
    for (int i = 0; i < nvec; ++i) acc = fma(-(double)V[(size_t)i * D + r], hs[i], acc);
    w[r] = acc;
    return acc * acc;
}

__device__ void sq_partial_body(const double *__restrict__ w, int64_t D, double *partial, int vb, int vg,
                                double *sh) {
    double s = 0.0;
    for (int64_t r = (int64_t)vb * blockDim.x + threadIdx.x; r < D; r += (int64_t)vg * blockDim.x)
        s = fma(w[r], w[r], s);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) partial[vb] = s;
}

__global__ void k_sq_partial(const double *__restrict__ w, int64_t D, double *partial) {
    __shared__ double sh[32];
    sq_partial_body(w, D, partial, blockIdx.x, gridDim.x, sh);
}

// out[jdev ? *jdev + 1 : 0] = sqrt(sum partial)
__device__ void sqrt_sum_body(const double *__restrict__ partial, int B, double *out, double *sh) {
    double s = 0.0;
    for (int b = threadIdx.x; b < B; b += blockDim.x) s += partial[b];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) *out = sqrt(s);
}

__global__ void k_sqrt_sum(const double *__restrict__ partial, int B, double *out, const int *__restrict__ jdev) {
    __shared__ double sh[32];
    sqrt_sum_body(partial, B, out + (jdev ? *jdev + 1 : 0), sh);
}

// v = w / nrm[jdev ? *jdev + 1 : 0] into V[j+1] (when j + 1 <= m) and vcur
template <typename TV>
__device__ void next_body(const double *__restrict__ w, double s, int j1, int64_t D, int m, TV *V, TV *vcur,
                          int vb) {
    const int64_t r = (int64_t)vb * blockDim.x + threadIdx.x;
    if (r >= D) return;
    const TV v = (TV)(s > 0.0 ? w[r] / s : 0.0);
    if (V && j1 <= m) V[(size_t)j1 * D + r] = v;
    if (vcur) vcur[r] = v;
}

template <typename TV>
__global__ void k_next(const double *__restrict__ w, const double *__restrict__ nrm, const int *__restrict__ jdev,
                       int64_t D, int m, TV *V, TV *vcur) {
    const int j1 = jdev ? *jdev + 1 : 0;
    next_body<TV>(w, nrm[j1], j1, D, m, V, vcur, blockIdx.x);
}


// ---- subtraction pass and normalisation (single-job path)
// The subtraction pass also sums w^2 per 256-row block; the last of its
// blocks to finish (an atomic count, no waiting) sums those partials in block
// order into beta_{j+1} = |w| and advances the step counter (every block has
// read it by then), and k_norm_next writes q_{j+1} = w beta_{j+1}^-1: 6
// launches per step (product, q_j.u, dot pass, its sums, subtraction,
// normalisation).  Block 0 also writes alpha_j = alpha0 + c_j.
template <typename TV>
__global__ void k_sub1(const TV *__restrict__ V, int64_t D, int *jdev, const double *__restrict__ h, double *w,
                       double *part, unsigned *count, double *alpha, double *beta, const double *__restrict__ sc) {
    extern __shared__ double hs[];
    __shared__ double sh[32];
    __shared__ bool last;
    const int j = *jdev, nvec = j + 1;
    for (int i = threadIdx.x; i < nvec; i += blockDim.x) hs[i] = h[i];
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) alpha[j] = sc[0] + hs[j];
    double sq = sub_row<TV>(V, D, nvec, hs, w, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    sq = block_sum(sq, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = sq;
        __threadfence();
        last = atomicAdd(count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double t = 0.0;
#pragma unroll 8
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t += __ldcg(part + b);
    t = block_sum(t, sh);
    if (threadIdx.x == 0) {
        beta[nvec] = sqrt(t);
        *count = 0u;
        *jdev = nvec;
    }
}

// q_{j1} = w / beta_{j1} into V[j1] (when j1 <= m) and vcur, j1 = the
// advanced step counter
template <typename TV>
__global__ void k_norm_next(const double *__restrict__ w, const int *__restrict__ jdev, int64_t D, int m, TV *V,
                            TV *vcur, const double *__restrict__ beta) {
    const int j1 = *jdev;
    const double nrm = beta[j1];
    const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < D; r += (int64_t)gridDim.x * blockDim.x) {
        const TV v = (TV)(w[r] * inv);
        if (j1 <= m) V[(size_t)j1 * D + r] = v;
        vcur[r] = v;
    }
}

__global__ void k_scale(double *u, const double *__restrict__ nrm, int64_t D) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= D) return;
    const double s = *nrm;
    u[r] = s > 0.0 ? u[r] / s : 0.0;
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

// r = hu - (sc[0] / sc[1]) u
__global__ void k_residual(const double *__restrict__ hu, const double *__restrict__ u, const double *__restrict__ sc,
                           int64_t D, double *r) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= D) return;
    r[i] = hu[i] - (sc[0] / sc[1]) * u[i];
}

// ------------------------------------------------------------- tridiagonal
// Number of eigenvalues of T (diagonal a[0..m), off-diagonal b[1..m)) below
// x: the sign changes of the Sturm sequence p_0 = 1, p_k = det(T_k - x I) =
// (a_k - x) p_{k-1} - b_k^2 p_{k-2} (a zero takes the sign opposite to its
// predecessor).  No division: the GB300's FP64 pipe runs at 1/64 of the FP32
// rate and a division costs several of its operations; the pair (p_{k-1},
// p_k) is rescaled by 2^-600 whenever it grows past 2^600, and by 2^600 when
// both fall below 2^-600 (exact scalings that keep every sign).
__device__ int sturm(const double *a, const double *bb, int m, double x) {
    // bb[i] = b_i^2.  Signs, zeros and the rescaling tests read the IEEE
    // encodings with integer operations: per step the FP64 pipe (1/64 of the
    // FP32 rate, shared by the 64 points on one SM) sees one add, one
    // multiply and one FMA.  Thresholds 2^601 and 2^-600 (exponent fields
    // 1624 and 423): scaling by a power of two is exact and keeps every sign.
    auto expo = [](double v) { return ((uint32_t)__double2hiint(v) >> 20) & 0x7ffu; };
    int c = 0;
    double p0 = 1.0, p1 = a[0] - x;
    long long bits = __double_as_longlong(p1);
    bool neg = bits < 0 || (bits << 1) == 0;  // p_1 of sign opposite to p_0 = 1 (zero included)
    c += neg;
    for (int i = 1; i < m; ++i) {
        double p2 = fma(a[i] - x, p1, -bb[i] * p0);
        const uint32_t e1 = expo(p1), e2 = expo(p2);
        if (e2 >= 1624u || e1 >= 1624u) {
            p2 *= 0x1p-600;
            p1 *= 0x1p-600;
        } else if (e2 < 423u && e1 < 423u) {
            p2 *= 0x1p600;
            p1 *= 0x1p600;
        }
        const bool prev_neg = neg;
        bits = __double_as_longlong(p2);
        neg = (bits << 1) == 0 ? !prev_neg : bits < 0;
        c += (neg != prev_neg);
        p0 = p1;
        p1 = p2;
    }
    return c;
}

// One CTA, m = *jdev steps.  out[0] = theta (lowest eigenvalue), out[1] =
// |beta_m s_{m-1}| (residual estimate), out[2] = beta_m, out[3] = m,
// out[4..4+m) = unit eigenvector s.
__device__ void tridiag_body(const double *__restrict__ alpha, const double *__restrict__ beta, int m, double *out,
                             double *sm);

__global__ void k_tridiag(const double *__restrict__ alpha, const double *__restrict__ beta,
                          const int *__restrict__ jdev, double *out) {
    extern __shared__ double sm[];
    tridiag_body(alpha, beta, *jdev, out, sm);
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// The serial parts run on lane 0 of warp 0; the loops without a chain
// (bounds, scale, pivot reciprocals, normalisation) are spread over warp 0's
// lanes: on the GB300 a lone FP64 instruction costs about as much of the FP64
// pipe as a full warp's.
__device__ void tridiag_body(const double *__restrict__ alpha, const double *__restrict__ beta, int m, double *out,
                             double *sm) {
    if (m <= 0) return;
    double *a = sm, *b = sm + m, *s = sm + 2 * m;
    __shared__ double lo_hi[2];
    const int lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        a[i] = alpha[i];
        b[i] = i ? beta[i] : 0.0;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        // Gershgorin bounds (min and max are exact in any order)
        double lo = a[0], hi = a[0];
        for (int i = lane; i < m; i += 32) {
            const double rad = (i ? fabs(b[i]) : 0.0) + (i + 1 < m ? fabs(b[i + 1]) : 0.0);
            lo = fmin(lo, a[i] - rad);
            hi = fmax(hi, a[i] + rad);
        }
        lo = warp_min(lo);
        hi = warp_max(hi);
        if (lane == 0) {
            const double pad = 1e-12 * fmax(fabs(lo), fabs(hi)) + 1e-300;
            lo_hi[0] = lo - pad;
            lo_hi[1] = hi + pad;
        }
    }
    // b_i^2 for the Sturm counts, in the eigenvector's space (free until then)
    for (int i = threadIdx.x; i < m; i += blockDim.x) s[i] = b[i] * b[i];
    __syncthreads();
    // multisection: the first kTriPoints threads test one interior point
    // each; the Sturm count is monotone in x, so the number of points with no
    // eigenvalue below them is the index of the subinterval that holds the
    // lowest one.  Stop at a few ulps, or when rounding stops the shrinking.
    constexpr int kTriPoints = 64;
    constexpr double kStep = 1.0 / (kTriPoints + 1);  // point q at lo + (hi - lo) (q kStep): the same
                                                       // expression for a point and for the bound it becomes
    for (int it = 0; it < 64; ++it) {
        const double lo = lo_hi[0], hi = lo_hi[1];
        bool below = false;
        if (threadIdx.x < kTriPoints) {
            const double x = lo + (hi - lo) * ((double)(threadIdx.x + 1) * kStep);
            below = sturm(a, s, m, x) < 1;
        }
        const int k = __syncthreads_count(below);
        const double nlo = k == 0 ? lo : lo + (hi - lo) * ((double)k * kStep);
        const double nhi = k == kTriPoints ? hi : lo + (hi - lo) * ((double)(k + 1) * kStep);
        __syncthreads();
        if (threadIdx.x == 0) {
            lo_hi[0] = nlo;
            lo_hi[1] = nhi;
        }
        __syncthreads();
        if (nhi - nlo <= 4e-16 * fmax(fabs(nlo), fabs(nhi)) + 1e-300 || (nlo == lo && nhi == hi)) break;
    }
    if (threadIdx.x >= 32) return;
    const double theta = 0.5 * (lo_hi[0] + lo_hi[1]);
    // Inverse iteration (T - theta I) s = rhs.  Gaussian elimination with
    // partial pivoting on the tridiagonal matrix gives an upper factor with
    // two super-diagonals (D_, U1, U2), multipliers Lm and swap flags piv.
    double scale = 0.0;
    for (int i = lane; i < m; i += 32) scale = fmax(scale, fabs(a[i]) + fabs(b[i]));
    scale = warp_max(scale);
    const double tiny = 1e-14 * fmax(scale, 1e-300);
    double *D_ = sm + 3 * m, *U1 = sm + 4 * m, *U2 = sm + 5 * m, *Lm = sm + 6 * m;
    int *piv = reinterpret_cast<int *>(sm + 7 * m);
    for (int i = lane; i < m; i += 32) {
        D_[i] = a[i] - theta;
        U1[i] = i + 1 < m ? b[i + 1] : 0.0;
        U2[i] = 0.0;
        s[i] = 1.0;
    }
    __syncwarp();
    if (lane == 0) {
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
    }
    __syncwarp();
    // the pivots' reciprocals, once: the iterations below multiply
    for (int i = lane; i < m; i += 32) D_[i] = 1.0 / D_[i];
    __syncwarp();
    // up to three iterations; the solve's residual is |rhs| / |x| exactly,
    // so once |x| >= |rhs| / (1e-15 scale) the normalised s is an
    // eigenvector to working precision (one iteration when theta is within
    // a few ulps of the eigenvalue and the start has a fair component on it)
    double rhs2 = (double)m;  // |rhs|^2 of the first iteration (all ones)
    for (int iter = 0; iter < 3; ++iter) {
        if (lane == 0) {
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
                s[i] = v * D_[i];
            }
        }
        __syncwarp();
        double nrm = 0.0;
        for (int i = lane; i < m; i += 32) nrm = fma(s[i], s[i], nrm);
        nrm = warp_sum(nrm);  // the same value in every lane
        const double inv = 1.0 / sqrt(nrm);
        for (int i = lane; i < m; i += 32) s[i] *= inv;
        __syncwarp();
        const double q = 1e-15 * scale;
        if (nrm * (q * q) >= rhs2) break;
        rhs2 = 1.0;
    }
    if (lane == 0) {
        out[0] = theta;
        out[1] = fabs(beta[m] * s[m - 1]);
        out[2] = beta[m];
        out[3] = (double)m;
    }
    for (int i = lane; i < m; i += 32) out[4 + i] = s[i];
}

// u[r] = sum_{i < m} V[i][r] s[i], m = *jdev
template <typename TV>
__global__ void k_ritz(const TV *__restrict__ V, int64_t D, const int *__restrict__ jdev, const double *__restrict__ s,
                       double *u) {
    extern __shared__ double ss[];
    const int nvec = *jdev;
    for (int i = threadIdx.x; i < nvec; i += blockDim.x) ss[i] = s[i];
    __syncthreads();
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= D) return;
    double acc = 0.0;
    for (int i = 0; i < nvec; ++i) acc = fma((double)V[(size_t)i * D + r], ss[i], acc);
    u[r] = acc;
}

size_t tri_smem(int m) { return (size_t)8 * m * 8 + 64; }

// ---------------------------------------------------------------- packed
// One launch per kernel of the Lanczos step serves every job of a pack.  The
// grids are fixed (a multiple of the SM count): each block walks the virtual
// blocks of all jobs -- job i owns virtual blocks [first[i], first[i+1]) of
// each kernel family -- and runs the single-job body with the job's own block
// index and count, so a packed job's dots, norms and basis vectors are
// bitwise those it computes alone.  A job takes part in the steps of a chunk
// until its step counter reaches `jstop`.  The job count, the first arrays
// and the descriptors live in the pack's device block, so the launches (and
// a CUDA graph of them) do not change with the membership.
struct PackJob {
    const void *V;
    void *vcur, *hv;
    double *w, *h, *part, *alpha, *beta, *tri;
    int *jdev;
    int64_t D;
    int m, B, nbD, nb, jstop, pad;
};

// Each block stages the launch family's first array and every job's step
// (-1 once the job has finished its part of the chunk) in shared memory, so
// that resolving a virtual block costs a few shared-memory reads instead of
// a chain of dependent global loads.
constexpr int kPackMaxJobs = 256;

struct PackStage {
    int first[kPackMaxJobs + 1];
    int j[kPackMaxJobs];
};

__device__ __forceinline__ int stage_pack(const PackJob *__restrict__ jobs, const int *__restrict__ first,
                                          const int *__restrict__ np, PackStage &st) {
    const int n = *np;
    for (int k = threadIdx.x; k <= n; k += blockDim.x) st.first[k] = first[k];
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int j = *jobs[k].jdev;
        st.j[k] = j < jobs[k].jstop ? j : -1;
    }
    __syncthreads();
    return n;
}

__device__ __forceinline__ int find_job(const int *first, int n, int b) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (first[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// q_j.u for every job (job i's virtual grid: its B dot-pass row blocks)
template <typename TV>
__global__ void kq_adot(const PackJob *__restrict__ jobs, const int *__restrict__ first, const int *__restrict__ np) {
    __shared__ PackStage st;
    __shared__ double sh[32];
    const int n = stage_pack(jobs, first, np, st), total = st.first[n];
    for (int b = blockIdx.x; b < total; b += gridDim.x) {
        const int i = find_job(st.first, n, b), j = st.j[i];
        if (j < 0) continue;  // block-uniform
        const PackJob &J = jobs[i];
        adot_body<TV>(static_cast<const TV *>(J.vcur), static_cast<const TV *>(J.hv), J.D,
                      J.part + (size_t)(J.m + 1) * J.B, b - st.first[i], J.B, sh);  // ends on a barrier
    }
}

// the dot pass for every job
template <typename TV>
__global__ void kq_dot1(const PackJob *__restrict__ jobs, const int *__restrict__ first, const int *__restrict__ np) {
    __shared__ PackStage st;
    __shared__ double sh[32];
    __shared__ double a0s;
    const int n = stage_pack(jobs, first, np, st), total = st.first[n];
    for (int b = blockIdx.x; b < total; b += gridDim.x) {
        const int i = find_job(st.first, n, b), j = st.j[i];
        if (j < 0) continue;
        const PackJob &J = jobs[i];
        const int m = J.m;
        dot1_body<TV>(static_cast<const TV *>(J.V), J.D, j, static_cast<const TV *>(J.hv),
                      J.part + (size_t)(m + 1) * J.B, j > 0 ? J.beta[j] : 0.0, J.w, J.part, J.h + (m + 1),
                      b - st.first[i], J.B, sh, a0s);
        __syncthreads();  // a0s and sh are rewritten next round
    }
}

__global__ void kq_reduce(const PackJob *__restrict__ jobs, const int *__restrict__ first,
                          const int *__restrict__ np) {
    __shared__ PackStage st;
    __shared__ double sh[32];
    const int n = stage_pack(jobs, first, np, st), total = st.first[n];
    for (int b = blockIdx.x; b < total; b += gridDim.x) {
        const int i = find_job(st.first, n, b), j = st.j[i], row = b - st.first[i];
        if (j < 0 || row > j) continue;
        const PackJob &J = jobs[i];
        reduce_body(J.part, J.B, J.h, row, sh);  // ends on a barrier
    }
}

// the subtraction pass for every job: w -= V c, squares of w per 256-row
// block; a job's block 0 writes its alpha_j
template <typename TV>
__global__ void kq_sub1(const PackJob *__restrict__ jobs, const int *__restrict__ first, const int *__restrict__ np) {
    extern __shared__ double hs[];
    __shared__ PackStage st;
    __shared__ double sh[32];
    const int n = stage_pack(jobs, first, np, st), total = st.first[n];
    for (int b = blockIdx.x; b < total; b += gridDim.x) {
        const int i = find_job(st.first, n, b), j = st.j[i];
        if (j < 0) continue;
        const PackJob &J = jobs[i];
        const int nvec = j + 1, vb = b - st.first[i], m = J.m;
        for (int k = threadIdx.x; k < nvec; k += blockDim.x) hs[k] = J.h[k];
        __syncthreads();
        if (vb == 0 && threadIdx.x == 0) J.alpha[j] = J.h[m + 1] + hs[j];
        double sq = sub_row<TV>(static_cast<const TV *>(J.V), J.D, nvec, hs, J.w,
                                (int64_t)vb * blockDim.x + threadIdx.x);
        sq = block_sum(sq, sh);  // ends on a barrier: hs is free again
        if (threadIdx.x == 0) J.part[(size_t)(m + 2) * J.B + vb] = sq;
    }
}

// k_norm_next for every job (job i's virtual grid: nb blocks); each block
// sums the job's squares in the order of k_sub1's last block
template <typename TV>
__global__ void kq_norm_next(const PackJob *__restrict__ jobs, const int *__restrict__ first,
                             const int *__restrict__ np) {
    __shared__ PackStage st;
    __shared__ double sh[32];
    __shared__ double nrm_s;
    const int n = stage_pack(jobs, first, np, st), total = st.first[n];
    for (int b = blockIdx.x; b < total; b += gridDim.x) {
        const int i = find_job(st.first, n, b), j = st.j[i];
        if (j < 0) continue;
        const PackJob &J = jobs[i];
        const int vb = b - st.first[i], nbD = J.nbD, nb = J.nb, m = J.m;
        const int64_t D = J.D;
        const double *__restrict__ part = J.part + (size_t)(m + 2) * J.B;
        double t = 0.0;
#pragma unroll 8
        for (int k = threadIdx.x; k < nbD; k += blockDim.x) t += part[k];
        t = block_sum(t, sh);
        if (threadIdx.x == 0) nrm_s = sqrt(t);
        __syncthreads();
        const double nrm = nrm_s;
        const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
        const int j1 = j + 1;
        if (vb == 0 && threadIdx.x == 0) J.beta[j1] = nrm;
        TV *V = static_cast<TV *>(const_cast<void *>(J.V));
        TV *vc = static_cast<TV *>(J.vcur);
        const double *__restrict__ w = J.w;
        for (int64_t r = (int64_t)vb * blockDim.x + threadIdx.x; r < D; r += (int64_t)nb * blockDim.x) {
            const TV v = (TV)(w[r] * inv);
            if (j1 <= m) V[(size_t)j1 * D + r] = v;
            vc[r] = v;
        }
        __syncthreads();  // nrm_s is rewritten next round
    }
}

__global__ void kq_incr(const PackJob *__restrict__ jobs, const int *__restrict__ np) {
    const int n = *np;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (*jobs[i].jdev < jobs[i].jstop) *jobs[i].jdev += 1;
}

// block i < n: the tridiagonal problem of job i, then its four results to out[4 i]
__global__ void kq_tridiag(const PackJob *__restrict__ jobs, const int *__restrict__ np, double *out) {
    extern __shared__ double sm[];
    if ((int)blockIdx.x >= *np) return;
    const PackJob &J = jobs[blockIdx.x];
    tridiag_body(J.alpha, J.beta, *J.jdev, J.tri, sm);
    __syncthreads();
    if (threadIdx.x < 4) out[4 * (size_t)blockIdx.x + threadIdx.x] = J.tri[threadIdx.x];
}

}  // namespace

bool packable(qsd_ctx ctx, qsd_op op, qsd_sub sub) {
    const int c = pack_class(ctx, op, sub, true);
    return c >= kPackFacClass || (c >= 0 && op->G <= kPackMaxScanGroups);
}

namespace {

// Fixed layout of a pack's device block (and of its pinned staging) for
// `cap` members: header (member count), descriptors, the first virtual block
// of each job per kernel family (B dot blocks, m + 1 reduction blocks,
// 256-row blocks, normalisation blocks), one tile queue and the first tiles
// per product class, the product parameters per class, the results.
struct PackLayout {
    size_t o_jobs, o_first, o_q, o_t0, o_par[kPackClasses], o_out, bytes;
    explicit PackLayout(int cap) {
        o_jobs = 256;
        o_first = align_up(o_jobs + (size_t)cap * sizeof(PackJob), 256);
        o_q = align_up(o_first + (size_t)4 * (cap + 1) * sizeof(int), 256);
        o_t0 = align_up(o_q + (size_t)kPackClasses * sizeof(TileQueue), 256);
        size_t o = align_up(o_t0 + (size_t)kPackClasses * cap * 8, 256);
        for (int c = 0; c < kPackClasses; ++c) {
            o_par[c] = o;
            o = align_up(o + (size_t)cap * rec(c), 256);
        }
        o_out = o;
        bytes = align_up(o_out + (size_t)cap * 4 * sizeof(double), 256);
    }
    static size_t rec(int c) { return c >= kPackFacClass ? sizeof(FacPair) : sizeof(ApplyParams); }
};

constexpr int kPackGridPerSm = 4;  // blocks of the packed Lanczos kernels per SM

// The launches of one chunk of `steps` steps for the product classes in
// `mask` (captured into a graph by Pack::enqueue_chunk).
template <typename TV>
void enqueue_pack_steps(qsd_ctx ctx, unsigned char *d, const PackLayout &L, int cap, int prec, unsigned mask,
                        int steps, double *host_out, cudaStream_t s) {
    const PackJob *dj = reinterpret_cast<const PackJob *>(d + L.o_jobs);
    const int *np = reinterpret_cast<const int *>(d);
    const int *fB = reinterpret_cast<const int *>(d + L.o_first), *fM = fB + (cap + 1), *fD = fB + 2 * (cap + 1),
              *fN = fB + 3 * (cap + 1);
    TileQueue *q = reinterpret_cast<TileQueue *>(d + L.o_q);
    const int64_t *t0 = reinterpret_cast<const int64_t *>(d + L.o_t0);
    const int G = kPackGridPerSm * ctx->num_sms;
    const size_t hsm = (size_t)(kLanczosMaxSteps + 1) * 8;
    constexpr int64_t kAnyTiles = (int64_t)1 << 40;  // the resident grid: the tile count is in the queue
    for (int t = 0; t < steps; ++t) {
        for (int c = 0; c < kPackClasses; ++c) {
            if (!(mask >> c & 1u)) continue;
            const int64_t *tc = t0 + (size_t)c * cap;
            if (c >= kPackFacClass) {
                const FacPair *par = reinterpret_cast<const FacPair *>(d + L.o_par[c]);
                const int W = pack_class_width(c);
                if (prec == QSD_FP64) launch_apply_fac_queue<QSD_FP64>(par, tc, q + c, kAnyTiles, W, 1, ctx->num_sms, s);
                else if (prec == QSD_FP32_MIXED)
                    launch_apply_fac_queue<QSD_FP32_MIXED>(par, tc, q + c, kAnyTiles, W, 1, ctx->num_sms, s);
                else launch_apply_fac_queue<QSD_FP32_DOT2>(par, tc, q + c, kAnyTiles, W, 1, ctx->num_sms, s);
            } else {
                launch_apply_queue(reinterpret_cast<const ApplyParams *>(d + L.o_par[c]), tc, q + c, kAnyTiles,
                                   pack_class_width(c), pack_class_lanes(c), 1, prec, ctx->num_sms, s);
            }
        }
        kq_adot<TV><<<G, kLanczosThreads, 0, s>>>(dj, fB, np);
        kq_dot1<TV><<<G, kLanczosThreads, 0, s>>>(dj, fB, np);
        kq_reduce<<<2 * G, 128, 0, s>>>(dj, fM, np);
        kq_sub1<TV><<<G, 256, hsm, s>>>(dj, fD, np);
        kq_norm_next<TV><<<G, 256, 0, s>>>(dj, fN, np);
        kq_incr<<<1, 256, 0, s>>>(dj, np);
    }
    double *dout = reinterpret_cast<double *>(d + L.o_out);
    kq_tridiag<<<cap, kLanczosThreads, tri_smem(kLanczosMaxSteps), s>>>(dj, np, dout);
    QSD_LAUNCH_CHECK();
    QSD_CUDA(cudaMemcpyAsync(host_out, dout, (size_t)cap * 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
}

}  // namespace

void Pack::init(qsd_ctx c, int capacity, cudaStream_t st) {
    if (capacity > kPackMaxJobs) fail(QSD_ERR_INVALID_ARG, "pack: more members than the packed kernels stage");
    ctx = c;
    cap = std::max(capacity, 1);
    s = st;
    const PackLayout L(cap);
    bytes = L.bytes;
    dev.alloc_async(bytes, s);
    QSD_CUDA(cudaMallocHost(reinterpret_cast<void **>(&host), bytes));
    std::memset(host, 0, bytes);
}

void Pack::release() {
    if (s) cudaStreamSynchronize(s);
    for (auto &kv : graphs) cudaGraphExecDestroy(kv.second);
    graphs.clear();
    dev.release();
    if (host) cudaFreeHost(host);
    host = nullptr;
    if (s) cudaStreamSynchronize(s);
    members.clear();
    s = nullptr;
}

Pack::~Pack() { release(); }

void Pack::enqueue_chunk(const std::vector<LanczosJob *> &jobs) {
    const int n = (int)jobs.size();
    if (n == 0) return;
    if (n > cap) fail(QSD_ERR_INTERNAL, "packed chunk: more jobs than the pack holds");
    const PackLayout L(cap);
    const bool fp32 = jobs[0]->fp32;
    const int prec = jobs[0]->prec;
    int steps = 0;
    std::vector<PackJob> pj(n);
    std::vector<int> first(4 * (cap + 1), 0);
    int *fB = first.data(), *fM = fB + (cap + 1), *fD = fB + 2 * (cap + 1), *fN = fB + 3 * (cap + 1);
    std::vector<std::vector<int>> by_class(kPackClasses);
    for (int i = 0; i < n; ++i) {
        LanczosJob &J = *jobs[i];
        if (J.fp32 != fp32 || J.prec != prec) fail(QSD_ERR_INTERNAL, "packed chunk: mixed precisions");
        if (J.m > kLanczosMaxSteps) fail(QSD_ERR_INTERNAL, "packed chunk: basis larger than the packed kernels hold");
        const int cls = pack_class(ctx, J.op, J.sub, true);
        if (cls < 0) fail(QSD_ERR_INTERNAL, "packed chunk: product cannot be packed");
        const int len = std::max(std::min(J.check_every, J.m - J.steps_done), 0);
        steps = std::max(steps, len);
        PackJob &P = pj[i];
        P.V = J.V.p;
        P.vcur = J.vcur.p;
        P.hv = J.hv.p;
        P.w = J.w.as<double>();
        P.h = J.h.as<double>();
        P.part = J.part.as<double>();
        P.alpha = J.alpha.as<double>();
        P.beta = J.beta.as<double>();
        P.tri = J.tri.as<double>();
        P.jdev = J.jdev.as<int>();
        P.D = J.D;
        P.m = J.m;
        P.B = J.B;
        P.nbD = J.nbD;
        P.nb = std::min<int>(J.nbD, 4 * ctx->num_sms);  // the single job's normalisation grid
        P.jstop = J.steps_done + len;
        P.pad = 0;
        fB[i + 1] = fB[i] + J.B;
        fM[i + 1] = fM[i] + J.m + 1;
        fD[i + 1] = fD[i] + J.nbD;
        fN[i + 1] = fN[i] + P.nb;
        by_class[cls].push_back(i);
    }
    if (steps <= 0) return;
    // staging: header, descriptors, first arrays, queues, first tiles (one
    // copy), then each present class's parameters where they changed
    unsigned char *h = host, *d = static_cast<unsigned char *>(dev.p);
    std::memset(h, 0, L.o_par[0]);
    *reinterpret_cast<int *>(h) = n;
    std::memcpy(h + L.o_jobs, pj.data(), (size_t)n * sizeof(PackJob));
    std::memcpy(h + L.o_first, first.data(), first.size() * sizeof(int));
    TileQueue *hq = reinterpret_cast<TileQueue *>(h + L.o_q);
    int64_t *ht0 = reinterpret_cast<int64_t *>(h + L.o_t0);
    unsigned mask = 0;
    std::vector<unsigned char> rec;
    std::vector<std::pair<size_t, size_t>> dirty;
    for (int c = 0; c < kPackClasses; ++c) {
        const std::vector<int> &idx = by_class[c];
        if (idx.empty()) continue;
        mask |= 1u << c;
        const int rows = pack_class_rows(c);
        const size_t rb = PackLayout::rec(c);
        rec.assign(idx.size() * rb, 0);
        int64_t tiles = 0;
        for (size_t k = 0; k < idx.size(); ++k) {
            LanczosJob &J = *jobs[idx[k]];
            ht0[(size_t)c * cap + k] = tiles;
            tiles += (J.D + rows - 1) / rows;
            if (c >= kPackFacClass) {
                const FacPair fp = factored_params(ctx, J.op, J.sub, J.diag, 1, J.vcur.p, J.hv.p);
                std::memcpy(rec.data() + k * rb, &fp, rb);
            } else {
                const ApplyParams ap = product_params(ctx, J.op, J.sub, J.diag, 1, J.vcur.p, J.hv.p);
                std::memcpy(rec.data() + k * rb, &ap, rb);
            }
        }
        hq[c].n = (int32_t)idx.size();
        hq[c].tiles = tiles;  // claim counters zero
        if (std::memcmp(h + L.o_par[c], rec.data(), rec.size()) != 0) {
            std::memcpy(h + L.o_par[c], rec.data(), rec.size());
            dirty.emplace_back(L.o_par[c], rec.size());
        }
    }
    QSD_CUDA(cudaMemcpyAsync(d, h, L.o_par[0], cudaMemcpyHostToDevice, s));
    for (auto &[o, len] : dirty) QSD_CUDA(cudaMemcpyAsync(d + o, h + o, len, cudaMemcpyHostToDevice, s));
    // the chunk: a graph per (classes present, steps), captured on first use
    static_assert(kPackClasses <= 16, "class mask in the low 16 bits of the graph key");
    const uint32_t key = mask | ((uint32_t)steps << 16);
    auto it = graphs.find(key);
    if (it == graphs.end()) {
        if (graphs.size() >= 64) {
            for (auto &kv : graphs) cudaGraphExecDestroy(kv.second);
            graphs.clear();
        }
        double *hout = reinterpret_cast<double *>(h + L.o_out);
        cudaGraph_t g = nullptr;
        QSD_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        try {
            if (fp32) enqueue_pack_steps<float>(ctx, d, L, cap, prec, mask, steps, hout, s);
            else enqueue_pack_steps<double>(ctx, d, L, cap, prec, mask, steps, hout, s);
        } catch (...) {
            cudaStreamEndCapture(s, &g);
            if (g) cudaGraphDestroy(g);
            throw;
        }
        QSD_CUDA(cudaStreamEndCapture(s, &g));
        cudaGraphExec_t ge = nullptr;
        const cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        QSD_CUDA(e);
        it = graphs.emplace(key, ge).first;
        ++graph_builds;
    }
    QSD_CUDA(cudaGraphLaunch(it->second, s));
    for (int i = 0; i < n; ++i) {
        jobs[i]->steps_done = pj[i].jstop;
        ++jobs[i]->chunks;
    }
    members = jobs;
    ++chunks;
}

void Pack::finish_chunk() {
    const PackLayout L(cap);
    const double *out = reinterpret_cast<const double *>(host + L.o_out);
    for (size_t i = 0; i < members.size(); ++i) std::memcpy(members[i]->hpin, out + 4 * i, 4 * sizeof(double));
    members.clear();
}

// ---------------------------------------------------------------- job
LanczosJob::~LanczosJob() {
    if (graph) cudaGraphExecDestroy(graph);
    if (hpin && own_pin) cudaFreeHost(hpin);
}

void LanczosJob::init(qsd_ctx c, qsd_op o, qsd_sub su, const double *d, int product_precision, int steps,
                      int check, cudaStream_t st, bool stream_ordered) {
    ctx = c;
    op = o;
    sub = su;
    diag = d;
    prec = product_precision;
    fp32 = product_precision != QSD_FP64;
    D = su->D;
    m = (int)std::min<int64_t>(std::min(steps, kLanczosMaxSteps), D);
    check_every = std::max(1, std::min(check, m));
    s = st;
    B = dot_blocks(D, ctx->num_sms);
    nbD = blocks_for(D, 256);
    // whatever the product builds on first use, before any chunk is captured
    prepare_product(ctx, op, sub, st);
    const size_t sv = fp32 ? 4 : 8;
    auto A = [&](DevBuf &b, size_t n) {
        if (pool) b.alloc_pool(n, pool, s);
        else if (stream_ordered) b.alloc_async(n, s);
        else b.alloc(n);
    };
    A(V, (size_t)(m + 1) * D * sv);
    A(vcur, (size_t)D * sv);
    A(hv, (size_t)D * sv);
    A(w, (size_t)D * 8);
    A(h, ((size_t)m + 9) * 8);
    A(part, ((size_t)(m + 2) * B + nbD) * 8);
    A(alpha, (size_t)(m + 2) * 8);
    A(beta, (size_t)(m + 3) * 8);
    A(tri, (size_t)(m + 8) * 8);
    A(jdev, 16);
    if (!hpin) QSD_CUDA(cudaMallocHost(&hpin, 8 * sizeof(double)));
}

size_t LanczosJob::footprint(int64_t D, int steps, bool fp32, int num_sms) {
    const int m = (int)std::min<int64_t>(std::min(steps, kLanczosMaxSteps), D);
    const int B = dot_blocks(D, num_sms);
    const size_t sv = fp32 ? 4 : 8;
    return (size_t)(m + 3) * D * sv + (size_t)D * 8 + ((size_t)(m + 2) * B + (D + 255) / 256) * 8 +
           (size_t)(m + 16) * 40;
}

template <typename TV>
static void enqueue_start_t(LanczosJob &J, const double *start, uint64_t seed) {
    cudaStream_t s = J.s;
    QSD_CUDA(cudaMemsetAsync(J.alpha.p, 0, J.alpha.bytes, s));
    QSD_CUDA(cudaMemsetAsync(J.beta.p, 0, J.beta.bytes, s));
    double *w = J.w.as<double>(), *part = J.part.as<double>();
    double *nrm = J.tri.as<double>() + J.m + 7;
    k_start<<<J.nbD, 256, 0, s>>>(J.D, seed, start, w, J.jdev.as<int>());
    k_sq_partial<<<J.B, kLanczosThreads, 0, s>>>(w, J.D, part);
    k_sqrt_sum<<<1, kLanczosThreads, 0, s>>>(part, J.B, nrm, nullptr);
    k_next<TV><<<J.nbD, 256, 0, s>>>(w, nrm, nullptr, J.D, J.m, J.V.as<TV>(), J.vcur.as<TV>());
    QSD_LAUNCH_CHECK();
    J.steps_done = 0;
}

void LanczosJob::enqueue_start(const double *start, uint64_t seed) {
    if (fp32) enqueue_start_t<float>(*this, start, seed);
    else enqueue_start_t<double>(*this, start, seed);
}

static int ctx_sms(qsd_ctx c) { return c->num_sms; }

template <typename TV>
static void enqueue_steps_t(LanczosJob &J, int n) {
    cudaStream_t s = J.s;
    TV *V = J.V.as<TV>(), *hv = J.hv.as<TV>(), *vc = J.vcur.as<TV>();
    double *w = J.w.as<double>(), *h = J.h.as<double>(), *part = J.part.as<double>();
    double *alpha = J.alpha.as<double>(), *beta = J.beta.as<double>();
    const int *j = J.jdev.as<int>();
    const size_t hsm = (size_t)(J.m + 1) * 8;
    // part: the dot pass's partials ((m + 1) B), those of q_j.u (B), the
    // squares of w per 256-row block (nbD); h: c_0..c_m, then alpha0
    double *pa = part + (size_t)(J.m + 1) * J.B, *psq = part + (size_t)(J.m + 2) * J.B, *sc = h + (J.m + 1);
    int *jm = J.jdev.as<int>();
    unsigned *count = reinterpret_cast<unsigned *>(jm + 2);
    const int nb = std::min<int>(J.nbD, 4 * ctx_sms(J.ctx));
    for (int t = 0; t < n; ++t) {
        apply_H(J.ctx, J.op, J.sub, J.diag, J.prec, 1, vc, hv, s);
        k_adot<TV><<<J.B, kLanczosThreads, 0, s>>>(vc, hv, J.D, pa);
        k_dot1<TV><<<J.B, kLanczosThreads, 0, s>>>(V, J.D, j, hv, pa, beta, w, part, sc);
        k_reduce<<<J.m + 1, 128, 0, s>>>(part, j, J.B, h);
        k_sub1<TV><<<J.nbD, 256, hsm, s>>>(V, J.D, jm, h, w, psq, count, alpha, beta, sc);
        k_norm_next<TV><<<nb, 256, 0, s>>>(w, j, J.D, J.m, V, vc, beta);
    }
    k_tridiag<<<1, kLanczosThreads, tri_smem(J.m), s>>>(alpha, beta, j, J.tri.as<double>());
    QSD_LAUNCH_CHECK();
    QSD_CUDA(cudaMemcpyAsync(J.hpin, J.tri.p, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
}

void LanczosJob::enqueue_chunk(bool use_graph) {
    const int n = std::min(check_every, m - steps_done);
    if (n <= 0) return;
    if (use_graph && n == check_every) {
        if (!graph) {
            cudaGraph_t g = nullptr;
            QSD_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            try {
                if (fp32) enqueue_steps_t<float>(*this, n);
                else enqueue_steps_t<double>(*this, n);
            } catch (...) {
                cudaStreamEndCapture(s, &g);
                if (g) cudaGraphDestroy(g);
                throw;
            }
            QSD_CUDA(cudaStreamEndCapture(s, &g));
            const cudaError_t e = cudaGraphInstantiate(&graph, g, 0);
            cudaGraphDestroy(g);
            QSD_CUDA(e);
        }
        QSD_CUDA(cudaGraphLaunch(graph, s));
    } else {
        if (fp32) enqueue_steps_t<float>(*this, n);
        else enqueue_steps_t<double>(*this, n);
    }
    steps_done += n;
    ++chunks;
}

void LanczosJob::read(double &theta, double &est, double &beta_last, int &nvec) const {
    theta = hpin[0];
    est = hpin[1];
    beta_last = hpin[2];
    nvec = (int)hpin[3];
}

void LanczosJob::enqueue_ritz(double *u) {
    const int *j = jdev.as<int>();
    const size_t ssm = (size_t)(m + 1) * 8;
    double *nrm = tri.as<double>() + m + 7;
    if (fp32) k_ritz<float><<<nbD, 256, ssm, s>>>(V.as<float>(), D, j, tri.as<double>() + 4, u);
    else k_ritz<double><<<nbD, 256, ssm, s>>>(V.as<double>(), D, j, tri.as<double>() + 4, u);
    k_sq_partial<<<B, kLanczosThreads, 0, s>>>(u, D, part.as<double>());
    k_sqrt_sum<<<1, kLanczosThreads, 0, s>>>(part.as<double>(), B, nrm, nullptr);
    k_scale<<<nbD, 256, 0, s>>>(u, nrm, D);
    QSD_LAUNCH_CHECK();
}

bool LanczosJob::converged(double tol) const {
    double theta, est, hb;
    int n;
    read(theta, est, hb, n);
    const double at = std::max(std::fabs(theta), 1e-300);
    return est <= tol * at || hb <= 1e-13 * at;
}

// ---------------------------------------------------------------- residual
void ResidJob::init(qsd_ctx c, int64_t Dn, cudaStream_t st, bool stream_ordered) {
    ctx = c;
    D = Dn;
    s = st;
    B = dot_blocks(D, ctx->num_sms);
    if (pool || stream_ordered) {
        hu.alloc_pool((size_t)D * 8, pool, s);
        r.alloc_pool((size_t)D * 8, pool, s);
        part.alloc_pool((size_t)2 * B * 8 + 64, pool, s);
    } else {
        hu.alloc((size_t)D * 8);
        r.alloc((size_t)D * 8);
        part.alloc((size_t)2 * B * 8 + 64);
    }
    if (!hpin) QSD_CUDA(cudaMallocHost(&hpin, 4 * sizeof(double)));
}

ResidJob::~ResidJob() {
    if (hpin && own_pin) cudaFreeHost(hpin);
}

// hpin = [u^T H u, u^T u, |H u - theta u|]
void ResidJob::enqueue(qsd_op op, qsd_sub sub, const double *diag, const double *u) {
    double *p = part.as<double>(), *sc = p + 2 * B;
    apply_H(ctx, op, sub, diag, QSD_FP64, 1, u, hu.as<double>(), s);
    k_dot_partial<<<B, kLanczosThreads, 0, s>>>(u, hu.as<double>(), D, p);
    k_sum<<<1, kLanczosThreads, 0, s>>>(p, B, sc);
    k_dot_partial<<<B, kLanczosThreads, 0, s>>>(u, u, D, p + B);
    k_sum<<<1, kLanczosThreads, 0, s>>>(p + B, B, sc + 1);
    k_residual<<<blocks_for(D, 256), 256, 0, s>>>(hu.as<double>(), u, sc, D, r.as<double>());
    k_sq_partial<<<B, kLanczosThreads, 0, s>>>(r.as<double>(), D, p);
    k_sqrt_sum<<<1, kLanczosThreads, 0, s>>>(p, B, sc + 2, nullptr);
    QSD_LAUNCH_CHECK();
    QSD_CUDA(cudaMemcpyAsync(hpin, sc, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
}

void ResidJob::read(double &theta, double &resid_rel) const {
    theta = hpin[0] / hpin[1];
    resid_rel = hpin[2] / std::sqrt(hpin[1]) / std::max(std::fabs(theta), 1e-300);
}

void rayleigh_quotient(qsd_ctx ctx, qsd_op op, qsd_sub sub, const double *diag, const double *u, double *out) {
    cudaStream_t s = ctx->stream;
    const int64_t D = sub->D;
    const int B = std::max(1, std::min<int>(2 * ctx->num_sms, (int)((D + 255) / 256)));
    double *hu = static_cast<double *>(ctx->scratch[2].get((size_t)D * 8));
    double *part = static_cast<double *>(ctx->scratch[3].get((size_t)4 * 2048 * 8));
    double *sc = part + 3 * 2048;
    apply_H(ctx, op, sub, diag, QSD_FP64, 1, u, hu, s);
    k_dot_partial<<<B, kLanczosThreads, 0, s>>>(u, hu, D, part);
    k_sum<<<1, kLanczosThreads, 0, s>>>(part, B, sc);            // u^T H u
    k_dot_partial<<<B, kLanczosThreads, 0, s>>>(u, u, D, part + 2048);
    k_sum<<<1, kLanczosThreads, 0, s>>>(part + 2048, B, sc + 1); // u^T u
    k_residual<<<blocks_for(D, 256), 256, 0, s>>>(hu, u, sc, D, hu);
    k_sq_partial<<<B, kLanczosThreads, 0, s>>>(hu, D, part);
    k_sqrt_sum<<<1, kLanczosThreads, 0, s>>>(part, B, sc + 2, nullptr);
    QSD_LAUNCH_CHECK();
    double h[3];
    QSD_CUDA(cudaMemcpyAsync(h, sc, 24, cudaMemcpyDeviceToHost, s));
    QSD_CUDA(cudaStreamSynchronize(s));
    if (!(h[1] > 0.0)) fail(QSD_ERR_INVALID_ARG, "rayleigh_quotient: u is zero");
    out[0] = h[0] / h[1];
    out[1] = h[2] / std::sqrt(h[1]);
    out[2] = h[1];
}

// ---------------------------------------------------------------- driver
int lanczos_ground_state(qsd_ctx ctx, qsd_op op, qsd_sub sub, const qsd_lanczos_params &p, double *energy,
                         double *vec_out, qsd_lanczos_info *info) {
    const auto t0 = std::chrono::steady_clock::now();
    const bool has_deadline = p.time_limit_s > 0.0;
    const auto deadline = t0 + std::chrono::microseconds((int64_t)(p.time_limit_s * 1e6));
    auto late = [&]() { return has_deadline && std::chrono::steady_clock::now() > deadline; };
    Binding *bind = get_binding(ctx, op, sub);
    const double *diag = bind->diag.as<double>();
    cudaStream_t s = ctx->stream;
    const int64_t D = sub->D;
    const bool mixed = p.precision != QSD_FP64;
    const double tol = p.tol > 0 ? p.tol : 1e-9;
    const bool graphs = p.use_graphs != 0;
    int applies = 0, total_steps = 0, restarts = 0;
    bool timeout = false;
    // workspace from the context's pool: a repeated solve maps nothing.  The
    // guard, destroyed after every buffer below, synchronises the stream once
    // their stream-ordered frees are enqueued: the pool then gives back what
    // it holds above its release threshold within this call, not at some
    // later caller's synchronisation.
    struct SyncAtExit {
        cudaStream_t s;
        ~SyncAtExit() { cudaStreamSynchronize(s); }
    } sync_at_exit{s};
    cudaMemPool_t pool = ctx->pool;
    DevBuf u;
    u.alloc_pool((size_t)D * 8, pool, s);
    ResidJob R;
    R.pool = pool;
    R.init(ctx, D, s, false);

    // main phase: FP64, or FP32 until FP32 round-off limits the estimate
    LanczosJob J;
    J.pool = pool;
    J.init(ctx, op, sub, diag, p.precision, p.max_steps, p.check_every, s, false);
    // pick the product paths now: graph capture must not time anything
    QSD_CUDA(cudaMemsetAsync(J.vcur.p, 0, J.vcur.bytes, s));
    QSD_CUDA(cudaMemsetAsync(u.p, 0, u.bytes, s));
    product_path(ctx, op, sub, diag, p.precision, 1, J.vcur.p, J.hv.p, 1, 0, s, true);
    if (p.precision != QSD_FP64) product_path(ctx, op, sub, diag, QSD_FP64, 1, u.p, R.hu.p, 1, 0, s, true);
    const double phase_tol = mixed ? std::max(tol, 1e-5) : tol;
    J.enqueue_start(p.v0, p.seed);
    while (J.steps_done < J.m) {
        J.enqueue_chunk(graphs);
        QSD_CUDA(cudaStreamSynchronize(s));
        if (J.converged(phase_tol)) break;
        if (late()) { timeout = true; break; }
    }
    double theta, est, hb;
    int nvec;
    J.read(theta, est, hb, nvec);
    total_steps += J.steps_done;
    applies += J.steps_done;
    const double e_unrefined = theta;
    const bool main_converged = J.converged(tol);
    J.enqueue_ritz(u.as<double>());
    R.enqueue(op, sub, diag, u.as<double>());
    ++applies;
    QSD_CUDA(cudaStreamSynchronize(s));
    double rq, resid;
    R.read(rq, resid);
    double result = mixed ? rq : theta;
    bool converged = resid <= tol || (!mixed && main_converged);
    if (mixed && !converged && !timeout) {
        // FP64 restarts from the current Ritz vector
        LanczosJob K;
        K.pool = pool;
        K.init(ctx, op, sub, diag, QSD_FP64, std::max(p.refine_steps, 2), p.check_every, s, false);
        double prev = rq;
        const double rtol = p.refine_tol > 0 ? p.refine_tol : 1e-10;
        DevBuf start;
        start.alloc_pool((size_t)D * 8, pool, s);
        while (!converged && restarts < std::max(p.max_refine, 0)) {
            if (late()) { timeout = true; break; }
            QSD_CUDA(cudaMemcpyAsync(start.p, u.p, (size_t)D * 8, cudaMemcpyDeviceToDevice, s));
            K.enqueue_start(start.as<double>(), p.seed);
            while (K.steps_done < K.m) {
                K.enqueue_chunk(graphs);
                QSD_CUDA(cudaStreamSynchronize(s));
                if (K.converged(tol)) break;
            }
            total_steps += K.steps_done;
            applies += K.steps_done;
            K.enqueue_ritz(u.as<double>());
            R.enqueue(op, sub, diag, u.as<double>());
            ++applies;
            QSD_CUDA(cudaStreamSynchronize(s));
            ++restarts;
            R.read(rq, resid);
            result = rq;
            const double change = std::fabs(rq - prev) / std::max(std::fabs(rq), 1e-300);
            prev = rq;
            if (resid <= tol || change <= rtol) converged = true;
        }
    }
    *energy = result;
    if (vec_out) QSD_CUDA(cudaMemcpyAsync(vec_out, u.p, (size_t)D * 8, cudaMemcpyDeviceToDevice, s));
    QSD_CUDA(cudaStreamSynchronize(s));
    if (info) {
        info->steps = total_steps;
        info->refine_restarts = restarts;
        info->residual = resid;
        info->energy_unrefined = e_unrefined;
        info->applies = applies;
    }
    if (take_device_error(ctx)) fail(QSD_ERR_INTERNAL, "lanczos: hash probe exceeded the table size");
    if (timeout) return QSD_ERR_TIMEOUT;
    return converged ? QSD_OK : QSD_ERR_NOT_CONVERGED;
}

}  // namespace qsd
