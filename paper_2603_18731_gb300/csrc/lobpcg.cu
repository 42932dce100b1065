// Block eigensolver: LOBPCG (Knyazev, SIAM J. Sci. Comput. 23, 2001) with a
// shifted Jacobi (diagonal) preconditioner, the solver the paper uses for its
// chemistry runs (Results, chemistry: PRIMME's LOBPCG started from a vector
// spiked at the lowest diagonal, with a diagonal preconditioner shifted by
// the current eigenvalue estimate).
//
// The k lowest eigenpairs of the real symmetric H_S.  Per iteration:
// residuals R = H X - X Theta; preconditioned directions W = R / |d - theta|
// column by column (d the cached diagonal; the modulus keeps the
// preconditioner positive definite, as LOBPCG requires, and a floor keeps it
// bounded); W and the previous directions P projected off X (P also off W)
// and orthonormalised, so the basis [X, W, P] stays orthonormal and the
// images of W and P, updated by the same combinations, stay equal to H times
// them; the Rayleigh-Ritz problem on the basis (Gram matrices of the basis and
// of its image reduced on the device in a fixed order, the small eigenproblem
// solved on the host by cyclic Jacobi rotations with null directions
// dropped); X, P and their images updated from the Ritz coefficients.
// Products are FP64 block products (one lookup per group serves the k
// columns); every reduction has a fixed order, so a run is reproducible.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "lanczos.cuh"

namespace qsd {

namespace {

constexpr int kMaxBlock = 16;
constexpr int kMaxBasis = 3 * kMaxBlock;
constexpr int kGramRows = 32;  // rows staged in shared memory per tile

__device__ __forceinline__ double start_entry(uint64_t seed, uint64_t i) {
    uint64_t z = (seed ^ i) + 0x9E3779B97F4A7C15ull;
    z = fmix64(z);
    return 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
}

// X[r][c] = scale U(-1,1) (SplitMix64 of seed xor (r k + c)) + [r == rows[c]]
__global__ void k_start_block(int64_t D, int k, uint64_t seed, double scale, const int64_t *__restrict__ rows,
                              double *X) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= D * k) return;
    const int c = (int)(e % k);
    double v = scale * start_entry(seed, (uint64_t)e);
    if (rows && rows[c] == e / k) v += 1.0;
    X[e] = v;
}

// Columns of a basis: up to three [D][k] blocks side by side.
struct Cols {
    const double *b[3];
    int nb;
};

__device__ __forceinline__ double col_at(const Cols &c, int k, int64_t r, int i) {
    return c.b[i / k][r * k + (i % k)];
}

// partial[blk][i * mb + j] = sum over the block's rows of A[r][i] B[r][j]
__global__ void __launch_bounds__(256) k_gram_partial(const Cols A, int ma, const Cols B, int mb, int k, int64_t D,
                                                      double *partial) {
    __shared__ double sa[kGramRows][kMaxBasis], sb[kGramRows][kMaxBasis];
    const int np = ma * mb;
    double acc[(kMaxBasis * kMaxBasis + 255) / 256];
    const int nacc = (np + (int)blockDim.x - 1) / (int)blockDim.x;
    for (int q = 0; q < nacc; ++q) acc[q] = 0.0;
    const int64_t rows_per_block = (D + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_block, r1 = min(D, r0 + rows_per_block);
    for (int64_t t0 = r0; t0 < r1; t0 += kGramRows) {
        const int nr = (int)min((int64_t)kGramRows, r1 - t0);
        for (int e = threadIdx.x; e < nr * ma; e += blockDim.x) sa[e / ma][e % ma] = col_at(A, k, t0 + e / ma, e % ma);
        for (int e = threadIdx.x; e < nr * mb; e += blockDim.x) sb[e / mb][e % mb] = col_at(B, k, t0 + e / mb, e % mb);
        __syncthreads();
        for (int q = 0; q < nacc; ++q) {
            const int pidx = threadIdx.x + q * blockDim.x;
            if (pidx >= np) break;
            const int i = pidx / mb, j = pidx % mb;
            double s = acc[q];
            for (int rr = 0; rr < nr; ++rr) s = fma(sa[rr][i], sb[rr][j], s);
            acc[q] = s;
        }
        __syncthreads();
    }
    for (int q = 0; q < nacc; ++q) {
        const int pidx = threadIdx.x + q * blockDim.x;
        if (pidx < np) partial[(size_t)blockIdx.x * np + pidx] = acc[q];
    }
}

__global__ void k_gram_reduce(const double *__restrict__ partial, int nblk, int np, double *G) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += partial[(size_t)b * np + p];
    G[p] = s;
}

// Y[r][c] = sum_i S[r][i] C[i][c], c < kout (C row-major [m][kout])
__global__ void k_combine(const Cols S, int m, int k, int64_t D, const double *__restrict__ C, int kout, double *Y) {
    __shared__ double sc[kMaxBasis * kMaxBlock];
    for (int e = threadIdx.x; e < m * kout; e += blockDim.x) sc[e] = C[e];
    __syncthreads();
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= D) return;
    double y[kMaxBlock];
#pragma unroll
    for (int c = 0; c < kMaxBlock; ++c) y[c] = 0.0;
    for (int i = 0; i < m; ++i) {
        const double v = col_at(S, k, r, i);
#pragma unroll
        for (int c = 0; c < kMaxBlock; ++c)
            if (c < kout) y[c] = fma(v, sc[i * kout + c], y[c]);
    }
    for (int c = 0; c < kout; ++c) Y[r * kout + c] = y[c];
}

// R = AX - X diag(theta); W = R / max(|d - theta|, floor) (or W = R)
__global__ void k_residual_precond(const double *__restrict__ X, const double *__restrict__ AX,
                                   const double *__restrict__ theta, const double *__restrict__ d, int64_t D, int k,
                                   double floor_, int precond, double *R, double *W) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= D * k) return;
    const int c = (int)(e % k);
    const double res = AX[e] - theta[c] * X[e];
    R[e] = res;
    W[e] = precond ? res / fmax(fabs(d[e / k] - theta[c]), floor_) : res;
}

// ---------------------------------------------------------------- host
// Eigenvalues (ascending) and eigenvectors (columns of V, row-major) of the
// symmetric m x m matrix A by cyclic Jacobi rotations (Golub & Van Loan,
// Matrix Computations, the symmetric Jacobi method).
void jacobi_eigen(int m, std::vector<double> A, std::vector<double> &evals, std::vector<double> &V) {
    V.assign((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) V[(size_t)i * m + i] = 1.0;
    auto a = [&](int i, int j) -> double & { return A[(size_t)i * m + j]; };
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) {
                tot += a(i, j) * a(i, j);
                if (i != j) off += a(i, j) * a(i, j);
            }
        if (off <= 1e-30 * tot) break;
        for (int p = 0; p < m - 1; ++p)
            for (int q = p + 1; q < m; ++q) {
                const double apq = a(p, q);
                if (std::fabs(apq) < 1e-300) continue;
                const double tau = (a(q, q) - a(p, p)) / (2.0 * apq);
                const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
                const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
                for (int r = 0; r < m; ++r) {  // columns p, q
                    const double arp = a(r, p), arq = a(r, q);
                    a(r, p) = c * arp - s * arq;
                    a(r, q) = s * arp + c * arq;
                }
                for (int r = 0; r < m; ++r) {  // rows p, q
                    const double apr = a(p, r), aqr = a(q, r);
                    a(p, r) = c * apr - s * aqr;
                    a(q, r) = s * apr + c * aqr;
                }
                for (int r = 0; r < m; ++r) {
                    const double vrp = V[(size_t)r * m + p], vrq = V[(size_t)r * m + q];
                    V[(size_t)r * m + p] = c * vrp - s * vrq;
                    V[(size_t)r * m + q] = s * vrp + c * vrq;
                }
            }
    }
    std::vector<int> ord(m);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return a(x, x) < a(y, y); });
    std::vector<double> Vs((size_t)m * m);
    evals.resize(m);
    for (int c = 0; c < m; ++c) {
        evals[c] = a(ord[c], ord[c]);
        for (int r = 0; r < m; ++r) Vs[(size_t)r * m + c] = V[(size_t)r * m + ord[c]];
    }
    V.swap(Vs);
}

// Lowest k eigenpairs of (GA, GB) with coefficients C [m][k] (row-major).
// GB is diagonalised first and directions with eigenvalues below 1e-12 of
// the largest (null columns of the basis) are dropped; false when fewer than
// k directions remain.
bool rayleigh_ritz(int m, int k, std::vector<double> GA, const std::vector<double> &GB, std::vector<double> &theta,
                   std::vector<double> &C) {
    for (int i = 0; i < m; ++i)  // symmetrise the image Gram matrix
        for (int j = i + 1; j < m; ++j) {
            const double v = 0.5 * (GA[(size_t)i * m + j] + GA[(size_t)j * m + i]);
            GA[(size_t)i * m + j] = GA[(size_t)j * m + i] = v;
        }
    std::vector<double> lam, V;
    jacobi_eigen(m, GB, lam, V);
    const double lmax = lam.empty() ? 0.0 : lam.back();
    std::vector<int> keep;
    for (int i = 0; i < m; ++i)
        if (lam[i] > 1e-12 * lmax) keep.push_back(i);
    const int r = (int)keep.size();
    if (r < k) return false;
    // B = V[:, keep] diag(1 / sqrt(lam)) (m x r); M = B^T GA B (r x r)
    std::vector<double> B((size_t)m * r), T((size_t)m * r), M((size_t)r * r);
    for (int i = 0; i < m; ++i)
        for (int c = 0; c < r; ++c) B[(size_t)i * r + c] = V[(size_t)i * m + keep[c]] / std::sqrt(lam[keep[c]]);
    for (int i = 0; i < m; ++i)
        for (int c = 0; c < r; ++c) {
            double sum = 0.0;
            for (int q = 0; q < m; ++q) sum += GA[(size_t)i * m + q] * B[(size_t)q * r + c];
            T[(size_t)i * r + c] = sum;
        }
    for (int a = 0; a < r; ++a)
        for (int c = 0; c < r; ++c) {
            double sum = 0.0;
            for (int i = 0; i < m; ++i) sum += B[(size_t)i * r + a] * T[(size_t)i * r + c];
            M[(size_t)a * r + c] = sum;
        }
    std::vector<double> ev, U;
    jacobi_eigen(r, M, ev, U);
    theta.assign(ev.begin(), ev.begin() + k);
    C.assign((size_t)m * k, 0.0);
    for (int i = 0; i < m; ++i)
        for (int c = 0; c < k; ++c) {
            double sum = 0.0;
            for (int q = 0; q < r; ++q) sum += B[(size_t)i * r + q] * U[(size_t)q * r + c];
            C[(size_t)i * k + c] = sum;
        }
    return true;
}

struct Gram {
    qsd_ctx ctx = nullptr;
    int64_t D = 0;
    int k = 1, nblk = 1;
    DevBuf partial, G;
    std::vector<double> host;
    void init(qsd_ctx c, int64_t Dn, int kk) {
        ctx = c;
        D = Dn;
        k = kk;
        nblk = (int)std::max<int64_t>(1, std::min<int64_t>(2 * c->num_sms, (D + kGramRows - 1) / kGramRows));
        partial.alloc((size_t)nblk * kMaxBasis * kMaxBasis * 8);
        G.alloc((size_t)kMaxBasis * kMaxBasis * 8);
    }
    // host [ma][mb] = A^T B
    const std::vector<double> &run(const Cols &A, int ma, const Cols &B, int mb) {
        cudaStream_t s = ctx->stream;
        k_gram_partial<<<nblk, 256, 0, s>>>(A, ma, B, mb, k, D, partial.as<double>());
        k_gram_reduce<<<blocks_for(ma * mb, 256), 256, 0, s>>>(partial.as<double>(), nblk, ma * mb, G.as<double>());
        QSD_LAUNCH_CHECK();
        host.resize((size_t)ma * mb);
        QSD_CUDA(cudaMemcpyAsync(host.data(), G.p, host.size() * 8, cudaMemcpyDeviceToHost, s));
        QSD_CUDA(cudaStreamSynchronize(s));
        return host;
    }
};

}  // namespace

int lobpcg(qsd_ctx ctx, qsd_op op, qsd_sub sub, const double *diag, const qsd_lobpcg_params &p, double *evals,
           double *evecs, qsd_lobpcg_info *info) {
    cudaStream_t s = ctx->stream;
    const int64_t D = sub->D;
    const int k = p.k;
    const double tol = p.tol > 0 ? p.tol : 1e-9;
    const size_t nb = (size_t)D * k * 8;
    DevBuf X(nb), AX(nb), W(nb), AW(nb), P(nb), AP(nb), Xn(nb), AXn(nb), Pn(nb), APn(nb), R(nb);
    DevBuf C(8 * kMaxBasis * kMaxBlock), th(8 * kMaxBlock), spike(8 * kMaxBlock);
    Gram gram;
    gram.init(ctx, D, k);
    const int eb = blocks_for(D * k, 256), rb = blocks_for(D, 256);
    std::vector<double> hd((size_t)D);
    QSD_CUDA(cudaMemcpyAsync(hd.data(), diag, (size_t)D * 8, cudaMemcpyDeviceToHost, s));
    QSD_CUDA(cudaStreamSynchronize(s));

    // Y = S Cm (kout columns); Cm is uploaded and the call waits for the copy
    auto combine = [&](const Cols &S, int m, const std::vector<double> &Cm, int kout, double *Y) {
        QSD_CUDA(cudaMemcpyAsync(C.p, Cm.data(), Cm.size() * 8, cudaMemcpyHostToDevice, s));
        k_combine<<<rb, 256, 0, s>>>(S, m, k, D, C.as<double>(), kout, Y);
        QSD_LAUNCH_CHECK();
        QSD_CUDA(cudaStreamSynchronize(s));
    };
    auto product = [&](const double *x, double *y) { apply_H(ctx, op, sub, diag, QSD_FP64, k, x, y, s, true); };
    // Y <- Y - Q (Q^T Y), twice, and its image alongside
    auto project = [&](DevBuf &Y, DevBuf *AY, DevBuf &Q, DevBuf *AQ) {
        for (int rep = 0; rep < 2; ++rep) {
            const Cols cq{{Q.as<double>(), nullptr, nullptr}, 1}, cy{{Y.as<double>(), nullptr, nullptr}, 1};
            const std::vector<double> M = gram.run(cq, k, cy, k);
            std::vector<double> Cc((size_t)2 * k * k, 0.0);
            for (int i = 0; i < k; ++i)
                for (int c = 0; c < k; ++c) {
                    Cc[(size_t)i * k + c] = -M[(size_t)i * k + c];
                    Cc[(size_t)(k + i) * k + c] = (i == c) ? 1.0 : 0.0;
                }
            const Cols qy{{Q.as<double>(), Y.as<double>(), nullptr}, 2};
            combine(qy, 2 * k, Cc, k, Xn.as<double>());
            std::swap(Y, Xn);
            if (AY) {
                const Cols aqy{{AQ->as<double>(), AY->as<double>(), nullptr}, 2};
                combine(aqy, 2 * k, Cc, k, Xn.as<double>());
                std::swap(*AY, Xn);
            }
        }
    };
    // orthonormal columns through the eigen-decomposition of the Gram matrix;
    // directions below 1e-10 of the largest become zero columns
    auto orthonormalize = [&](DevBuf &Y, DevBuf *AY) {
        const Cols cy{{Y.as<double>(), nullptr, nullptr}, 1};
        const std::vector<double> G = gram.run(cy, k, cy, k);
        std::vector<double> lam, V;
        jacobi_eigen(k, G, lam, V);
        std::vector<double> T((size_t)k * k, 0.0);
        const double lmax = lam.back();
        int col = 0;
        for (int i = 0; i < k && lmax > 0.0; ++i) {
            if (!(lam[i] > 1e-10 * lmax)) continue;
            for (int r = 0; r < k; ++r) T[(size_t)r * k + col] = V[(size_t)r * k + i] / std::sqrt(lam[i]);
            ++col;
        }
        combine(cy, k, T, k, Xn.as<double>());
        std::swap(Y, Xn);
        if (AY) {
            const Cols cay{{AY->as<double>(), nullptr, nullptr}, 1};
            combine(cay, k, T, k, Xn.as<double>());
            std::swap(*AY, Xn);
        }
    };

    // start block: given, or unit spikes at the k lowest diagonal entries
    // (ties: lower index) plus 1e-3 U(-1,1), or U(-1,1)
    if (p.x0) {
        QSD_CUDA(cudaMemcpyAsync(X.p, p.x0, nb, cudaMemcpyDeviceToDevice, s));
    } else {
        std::vector<int64_t> rows;
        if (p.start == 0) {
            std::vector<int64_t> idx((size_t)D);
            std::iota(idx.begin(), idx.end(), (int64_t)0);
            std::partial_sort(idx.begin(), idx.begin() + k, idx.end(), [&](int64_t a, int64_t b) {
                return hd[a] < hd[b] || (hd[a] == hd[b] && a < b);
            });
            rows.assign(idx.begin(), idx.begin() + k);
            QSD_CUDA(cudaMemcpyAsync(spike.p, rows.data(), (size_t)k * 8, cudaMemcpyHostToDevice, s));
        }
        k_start_block<<<eb, 256, 0, s>>>(D, k, p.seed, p.start == 0 ? 1e-3 : 1.0,
                                         p.start == 0 ? spike.as<int64_t>() : nullptr, X.as<double>());
        QSD_LAUNCH_CHECK();
        QSD_CUDA(cudaStreamSynchronize(s));
    }
    orthonormalize(X, nullptr);
    product(X.as<double>(), AX.as<double>());
    std::vector<double> theta, Cm;
    {
        // Rayleigh-Ritz on X alone gives the first Ritz values
        const Cols cx{{X.as<double>(), nullptr, nullptr}, 1}, cax{{AX.as<double>(), nullptr, nullptr}, 1};
        const std::vector<double> GA = gram.run(cx, k, cax, k);
        const std::vector<double> GB = gram.run(cx, k, cx, k);
        if (!rayleigh_ritz(k, k, GA, GB, theta, Cm))
            fail(QSD_ERR_INVALID_ARG, "qsd_lobpcg: the start block does not have rank k");
        combine(cx, k, Cm, k, Xn.as<double>());
        combine(cax, k, Cm, k, AXn.as<double>());
        std::swap(X, Xn);
        std::swap(AX, AXn);
    }
    double dmax = 1.0;
    for (double v : hd) dmax = std::max(dmax, std::fabs(v));
    const double floor_ = 1e-8 * dmax;
    bool have_p = false;
    int it = 0;
    double max_res = 0.0;
    bool converged = false;
    for (; it < std::max(p.max_iters, 1); ++it) {
        QSD_CUDA(cudaMemcpyAsync(th.p, theta.data(), (size_t)k * 8, cudaMemcpyHostToDevice, s));
        k_residual_precond<<<eb, 256, 0, s>>>(X.as<double>(), AX.as<double>(), th.as<double>(), diag, D, k, floor_,
                                              p.precondition, R.as<double>(), W.as<double>());
        QSD_LAUNCH_CHECK();
        const Cols cr{{R.as<double>(), nullptr, nullptr}, 1};
        const std::vector<double> RR = gram.run(cr, k, cr, k);
        max_res = 0.0;
        for (int c = 0; c < k; ++c)
            max_res = std::max(max_res, std::sqrt(std::max(RR[(size_t)c * k + c], 0.0)) /
                                            std::max(std::fabs(theta[c]), 1e-300));
        if (max_res <= tol) {
            converged = true;
            break;
        }
        project(W, nullptr, X, &AX);
        orthonormalize(W, nullptr);
        product(W.as<double>(), AW.as<double>());
        if (have_p) {
            project(P, &AP, X, &AX);
            project(P, &AP, W, &AW);
            orthonormalize(P, &AP);
        }
        const int m = have_p ? 3 * k : 2 * k;
        const Cols S{{X.as<double>(), W.as<double>(), have_p ? P.as<double>() : nullptr}, have_p ? 3 : 2};
        const Cols AS{{AX.as<double>(), AW.as<double>(), have_p ? AP.as<double>() : nullptr}, have_p ? 3 : 2};
        const std::vector<double> GA = gram.run(S, m, AS, m);
        const std::vector<double> GB = gram.run(S, m, S, m);
        std::vector<double> nth;
        if (!rayleigh_ritz(m, k, GA, GB, nth, Cm)) fail(QSD_ERR_INTERNAL, "qsd_lobpcg: basis lost rank");
        combine(S, m, Cm, k, Xn.as<double>());
        combine(AS, m, Cm, k, AXn.as<double>());
        // search directions: the W and P parts of the Ritz vectors
        std::vector<double> Cp = Cm;
        for (size_t i = 0; i < (size_t)k * k; ++i) Cp[i] = 0.0;
        combine(S, m, Cp, k, Pn.as<double>());
        combine(AS, m, Cp, k, APn.as<double>());
        std::swap(X, Xn);
        std::swap(AX, AXn);
        std::swap(P, Pn);
        std::swap(AP, APn);
        theta = nth;
        have_p = true;
    }
    for (int c = 0; c < k; ++c) evals[c] = theta[c];
    if (evecs) QSD_CUDA(cudaMemcpyAsync(evecs, X.p, nb, cudaMemcpyDeviceToDevice, s));
    QSD_CUDA(cudaStreamSynchronize(s));
    info->iters = it;
    info->converged = converged ? 1 : 0;
    info->max_residual = max_res;
    info->status = converged ? QSD_OK : QSD_ERR_NOT_CONVERGED;
    return info->status;
}

}  // namespace qsd
