// Operator group trimming (Results, chemistry: groups whose matrix elements
// are small against the smallest diagonal energy splitting of the subspace
// are removed before matrix evaluation).
//
// A group's elements are bounded by m_g = sum over its terms of |phi_t|
// (each term contributes at most |phi_t| to <r|H|r xor F>).  The splitting is
// Delta = min over rows with d_r > d_min of (d_r - d_min), the gap between the
// subspace's lowest diagonal energy and the next one.  A group is kept when
// m_g / Delta >= tol; diagonal terms and the identity are always kept.  The
// trimmed operator is loaded from the kept input words, so it is an
// operator like any other (grouping, tables and excitation index rebuilt).
#include <algorithm>
#include <cmath>
#include <unordered_set>
#include <vector>

#include "qsd_internal.cuh"

namespace qsd {

namespace {

__global__ void k_group_mag(int64_t G, const int32_t *__restrict__ grange, const double *__restrict__ re,
                            const double *__restrict__ im, double *mag) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    double m = 0.0;
    for (int32_t t = grange[g]; t < grange[g + 1]; ++t) m += hypot(re[t], im[t]);
    mag[g] = m;
}

struct WordsHash {
    size_t operator()(const std::vector<uint64_t> &v) const {
        uint64_t h = 0x9E3779B97F4A7C15ull;
        for (uint64_t x : v) h = fmix64(h ^ x);
        return (size_t)h;
    }
};

}  // namespace

void trim_operator(qsd_ctx ctx, qsd_op op, qsd_sub sub, const double *diag, double tol, qsd_op out,
                   qsd_trim_info *info) {
    cudaStream_t s = ctx->stream;
    const int W = op->W;
    const int64_t G = op->G, D = sub->D;
    std::vector<double> mag((size_t)G), d((size_t)D);
    if (G > 0) {
        DevBuf dm((size_t)G * 8);
        k_group_mag<<<blocks_for(G, 256), 256, 0, s>>>(G, op->grange.as<int32_t>(), op->tphi.as<double>(),
                                                        op->tphi_im.as<double>(), dm.as<double>());
        QSD_LAUNCH_CHECK();
        QSD_CUDA(cudaMemcpyAsync(mag.data(), dm.p, (size_t)G * 8, cudaMemcpyDeviceToHost, s));
    }
    if (D > 0) QSD_CUDA(cudaMemcpyAsync(d.data(), diag, (size_t)D * 8, cudaMemcpyDeviceToHost, s));
    QSD_CUDA(cudaStreamSynchronize(s));
    double dmin = D > 0 ? *std::min_element(d.begin(), d.end()) : 0.0;
    double split = 0.0;  // 0: every diagonal equal, nothing to compare with
    for (double v : d)
        if (v > dmin && (split == 0.0 || v - dmin < split)) split = v - dmin;
    std::unordered_set<std::vector<uint64_t>, WordsHash> keep;
    int64_t kept_groups = 0;
    for (int64_t g = 0; g < G; ++g) {
        if (split > 0.0 && !(mag[g] / split >= tol)) continue;
        keep.insert(std::vector<uint64_t>(op->host_groups.begin() + g * W, op->host_groups.begin() + (g + 1) * W));
        ++kept_groups;
    }
    // kept input words: diagonal ones, and those whose flip set is a kept group
    const int64_t T = (int64_t)op->in_term_ptr.size() - 1;
    std::vector<int64_t> tp(1, 0);
    std::vector<int32_t> oq;
    std::vector<uint8_t> oc;
    std::vector<double> cr, ci;
    std::vector<uint64_t> F((size_t)W);
    for (int64_t t = 0; t < T; ++t) {
        std::fill(F.begin(), F.end(), 0ull);
        bool flips = false;
        for (int64_t a = op->in_term_ptr[t]; a < op->in_term_ptr[t + 1]; ++a) {
            const int c = op->in_code[a];
            if (c >= 3) {  // X, Y, -, + flip the qubit
                F[op->in_qubit[a] >> 6] |= 1ull << (op->in_qubit[a] & 63);
                flips = true;
            }
        }
        if (flips && !keep.count(F)) continue;
        for (int64_t a = op->in_term_ptr[t]; a < op->in_term_ptr[t + 1]; ++a) {
            oq.push_back(op->in_qubit[a]);
            oc.push_back(op->in_code[a]);
        }
        tp.push_back((int64_t)oq.size());
        cr.push_back(op->in_re[t]);
        ci.push_back(op->in_im[t]);
    }
    load_operator(ctx, out, (int64_t)cr.size(), tp.data(), oq.data(), oc.data(), cr.data(), ci.data());
    info->groups_in = G;
    info->groups_kept = kept_groups;
    info->terms_in = T;
    info->terms_kept = (int64_t)cr.size();
    info->d_min = dmin;
    info->splitting = split;
}

}  // namespace qsd
