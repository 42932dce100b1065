// Instantiations of the half-evaluation product (Hermitian real operators,
// FP64): lower-triangle groups only, mirrored by FP64 atomic adds.
#include "apply_kernel.cuh"

namespace qsd {

namespace {
template <int W, int R, bool HO = false>
void launch_kb(const ApplyParams &p, int KB, int64_t blocks, cudaStream_t s) {
    switch (KB) {
    case 16: k_apply<W, R, 16, 0, true, HO><<<(unsigned)blocks, 256, 0, s>>>(p); break;
    case 4: k_apply<W, R, 4, 0, true, HO><<<(unsigned)blocks, 256, 0, s>>>(p); break;
    default: k_apply<W, R, 1, 0, true, HO><<<(unsigned)blocks, 256, 0, s>>>(p); break;
    }
}

template <int W>
void launch_r(const ApplyParams &p, int R, int KB, cudaStream_t s, bool ho) {
    const int64_t blocks = (p.D * R + 255) / 256;
    if (ho) launch_kb<W, 1, true>(p, KB, blocks, s);
    else if (R == 8) launch_kb<W, 8>(p, KB, blocks, s);
    else launch_kb<W, 1>(p, KB, blocks, s);
}
}  // namespace

void launch_apply_sym(const ApplyParams &p, int W, int R, int KB, cudaStream_t s, bool hash_order) {
    if (p.D <= 0) return;
    if (hash_order && !p.hperm) fail(QSD_ERR_INTERNAL, "hash-order product without hash order");
    // the rows' atomic adds need this launch's columns of y zeroed first
    QSD_CUDA(cudaMemset2DAsync(static_cast<double *>(p.y) + p.col0, (size_t)p.ld * 8, 0, (size_t)KB * 8,
                               (size_t)p.D, s));
    switch (W) {
    case 1: launch_r<1>(p, R, KB, s, hash_order); break;
    case 2: launch_r<2>(p, R, KB, s, hash_order); break;
    case 3: launch_r<3>(p, R, KB, s, hash_order); break;
    case 4: launch_r<4>(p, R, KB, s, hash_order); break;
    default: fail(QSD_ERR_INTERNAL, "half-evaluation product: W > 4");
    }
    QSD_LAUNCH_CHECK();
}

}  // namespace qsd
