// Instantiations of the filter/verify product for one precision mode.
//
// The build compiles this file once per mode with -DQSD_PREC=0, 1, 2 or 3
// (QSD_FP64, QSD_FP32_MIXED, QSD_FP32_DOT2, and kFvWideX: the FP32-mixed
// block of 16 on a widened copy of x -- blocks of 16 only).
#include <algorithm>

#include "apply_fv.cuh"

#ifndef QSD_PREC
#error "compile with -DQSD_PREC=<precision mode>"
#endif

namespace qsd {

namespace {
constexpr int kPrec = QSD_PREC;

template <int W, int NB, int KB>
void launch_wc(const ApplyParams &p, int n_amp, int num_sms, cudaStream_t s) {
    const size_t smem = fv_smem_bytes(p.G, n_amp);
    const int64_t tiles = (p.D + kFvThreads - 1) / kFvThreads;
    int per_sm = 0;
    QSD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_apply_fv<W, kPrec, NB, KB>, kFvThreads, smem));
    const int64_t blocks = std::min<int64_t>(tiles, (int64_t)std::max(per_sm, 1) * num_sms);
    k_apply_fv<W, kPrec, NB, KB><<<(unsigned)blocks, kFvThreads, smem, s>>>(p, n_amp, tiles);
}

template <int W, int KB>
void launch_nb(const ApplyParams &p, int n_amp, int nb, int num_sms, cudaStream_t s) {
    if (nb == 0) launch_wc<W, 0, KB>(p, n_amp, num_sms, s);
    else if (nb == 2) launch_wc<W, 2, KB>(p, n_amp, num_sms, s);
    else launch_wc<W, -1, KB>(p, n_amp, num_sms, s);
}

template <int W>
void launch_w(const ApplyParams &p, int n_amp, int nb, int KB, int num_sms, cudaStream_t s) {
    if (KB == 16) launch_nb<W, 16>(p, n_amp, nb, num_sms, s);
#if QSD_PREC != 3
    else if (KB == 1) launch_nb<W, 1>(p, n_amp, nb, num_sms, s);
#endif
    else fail(QSD_ERR_INTERNAL, "filter/verify product: block widths 1 and 16 only (16 on widened x)");
}
}  // namespace

template <>
void launch_apply_fv<kPrec>(const ApplyParams &p, int n_amp, int W, int nb, int KB, int num_sms, cudaStream_t s) {
    if (p.D <= 0) return;
    if (p.G < 1 || p.G > kFvMaxGroups || n_amp > kFvMaxAmps || !p.hperm || fv_smem_bytes(p.G, n_amp) > 48 * 1024)
        fail(QSD_ERR_INTERNAL, "filter/verify product: operator or subspace outside its limits");
    switch (W) {
    case 1: launch_w<1>(p, n_amp, nb, KB, num_sms, s); break;
    case 2: launch_w<2>(p, n_amp, nb, KB, num_sms, s); break;
    case 3: launch_w<3>(p, n_amp, nb, KB, num_sms, s); break;
    case 4: launch_w<4>(p, n_amp, nb, KB, num_sms, s); break;
    default: fail(QSD_ERR_INTERNAL, "filter/verify product: W > 4");
    }
    QSD_LAUNCH_CHECK();
}

}  // namespace qsd
