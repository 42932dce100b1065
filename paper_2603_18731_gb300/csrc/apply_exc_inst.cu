// Instantiations of the excitation product for one precision mode.
//
// The build compiles this file once per mode with -DQSD_PREC=0, 1 or 2
// (QSD_FP64, QSD_FP32_MIXED, QSD_FP32_DOT2).
#include "excite_kernel.cuh"

#ifndef QSD_PREC
#error "compile with -DQSD_PREC=<precision mode>"
#endif

namespace qsd {

namespace {
constexpr int kPrec = QSD_PREC;

template <int W>
void launch_kb(const ApplyParams &p, const ExcParams &e, int KB, int64_t blocks, cudaStream_t s) {
    switch (KB) {
    case 16: k_apply_exc<W, 16, kPrec><<<(unsigned)blocks, 256, 0, s>>>(p, e); break;
    case 4: k_apply_exc<W, 4, kPrec><<<(unsigned)blocks, 256, 0, s>>>(p, e); break;
    default: k_apply_exc<W, 1, kPrec><<<(unsigned)blocks, 256, 0, s>>>(p, e); break;
    }
}
}  // namespace

template <>
void launch_apply_exc<kPrec>(const ApplyParams &p, const ExcParams &e, int W, int KB, cudaStream_t s) {
    if (p.D <= 0) return;
    const int64_t blocks = (p.D * 32 + 255) / 256;  // a warp per row
    switch (W) {
    case 1: launch_kb<1>(p, e, KB, blocks, s); break;
    case 2: launch_kb<2>(p, e, KB, blocks, s); break;
    case 3: launch_kb<3>(p, e, KB, blocks, s); break;
    default: launch_kb<4>(p, e, KB, blocks, s); break;
    }
    QSD_LAUNCH_CHECK();
}

}  // namespace qsd
