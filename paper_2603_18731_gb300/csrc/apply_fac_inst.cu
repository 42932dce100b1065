// Instantiations of the sector-factored product for one precision mode.
//
// The build compiles this file once per mode with -DQSD_PREC=0, 1 or 2
// (QSD_FP64, QSD_FP32_MIXED, QSD_FP32_DOT2).
#include "factor_kernel.cuh"

#ifndef QSD_PREC
#error "compile with -DQSD_PREC=<precision mode>"
#endif

namespace qsd {

namespace {
constexpr int kPrec = QSD_PREC;

template <int W>
void launch_kb(const ApplyParams &p, const ExcParams &e, const FacParams &f, int KB, int64_t blocks,
               cudaStream_t s) {
    switch (KB) {
    case 16: k_apply_fac<W, 16, kPrec><<<(unsigned)blocks, 256, 0, s>>>(p, e, f); break;
    case 4: k_apply_fac<W, 4, kPrec><<<(unsigned)blocks, 256, 0, s>>>(p, e, f); break;
    default: k_apply_fac<W, 1, kPrec><<<(unsigned)blocks, 256, 0, s>>>(p, e, f); break;
    }
}
}  // namespace

template <>
void launch_apply_fac<kPrec>(const ApplyParams &p, const ExcParams &e, const FacParams &f, int W, int KB,
                             cudaStream_t s) {
    if (p.D <= 0) return;
    if (W > 2 || !e.dense) fail(QSD_ERR_INTERNAL, "factored product: needs W <= 2 and a rank index");
    const int64_t blocks = (p.D * 32 + 255) / 256;  // a warp per row
    if (W == 1) launch_kb<1>(p, e, f, KB, blocks, s);
    else launch_kb<2>(p, e, f, KB, blocks, s);
    QSD_LAUNCH_CHECK();
}

}  // namespace qsd
