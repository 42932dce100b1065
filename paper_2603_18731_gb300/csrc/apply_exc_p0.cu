// Instantiations of the excitation product for precision mode 0.
#include "excite_kernel.cuh"

namespace qsd {

namespace {
template <int W>
void launch_kb(const ApplyParams &p, const ExcParams &e, int KB, int64_t blocks, cudaStream_t s) {
    switch (KB) {
    case 16: k_apply_exc<W, 16, 0><<<(unsigned)blocks, 256, 0, s>>>(p, e); break;
    case 4: k_apply_exc<W, 4, 0><<<(unsigned)blocks, 256, 0, s>>>(p, e); break;
    default: k_apply_exc<W, 1, 0><<<(unsigned)blocks, 256, 0, s>>>(p, e); break;
    }
}
}  // namespace

template <>
void launch_apply_exc<0>(const ApplyParams &p, const ExcParams &e, int W, int KB, cudaStream_t s) {
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
