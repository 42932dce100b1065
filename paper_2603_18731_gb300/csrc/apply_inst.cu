// Instantiations of the group-scan product kernel for one precision mode.
//
// The build compiles this file once per mode with -DQSD_PREC=0, 1 or 2
// (QSD_FP64, QSD_FP32_MIXED, QSD_FP32_DOT2), so the three modes compile in
// parallel from one source.
#include <algorithm>

#include "apply_kernel.cuh"

#ifndef QSD_PREC
#error "compile with -DQSD_PREC=<precision mode>"
#endif

namespace qsd {

namespace {
constexpr int kPrec = QSD_PREC;
// the run-time-W kernel keeps FP64 storage in mode 0, FP32 otherwise
using TDyn = typename std::conditional<kPrec == QSD_FP64, double, float>::type;

template <int W, int R, bool HO = false>
void launch_kb(const ApplyParams &p, int KB, int64_t blocks, cudaStream_t s) {
    switch (KB) {
    case 16: k_apply<W, R, 16, kPrec, false, HO><<<(unsigned)blocks, 256, 0, s>>>(p); break;
    case 4: k_apply<W, R, 4, kPrec, false, HO><<<(unsigned)blocks, 256, 0, s>>>(p); break;
    default: k_apply<W, R, 1, kPrec, false, HO><<<(unsigned)blocks, 256, 0, s>>>(p); break;
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

template <>
void launch_apply<kPrec>(const ApplyParams &p, int W, int R, int KB, cudaStream_t s, bool hash_order) {
    if (p.D <= 0) return;
    if (hash_order && (W > kMaxWordsStatic || !p.hperm)) fail(QSD_ERR_INTERNAL, "hash-order product without hash order");
    switch (W) {
    case 1: launch_r<1>(p, R, KB, s, hash_order); break;
    case 2: launch_r<2>(p, R, KB, s, hash_order); break;
    case 3: launch_r<3>(p, R, KB, s, hash_order); break;
    case 4: launch_r<4>(p, R, KB, s, hash_order); break;
    default: {
        const int64_t blocks = (p.D + 255) / 256;
        switch (KB) {
        case 16: k_apply_dyn<16, TDyn><<<(unsigned)blocks, 256, 0, s>>>(p, W); break;
        case 4: k_apply_dyn<4, TDyn><<<(unsigned)blocks, 256, 0, s>>>(p, W); break;
        default: k_apply_dyn<1, TDyn><<<(unsigned)blocks, 256, 0, s>>>(p, W); break;
        }
    }
    }
    QSD_LAUNCH_CHECK();
}

}  // namespace qsd
