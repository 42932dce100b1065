// Instantiations of the sector-factored product for one precision mode.
//
// The build compiles this file once per mode with -DQSD_PREC=0, 1, 2 or 3
// (QSD_FP64, QSD_FP32_MIXED, QSD_FP32_DOT2, and kPrecWideX: the FP32-mixed
// block products on a widened copy of x -- block kernels only, no packed
// variants).
#include <algorithm>

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
    default:
#if QSD_PREC == 3
        fail(QSD_ERR_INTERNAL, "factored product on widened x: block widths 4 and 16 only");
#else
        k_apply_fac<W, 1, kPrec><<<(unsigned)blocks, 256, 0, s>>>(p, e, f);
#endif
        break;
    }
}
#if QSD_PREC != 3
template <int W, int KB>
int fac_resident_blocks() {
    static const int n = [] {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_apply_fac_queue<W, KB, kPrec>, 256, 0) !=
            cudaSuccess)
            b = 1;
        return std::max(b, 1);
    }();
    return n;
}

template <int W, int KB>
void launch_queue_one(const FacPair *params, const int64_t *tile0, TileQueue *q, int64_t max_tiles, int num_sms,
                      cudaStream_t s) {
    const int64_t grid = std::min<int64_t>(max_tiles, (int64_t)fac_resident_blocks<W, KB>() * num_sms);
    k_apply_fac_queue<W, KB, kPrec><<<(unsigned)std::max<int64_t>(grid, 1), 256, 0, s>>>(params, tile0, q);
}

template <int W>
void launch_queue_kb(const FacPair *params, const int64_t *tile0, TileQueue *q, int64_t max_tiles, int KB,
                     int num_sms, cudaStream_t s) {
    switch (KB) {
    case 16: launch_queue_one<W, 16>(params, tile0, q, max_tiles, num_sms, s); break;
    case 4: launch_queue_one<W, 4>(params, tile0, q, max_tiles, num_sms, s); break;
    default: launch_queue_one<W, 1>(params, tile0, q, max_tiles, num_sms, s); break;
    }
}
#endif
}  // namespace

#if QSD_PREC != 3
template <>
void launch_apply_fac_queue<kPrec>(const FacPair *params, const int64_t *tile0, TileQueue *q, int64_t max_tiles,
                                   int W, int KB, int num_sms, cudaStream_t s) {
    if (max_tiles <= 0) return;
    if (W > 2) fail(QSD_ERR_INTERNAL, "packed factored product: needs W <= 2");
    if (W == 1) launch_queue_kb<1>(params, tile0, q, max_tiles, KB, num_sms, s);
    else launch_queue_kb<2>(params, tile0, q, max_tiles, KB, num_sms, s);
    QSD_LAUNCH_CHECK();
}

#endif

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
