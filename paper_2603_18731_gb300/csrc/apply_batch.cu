// Packed group-scan products: many (operator, subspace) pairs in one launch.
//
// A tile is 256 / R consecutive rows of one pair (R lanes per row).  A
// persistent grid serves the tiles of all pairs of one key width from a
// device tile queue (tile_queue.cuh): each block claims tiles until they run
// out, keeps the current pair's parameters in shared memory and evaluates
// its rows exactly as the single-pair group scan with R lanes per row, so
// every pair's result is bitwise the single-pair product on path
// QSD_PATH_SCAN_1 (R = 1) or QSD_PATH_SCAN_8 (R = 8).
#include <algorithm>

#include "apply_kernel.cuh"
#include "tile_queue.cuh"

namespace qsd {

namespace {

template <int W, int R, int KB, int PREC>
__global__ void __launch_bounds__(256, (ApplyShape<W, KB>::MINB))
    k_apply_queue(const ApplyParams *__restrict__ params, const int64_t *__restrict__ tile0, TileQueue *q) {
    __shared__ ApplyParams sp;
    run_tile_queue(params, tile0, q, sp, [](const ApplyParams &p, int, int64_t t) {
        apply_row<W, R, KB, PREC>(p, t * (256 / R) + threadIdx.x / R);
    });
}

// Blocks of one variant resident on an SM at once (cached per variant).
template <int W, int R, int KB, int PREC>
int resident_blocks() {
    static const int n = [] {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_apply_queue<W, R, KB, PREC>, 256, 0) != cudaSuccess)
            b = 1;
        return std::max(b, 1);
    }();
    return n;
}

template <int W, int R, int KB, int PREC>
void launch_one(const ApplyParams *params, const int64_t *tile0, TileQueue *q, int64_t max_tiles, int num_sms,
                cudaStream_t s) {
    const int64_t grid = std::min<int64_t>(max_tiles, (int64_t)resident_blocks<W, R, KB, PREC>() * num_sms);
    k_apply_queue<W, R, KB, PREC><<<(unsigned)std::max<int64_t>(grid, 1), 256, 0, s>>>(params, tile0, q);
}

// R = 8 (the single-column products of packed Lanczos chunks): KB = 1 only
template <int W, int PREC>
void launch_kb(const ApplyParams *params, const int64_t *tile0, TileQueue *q, int64_t max_tiles, int R, int KB,
               int num_sms, cudaStream_t s) {
    if (R == 8) {
        if (KB != 1) fail(QSD_ERR_INTERNAL, "packed scan: 8 lanes per row take single columns");
        launch_one<W, 8, 1, PREC>(params, tile0, q, max_tiles, num_sms, s);
        return;
    }
    switch (KB) {
    case 16: launch_one<W, 1, 16, PREC>(params, tile0, q, max_tiles, num_sms, s); break;
    case 4: launch_one<W, 1, 4, PREC>(params, tile0, q, max_tiles, num_sms, s); break;
    default: launch_one<W, 1, 1, PREC>(params, tile0, q, max_tiles, num_sms, s); break;
    }
}

template <int PREC>
void launch_w(const ApplyParams *params, const int64_t *tile0, TileQueue *q, int64_t max_tiles, int W, int R, int KB,
              int num_sms, cudaStream_t s) {
    switch (W) {
    case 1: launch_kb<1, PREC>(params, tile0, q, max_tiles, R, KB, num_sms, s); break;
    case 2: launch_kb<2, PREC>(params, tile0, q, max_tiles, R, KB, num_sms, s); break;
    case 3: launch_kb<3, PREC>(params, tile0, q, max_tiles, R, KB, num_sms, s); break;
    default: launch_kb<4, PREC>(params, tile0, q, max_tiles, R, KB, num_sms, s); break;
    }
}

}  // namespace

void launch_apply_queue(const ApplyParams *params, const int64_t *tile0, TileQueue *q, int64_t max_tiles, int W,
                        int R, int KB, int precision, int num_sms, cudaStream_t s) {
    if (max_tiles <= 0) return;
    if (precision == QSD_FP64) launch_w<QSD_FP64>(params, tile0, q, max_tiles, W, R, KB, num_sms, s);
    else if (precision == QSD_FP32_MIXED)
        launch_w<QSD_FP32_MIXED>(params, tile0, q, max_tiles, W, R, KB, num_sms, s);
    else launch_w<QSD_FP32_DOT2>(params, tile0, q, max_tiles, W, R, KB, num_sms, s);
    QSD_LAUNCH_CHECK();
}

}  // namespace qsd
