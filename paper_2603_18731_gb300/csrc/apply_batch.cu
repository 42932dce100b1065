// Packed products: many (operator, subspace) pairs in one launch.
//
// A tile is 256 consecutive rows of one pair; the tiles of all pairs form one
// grid, so small products that would each fill a few blocks share a launch
// and the SMs.  Each block finds its pair by binary search over the pairs'
// first tiles, copies the pair's parameters to shared memory and evaluates
// its rows exactly as the single-pair group scan (one lane per row), so every
// pair's result is bitwise the single-pair product on path QSD_PATH_SCAN_1.
#include "apply_kernel.cuh"

namespace qsd {

namespace {

template <int W, int KB, int PREC>
__global__ void __launch_bounds__(256, (ApplyShape<W, KB>::MINB))
    k_apply_batch(const ApplyParams *__restrict__ params, const int64_t *__restrict__ tile0, int n) {
    __shared__ ApplyParams sp;
    __shared__ int pair;
    if (threadIdx.x == 0) {
        int lo = 0, hi = n - 1;  // last pair whose first tile <= blockIdx.x
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tile0[mid] <= (int64_t)blockIdx.x) lo = mid;
            else hi = mid - 1;
        }
        pair = lo;
    }
    __syncthreads();
    {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(params + pair);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&sp);
        for (int i = threadIdx.x; i < (int)(sizeof(ApplyParams) / 4); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const int64_t row = ((int64_t)blockIdx.x - tile0[pair]) * blockDim.x + threadIdx.x;
    apply_row<W, 1, KB, PREC>(sp, row);
}

template <int W, int PREC>
void launch_kb(const ApplyParams *params, const int64_t *tile0, int n, int64_t tiles, int KB, cudaStream_t s) {
    switch (KB) {
    case 16: k_apply_batch<W, 16, PREC><<<(unsigned)tiles, 256, 0, s>>>(params, tile0, n); break;
    case 4: k_apply_batch<W, 4, PREC><<<(unsigned)tiles, 256, 0, s>>>(params, tile0, n); break;
    default: k_apply_batch<W, 1, PREC><<<(unsigned)tiles, 256, 0, s>>>(params, tile0, n); break;
    }
}

template <int PREC>
void launch_w(const ApplyParams *params, const int64_t *tile0, int n, int64_t tiles, int W, int KB,
              cudaStream_t s) {
    switch (W) {
    case 1: launch_kb<1, PREC>(params, tile0, n, tiles, KB, s); break;
    case 2: launch_kb<2, PREC>(params, tile0, n, tiles, KB, s); break;
    case 3: launch_kb<3, PREC>(params, tile0, n, tiles, KB, s); break;
    default: launch_kb<4, PREC>(params, tile0, n, tiles, KB, s); break;
    }
}

}  // namespace

void launch_apply_batch(const ApplyParams *params, const int64_t *tile0, int n, int64_t tiles, int W, int KB,
                        int precision, cudaStream_t s) {
    if (n <= 0 || tiles <= 0) return;
    static_assert(sizeof(ApplyParams) % 4 == 0, "parameter copy by words");
    if (precision == QSD_FP64) launch_w<QSD_FP64>(params, tile0, n, tiles, W, KB, s);
    else if (precision == QSD_FP32_MIXED) launch_w<QSD_FP32_MIXED>(params, tile0, n, tiles, W, KB, s);
    else launch_w<QSD_FP32_DOT2>(params, tile0, n, tiles, W, KB, s);
    QSD_LAUNCH_CHECK();
}

}  // namespace qsd
