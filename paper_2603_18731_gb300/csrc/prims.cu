// Device primitives used by the set-up steps: prefix sums, a stable LSD
// radix sort of multi-word keys, and deduplication of sorted keys.
#include "qsd_internal.cuh"

namespace qsd {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// Exclusive block-wide scan of one value per thread; *total gets the sum.
__device__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *warp_sums, uint32_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) warp_sums[lane] = w;
    }
    __syncthreads();
    const uint32_t before = warp ? warp_sums[warp - 1] : 0;
    *total = warp_sums[nw - 1];
    __syncthreads();
    return before + x - v;
}

__global__ void k_tile_sums(const uint32_t *__restrict__ in, int64_t n, uint32_t *sums) {
    __shared__ uint32_t ws[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) s += in[base + i];
    uint32_t total;
    block_exclusive_scan(s, ws, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void k_tile_scan(const uint32_t *__restrict__ in, uint32_t *out, int64_t n,
                            const uint32_t *__restrict__ offs) {
    __shared__ uint32_t ws[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = base + i < n ? in[base + i] : 0;
        s += v[i];
    }
    uint32_t total;
    uint32_t run = block_exclusive_scan(s, ws, &total) + (offs ? offs[blockIdx.x] : 0);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
}

// ---------------------------------------------------------------- radix sort
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortRounds = 16;
constexpr int kSortTile = kSortThreads * kSortRounds;

__global__ void k_or_and(const uint64_t *__restrict__ keys, int K, int64_t n, unsigned long long *oa) {
    const int w = blockIdx.y;
    const uint64_t *k = keys + (size_t)w * n;
    uint64_t o = 0, a = ~0ull;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t v = k[i];
        o |= v;
        a &= v;
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        o |= __shfl_xor_sync(0xffffffffu, o, s);
        a &= __shfl_xor_sync(0xffffffffu, a, s);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicOr(oa + 2 * w, (unsigned long long)o);
        atomicAnd(oa + 2 * w + 1, (unsigned long long)a);
    }
}

__global__ void k_sort_hist(const uint64_t *__restrict__ kw, int64_t n, int shift, uint32_t *hist, int nb) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int i = threadIdx.x; i < kSortTile; i += kSortThreads) {
        const int64_t j = base + i;
        if (j < n) atomicAdd(&h[(kw[j] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of one tile by one 8-bit digit.  Items of a tile are taken
// in 16 rounds of 256 consecutive items; within a round the rank of an item
// among equal digits is (items of lower warps) + (lower lanes of its warp).
__global__ void k_sort_scatter(const uint64_t *__restrict__ kin, uint64_t *__restrict__ kout, int K,
                               int64_t n, const uint32_t *__restrict__ pin, uint32_t *__restrict__ pout,
                               int word, int shift, const uint32_t *__restrict__ hist, int nb) {
    __shared__ uint32_t dig_off[256];
    __shared__ uint32_t wcnt[kSortWarps][256];
    __shared__ uint32_t tot[256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    dig_off[tid] = hist[(size_t)tid * nb + blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    const uint32_t lt = (1u << lane) - 1u;
    for (int r = 0; r < kSortRounds; ++r) {
        if (base + (int64_t)r * kSortThreads >= n) break;  // uniform across the block
#pragma unroll
        for (int wp = 0; wp < kSortWarps; ++wp) wcnt[wp][tid] = 0;
        __syncthreads();
        const int64_t j = base + (int64_t)r * kSortThreads + tid;
        const bool valid = j < n;
        const uint32_t d = valid ? (uint32_t)((kin[(size_t)word * n + j] >> shift) & 255u) : 256u;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t rank = __popc(peers & lt);
        if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        uint32_t run = 0;
#pragma unroll
        for (int wp = 0; wp < kSortWarps; ++wp) {
            const uint32_t c = wcnt[wp][tid];
            wcnt[wp][tid] = run;
            run += c;
        }
        tot[tid] = run;
        __syncthreads();
        if (valid) {
            const uint32_t dst = dig_off[d] + wcnt[warp][d] + rank;
            for (int k = 0; k < K; ++k) kout[(size_t)k * n + dst] = kin[(size_t)k * n + j];
            if (pin) pout[dst] = pin[j];
        }
        __syncthreads();
        dig_off[tid] += tot[tid];
    }
}

__global__ void k_diff_flags(const uint64_t *__restrict__ keys, int K, int64_t n, uint32_t *flags) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t f = 1;
    if (i > 0) {
        f = 0;
        for (int k = 0; k < K; ++k) f |= keys[(size_t)k * n + i] != keys[(size_t)k * n + i - 1];
    }
    flags[i] = f;
}

__global__ void k_compact_keys(const uint64_t *__restrict__ keys, int K, int64_t n,
                               const uint32_t *__restrict__ flags, const uint32_t *__restrict__ pos,
                               uint64_t *out, int64_t n_out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !flags[i]) return;
    const uint32_t d = pos[i];
    for (int k = 0; k < K; ++k) out[(size_t)k * n_out + d] = keys[(size_t)k * n + i];
}

}  // namespace

uint64_t exclusive_scan_u32(qsd_ctx ctx, const uint32_t *in, uint32_t *out, int64_t n, bool want_total) {
    if (n <= 0) return 0;
    cudaStream_t s = ctx->stream;
    uint32_t last_in = 0;
    if (want_total) QSD_CUDA(cudaMemcpyAsync(&last_in, in + n - 1, 4, cudaMemcpyDeviceToHost, s));
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb == 1) {
        k_tile_scan<<<1, kScanThreads, 0, s>>>(in, out, n, nullptr);
        QSD_LAUNCH_CHECK();
    } else {
        DevBuf sums((size_t)nb * 4);
        k_tile_sums<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, sums.as<uint32_t>());
        QSD_LAUNCH_CHECK();
        exclusive_scan_u32(ctx, sums.as<uint32_t>(), sums.as<uint32_t>(), nb, false);
        k_tile_scan<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, sums.as<uint32_t>());
        QSD_LAUNCH_CHECK();
        QSD_CUDA(cudaStreamSynchronize(s));  // sums is freed on return
    }
    if (!want_total) return 0;
    uint32_t last_out = 0;
    QSD_CUDA(cudaMemcpyAsync(&last_out, out + n - 1, 4, cudaMemcpyDeviceToHost, s));
    QSD_CUDA(cudaStreamSynchronize(s));
    return (uint64_t)last_out + last_in;
}

void radix_sort(qsd_ctx ctx, uint64_t *keys, int K, int64_t n, uint32_t *payload) {
    if (n <= 1) return;
    if (n >= (int64_t)0xffffffffLL) fail(QSD_ERR_CAPACITY, "radix_sort: more than 2^32-1 items");
    cudaStream_t s = ctx->stream;
    // which digits vary: bits where OR != AND
    DevBuf oa((size_t)K * 16);
    std::vector<unsigned long long> h_oa(2 * K);
    for (int w = 0; w < K; ++w) { h_oa[2 * w] = 0; h_oa[2 * w + 1] = ~0ull; }
    QSD_CUDA(cudaMemcpyAsync(oa.p, h_oa.data(), (size_t)K * 16, cudaMemcpyHostToDevice, s));
    {
        dim3 grid((unsigned)std::min<int64_t>(blocks_for(n, 256), 1024), (unsigned)K);
        k_or_and<<<grid, 256, 0, s>>>(keys, K, n, oa.as<unsigned long long>());
        QSD_LAUNCH_CHECK();
    }
    QSD_CUDA(cudaMemcpyAsync(h_oa.data(), oa.p, (size_t)K * 16, cudaMemcpyDeviceToHost, s));
    QSD_CUDA(cudaStreamSynchronize(s));
    std::vector<std::pair<int, int>> passes;
    for (int w = 0; w < K; ++w) {
        const uint64_t var = h_oa[2 * w] ^ h_oa[2 * w + 1];
        for (int b = 0; b < 8; ++b)
            if ((var >> (8 * b)) & 255u) passes.push_back({w, 8 * b});
    }
    if (passes.empty()) return;
    const int nb = (int)((n + kSortTile - 1) / kSortTile);
    DevBuf kalt((size_t)K * n * 8), palt(payload ? (size_t)n * 4 : 0), hist((size_t)256 * nb * 4);
    uint64_t *kin = keys, *kout = kalt.as<uint64_t>();
    uint32_t *pin = payload, *pout = palt.as<uint32_t>();
    for (auto [w, shift] : passes) {
        k_sort_hist<<<nb, kSortThreads, 0, s>>>(kin + (size_t)w * n, n, shift, hist.as<uint32_t>(), nb);
        QSD_LAUNCH_CHECK();
        exclusive_scan_u32(ctx, hist.as<uint32_t>(), hist.as<uint32_t>(), (int64_t)256 * nb, false);
        k_sort_scatter<<<nb, kSortThreads, 0, s>>>(kin, kout, K, n, pin, pout, w, shift, hist.as<uint32_t>(), nb);
        QSD_LAUNCH_CHECK();
        std::swap(kin, kout);
        std::swap(pin, pout);
    }
    if (kin != keys) {
        QSD_CUDA(cudaMemcpyAsync(keys, kin, (size_t)K * n * 8, cudaMemcpyDeviceToDevice, s));
        if (payload) QSD_CUDA(cudaMemcpyAsync(payload, pin, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
    }
    QSD_CUDA(cudaStreamSynchronize(s));  // temporaries are freed on return
}

void diff_flags(qsd_ctx ctx, const uint64_t *keys, int K, int64_t n, uint32_t *flags) {
    if (n <= 0) return;
    k_diff_flags<<<blocks_for(n, 256), 256, 0, ctx->stream>>>(keys, K, n, flags);
    QSD_LAUNCH_CHECK();
}

int64_t unique_sorted(qsd_ctx ctx, const uint64_t *keys, int K, int64_t n, uint64_t *out, int64_t out_cap) {
    if (n <= 0) return 0;
    cudaStream_t s = ctx->stream;
    DevBuf flags((size_t)n * 4), pos((size_t)n * 4);
    k_diff_flags<<<blocks_for(n, 256), 256, 0, s>>>(keys, K, n, flags.as<uint32_t>());
    QSD_LAUNCH_CHECK();
    const int64_t m = (int64_t)exclusive_scan_u32(ctx, flags.as<uint32_t>(), pos.as<uint32_t>(), n, true);
    if (out) {
        if (m > out_cap) fail(QSD_ERR_INTERNAL, "unique_sorted: output too small");
        k_compact_keys<<<blocks_for(n, 256), 256, 0, s>>>(keys, K, n, flags.as<uint32_t>(), pos.as<uint32_t>(), out, m);
        QSD_LAUNCH_CHECK();
        QSD_CUDA(cudaStreamSynchronize(s));
    }
    return m;
}

}  // namespace qsd
