// qsd_rayleigh_quotient_noalloc: the Rayleigh quotient without any device
// allocation, for callers that cannot call cudaMalloc:
//   * host programs that hand the whole device to their own memory pool or
//     allocator at start-up, so that an allocation by this library would fail
//     or fragment memory the host program owns;
//   * serving or real-time loops that reserve all their memory up front and
//     must not reach the allocator mid-flight, because cudaMalloc and cudaFree
//     can synchronise the device and stall the work of every other stream.
//
// The scratch it needs (H u, the diagonal of H_S and per-block partial sums)
// lives in one file-scope __device__ array of fixed size, so every GPU that
// loads this library holds kNoAllocBytes of it until the process exits.
// Host code cannot pass the array's name to a kernel (in host code the name is
// a host-side stand-in, not a device address), so the first call on a device
// looks the address up with cudaGetSymbolAddress, with that device current,
// and caches it; make that first call before any stream capture.  All calls
// share the one array and it keeps the last call's contents: calls whose work
// overlaps on the GPU (two streams, two threads) race and must be serialised
// by the caller.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "qsd_internal.cuh"

namespace qsd {

namespace {

constexpr int64_t kNoAllocMaxRows = 1 << 20;   // largest subspace served
constexpr int kNoAllocBlocks = 1024;           // reduction blocks (grid-stride)
constexpr int kNoAllocThreads = 256;
// doubles: H u [max rows], diagonal [max rows], 2 partial-sum rows, 4 scalars
constexpr int64_t kNoAllocDoubles = 2 * kNoAllocMaxRows + 2 * kNoAllocBlocks + 4;

__device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

std::mutex g_addr_mu;
double *g_addr[64] = {nullptr};  // device address of g_noalloc_scratch per device

double *scratch_address(int device) {
    if (device < 0 || device >= 64) fail(QSD_ERR_INVALID_ARG, "rayleigh_quotient_noalloc: device index above 63");
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            fail(QSD_ERR_CUDA, std::string("rayleigh_quotient_noalloc: cudaGetSymbolAddress failed: ") +
                                   cudaGetErrorString(e));
        g_addr[device] = static_cast<double *>(p);
    }
    return g_addr[device];
}

__device__ double nb_block_sum(double v) {
    __shared__ double sh[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x < 32) {
        r = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    }
    __syncthreads();
    return r;
}

// part_a[b] = sum u*hu, part_b[b] = sum u*u over the block's grid-stride rows
__global__ void k_nb_dots(const double *__restrict__ u, const double *__restrict__ hu, int64_t D, double *part_a,
                          double *part_b) {
    double a = 0.0, b = 0.0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < D; r += (int64_t)gridDim.x * blockDim.x) {
        a = fma(u[r], hu[r], a);
        b = fma(u[r], u[r], b);
    }
    a = nb_block_sum(a);
    b = nb_block_sum(b);
    if (threadIdx.x == 0) {
        part_a[blockIdx.x] = a;
        part_b[blockIdx.x] = b;
    }
}

// part_a[b] = sum (hu - theta u)^2, theta = sc[0] / sc[1]
__global__ void k_nb_resid(const double *__restrict__ u, const double *__restrict__ hu, int64_t D,
                           const double *__restrict__ sc, double *part_a) {
    const double theta = sc[0] / sc[1];
    double a = 0.0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < D; r += (int64_t)gridDim.x * blockDim.x) {
        const double d = hu[r] - theta * u[r];
        a = fma(d, d, a);
    }
    a = nb_block_sum(a);
    if (threadIdx.x == 0) part_a[blockIdx.x] = a;
}

// one block: sc[first + i] = sum of part_i (fixed order), i < n
__global__ void k_nb_finish(const double *__restrict__ part_a, const double *__restrict__ part_b, int nb, double *sc,
                            int first) {
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        a += part_a[i];
        if (part_b) b += part_b[i];
    }
    a = nb_block_sum(a);
    b = nb_block_sum(b);
    if (threadIdx.x == 0) {
        sc[first] = a;
        if (part_b) sc[first + 1] = b;
    }
}

}  // namespace

}  // namespace qsd

using namespace qsd;

extern "C" int qsd_rayleigh_quotient_noalloc(qsd_ctx ctx, qsd_op op, qsd_sub sub, const double *u, double *out) {
    if (!ctx) return QSD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    try {
        if (!op || !sub || op->ctx != ctx || sub->ctx != ctx || op->n_qubits != sub->n_qubits)
            fail(QSD_ERR_INVALID_ARG, "qsd_rayleigh_quotient_noalloc: bad operator or subspace");
        if (!u || !out || sub->D == 0) fail(QSD_ERR_INVALID_ARG, "qsd_rayleigh_quotient_noalloc: bad arguments");
        if (sub->D > kNoAllocMaxRows)
            fail(QSD_ERR_CAPACITY, "qsd_rayleigh_quotient_noalloc: subspace has " + std::to_string(sub->D) +
                                       " rows; this entry point serves at most " + std::to_string(kNoAllocMaxRows) +
                                       " (use qsd_rayleigh_quotient)");
        if (!op->info.is_real)
            fail(QSD_ERR_COMPLEX_UNSUPPORTED, "qsd_rayleigh_quotient_noalloc: complex operator");
        QSD_CUDA(cudaSetDevice(ctx->device));
        double *base = scratch_address(ctx->device);
        double *hu = base, *diag = base + kNoAllocMaxRows;
        double *part_a = base + 2 * kNoAllocMaxRows, *part_b = part_a + kNoAllocBlocks;
        double *sc = part_b + kNoAllocBlocks;
        cudaStream_t s = ctx->stream;
        const int64_t D = sub->D;
        const int nb = (int)std::min<int64_t>(kNoAllocBlocks, (D + kNoAllocThreads - 1) / kNoAllocThreads);
        // every value below is written before it is read: nothing to clear
        compute_diagonal(ctx, op, sub, diag);
        apply_H(ctx, op, sub, diag, QSD_FP64, 1, u, hu, s, false, false);
        k_nb_dots<<<nb, kNoAllocThreads, 0, s>>>(u, hu, D, part_a, part_b);
        k_nb_finish<<<1, kNoAllocThreads, 0, s>>>(part_a, part_b, nb, sc, 0);  // sc[0] = u.Hu, sc[1] = u.u
        k_nb_resid<<<nb, kNoAllocThreads, 0, s>>>(u, hu, D, sc, part_a);
        k_nb_finish<<<1, kNoAllocThreads, 0, s>>>(part_a, nullptr, nb, sc, 2);   // sc[2] = |Hu - theta u|^2
        QSD_LAUNCH_CHECK();
        double h[3];
        QSD_CUDA(cudaMemcpyAsync(h, sc, 24, cudaMemcpyDeviceToHost, s));
        QSD_CUDA(cudaStreamSynchronize(s));
        if (!(h[1] > 0.0)) fail(QSD_ERR_INVALID_ARG, "qsd_rayleigh_quotient_noalloc: u is zero");
        out[0] = h[0] / h[1];
        out[1] = std::sqrt(h[2]) / std::sqrt(h[1]);
        out[2] = h[1];
        return QSD_OK;
    } catch (const qsd::Error &e) {
        ctx->last_error = e.what();
        return e.code;
    } catch (const std::exception &e) {
        ctx->last_error = e.what();
        return QSD_ERR_INTERNAL;
    }
}
