// Warp-per-row product over a sector-factored product subspace (included by
// the apply_fac_inst.cu units).
//
// Row r = ib |A| + ia holds the string (a, b) = (A[ia], B[ib]).  For every
// shape of the operator's ladder terms -- (dOcc, dEmp) changes in sector 0
// and in sector 1 (see excite.cuh) -- the columns the row can reach inside S
// are the products of ia's neighbours of the sector-0 type and ib's
// neighbours of the sector-1 type (a type (0, 0) keeps the half).  The lanes
// split the concatenation of these products over all shapes; each candidate
// column (a', b') gives the flip mask F = (a ^ a', b ^ b'), whose group the
// dense rank index returns (one load; -1: no group has that mask), and the
// group's matrix element at the row (ladder-integer term range, projector
// tests, Jordan-Wigner signs: the same evaluation as every other path).  A
// nonzero element is multiplied by x at column ib' |A| + ia': no lookup.
// Groups outside the excitation index are scanned per row with a lookup.
// Each lane accumulates its candidates in a fixed order and the warp reduces
// with shuffles: the result is deterministic.
#pragma once

#include "excite.cuh"

namespace qsd {

struct FacParams {
    const uint64_t *A, *B;        // distinct halves
    const uint32_t *ptrA, *ptrB;  // [8 n + 1] neighbour list starts by (string, type)
    const uint32_t *nbrA, *nbrB;  // neighbour indices
    uint32_t nA, nB;
    int split;
};

// Rank of the set of bits of F (positions below 64) in the combinatorial
// number system: sum over the ascending positions p_1 < p_2 < ... of
// C(p_j, j).  F has at most four bits.
__device__ __forceinline__ uint32_t bits_rank(uint64_t F, const uint32_t (*binom)[64]) {
    uint32_t r = 0;
    int j = 1;
    while (F) {
        const int p = __ffsll((long long)F) - 1;
        r += binom[j][p];
        F &= F - 1;
        ++j;
    }
    return r;
}

// Neighbour type of (dOcc, dEmp) in the low (sector 0) or high (sector 1)
// fields of a shape; -1 for (0, 0): the half is kept.
__device__ __forceinline__ int shape_type(uint32_t occ, uint32_t emp) {
    return (occ | emp) ? (int)(3 * occ + emp) - 1 : -1;
}

constexpr uint32_t kKeepHalf = 0xffffffffu;

template <int W, int KB, int PREC>
__global__ void __launch_bounds__(256) k_apply_fac(const ApplyParams p, const ExcParams e, const FacParams f) {
    using TIO = typename std::conditional<PREC == QSD_FP64, double, float>::type;
    __shared__ uint32_t binom[5][64];
    __shared__ uint32_t pre[8][kMaxShapes + 1];  // per warp: first candidate of each shape
    __shared__ uint32_t sa[8][kMaxShapes], sb[8][kMaxShapes], lb[8][kMaxShapes];
    for (int i = threadIdx.x; i < 5 * 64; i += blockDim.x) {
        const int j = i / 64, x = i % 64;
        uint64_t c = 1;
        for (int t = 0; t < j; ++t) c = c * (uint64_t)(x - t) / (uint64_t)(t + 1);
        binom[j][x] = x >= j ? (uint32_t)c : 0u;
    }
    __syncthreads();
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= p.D) return;  // warp-uniform
    const uint32_t ib = (uint32_t)(row / f.nA), ia = (uint32_t)(row - (int64_t)ib * f.nA);
    uint64_t key[W];
#pragma unroll
    for (int w = 0; w < W; ++w) key[w] = __ldg(p.keys + (size_t)w * p.D + row);
    const uint64_t a = __ldg(f.A + ia), b = __ldg(f.B + ib);
    // lane s < n_shapes: the candidate lists of shape s and their product size
    uint32_t cnt = 0;
    if (lane < e.n_shapes) {
        const uint32_t sh = e.shapes[lane];
        const int tA = shape_type(sh & 15u, (sh >> 4) & 15u), tB = shape_type((sh >> 8) & 15u, (sh >> 12) & 15u);
        uint32_t s0 = kKeepHalf, l0 = 1, s1 = kKeepHalf, l1 = 1;
        if (tA >= 0) {
            s0 = __ldg(f.ptrA + 8 * (size_t)ia + tA);
            l0 = __ldg(f.ptrA + 8 * (size_t)ia + tA + 1) - s0;
        }
        if (tB >= 0) {
            s1 = __ldg(f.ptrB + 8 * (size_t)ib + tB);
            l1 = __ldg(f.ptrB + 8 * (size_t)ib + tB + 1) - s1;
        }
        sa[wib][lane] = s0;
        sb[wib][lane] = s1;
        lb[wib][lane] = l1;
        cnt = l0 * l1;
    }
    // inclusive scan of the counts over the shapes
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane < e.n_shapes) pre[wib][lane + 1] = incl;
    if (lane == 0) pre[wib][0] = 0;
    __syncwarp();
    const uint32_t total = pre[wib][e.n_shapes];

    const TIO *__restrict__ x = static_cast<const TIO *>(p.x);
    double acc[KB];
    float as[KB], ae[KB];
#pragma unroll
    for (int j = 0; j < KB; ++j) { acc[j] = 0.0; as[j] = 0.f; ae[j] = 0.f; }

    auto add = [&](double amp, uint64_t col) {
        const TIO *xc = x + col * p.ld + p.col0;
        if (PREC == QSD_FP32_DOT2) {
            const float h = (float)amp, l = (float)(amp - (double)h);
#pragma unroll
            for (int j = 0; j < KB; ++j) dot2_add(as[j], ae[j], h, l, (float)__ldg(xc + j));
        } else {
#pragma unroll
            for (int j = 0; j < KB; ++j) acc[j] = fma(amp, (double)__ldg(xc + j), acc[j]);
        }
    };

    int si = 0;
    for (uint32_t t = lane; t < total; t += 32) {
        while (pre[wib][si + 1] <= t) ++si;  // t ascends: the shape only moves forward
        const uint32_t u = t - pre[wib][si];
        const uint32_t l1 = lb[wib][si];
        const uint32_t ua = u / l1, ub = u - ua * l1;
        const uint32_t s0 = sa[wib][si], s1 = sb[wib][si];
        const uint32_t ia2 = s0 == kKeepHalf ? ia : __ldg(f.nbrA + s0 + ua);
        const uint32_t ib2 = s1 == kKeepHalf ? ib : __ldg(f.nbrB + s1 + ub);
        const uint64_t Fa = a ^ __ldg(f.A + ia2), Fb = b ^ __ldg(f.B + ib2);
        const uint32_t r0 = bits_rank(Fa, binom), r1 = bits_rank(Fb, binom);
        const int32_t g = __ldg(e.dense + e.dbase[si] + r0 * e.dstride[si] + r1);
        if (g < 0) continue;
        const double amp = scan_amp<W>(p, g, key);
        if (((uint64_t)__double_as_longlong(amp) << 1) == 0ull) continue;
        add(amp, (uint64_t)ib2 * f.nA + ia2);
    }
    // groups outside the excitation index: evaluated and looked up per row
    if (e.n_rest > 0) {
        const uint64_t hr = key_hash<W>(key, p.nib);
        for (int64_t i = lane; i < e.n_rest; i += 32) {
            const int64_t g = __ldg(e.rest_gid + i);
            const double amp = scan_amp<W>(p, g, key);
            if (((uint64_t)__double_as_longlong(amp) << 1) == 0ull) continue;
            uint64_t c[W];
#pragma unroll
            for (int w = 0; w < W; ++w) c[w] = key[w] ^ __ldg(p.gF + (size_t)w * p.G + g);
            const int64_t idx = probe<W>(c, hr ^ __ldg(&p.grec[g].hF), p.hv, p.err);
            if (idx >= 0) add(amp, (uint64_t)idx);
        }
    }
#pragma unroll
    for (int j = 0; j < KB; ++j) {
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            if (PREC == QSD_FP32_DOT2) {
                const float s2 = __shfl_xor_sync(0xffffffffu, as[j], o);
                const float e2 = __shfl_xor_sync(0xffffffffu, ae[j], o);
                dot2_merge(as[j], ae[j], s2, e2);
            } else {
                acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
            }
        }
    }
    if (lane == 0) {
        const double d = __ldg(p.diag + row);
        const TIO *xr = x + row * p.ld + p.col0;
        TIO *yr = static_cast<TIO *>(p.y) + row * p.ld + p.col0;
        if (PREC == QSD_FP32_DOT2) {
            const float dh = (float)d, dl = (float)(d - (double)dh);
#pragma unroll
            for (int j = 0; j < KB; ++j) {
                dot2_add(as[j], ae[j], dh, dl, (float)__ldg(xr + j));
                yr[j] = (TIO)(as[j] + ae[j]);
            }
        } else {
#pragma unroll
            for (int j = 0; j < KB; ++j) yr[j] = (TIO)fma(d, (double)__ldg(xr + j), acc[j]);
        }
    }
}

// Launch the factored product for precision mode PREC (W <= 2).
template <int PREC>
void launch_apply_fac(const ApplyParams &p, const ExcParams &e, const FacParams &f, int W, int KB, cudaStream_t s);

}  // namespace qsd
