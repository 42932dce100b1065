// The matrix-free product y = H_S x (Methods, "Matrix evaluation").
//
// Gather form, one output row per R consecutive lanes (R = 1: a lane per
// row with every group broadcast to the warp; R = 32: a warp per row with
// the groups split over lanes and a shuffle reduction).  Per row and group:
//   1. ladder groups: the row's bits at the group's flipped qubits form the
//      ladder integer, whose int_ptrs entry is the only term range that can
//      be nonzero; an empty range skips the group with no lookup (Fig. 3b);
//      other groups scan their term range;
//   2. each candidate term passes its projector test (r & P) == V and adds
//      phi (-1)^popc(r & Z) to the group's matrix element;
//   3. if any term passed, the column r xor F is looked up once for the
//      whole group (property 3: the terms of a group share the column);
//   4. the element times x[column] is accumulated in FP64.
// Finally y[r] = d[r] x[r] + sum, rounded once to the storage type.
#pragma once

#include "qsd_internal.cuh"

namespace qsd {

struct ApplyParams {
    const uint64_t *keys;   // [W][D]
    int64_t D;
    const uint64_t *slots;
    uint64_t bmask;
    const uint64_t *nib;
    int64_t G;
    const uint64_t *gF;      // [W][G]
    const uint64_t *ghash;   // [G]
    const int32_t *grange;   // [G+1]
    const uint8_t *gL;       // [G]
    const uint64_t *gpos;    // [G]
    const int32_t *gptr;     // [G][17]
    int64_t T;
    const uint64_t *tP, *tV, *tZ;  // [W][T]
    const double *tphi;      // [T]
    const uint8_t *tflag;    // [T]
    const double *diag;      // [D]
    const void *x;
    void *y;
    int64_t ld;              // row stride of x and y (= k)
    int64_t col0;            // first column handled by this launch
    uint32_t *err;
};

template <int W>
__device__ __forceinline__ uint64_t word_of(const uint64_t (&x)[W], int q) {
    uint64_t v = x[0];
#pragma unroll
    for (int w = 1; w < W; ++w)
        if ((q >> 6) == w) v = x[w];
    return v;
}

template <int W, int R, int KB, typename TIO>
__global__ void __launch_bounds__(256) k_apply(const ApplyParams p) {
    const int sub = threadIdx.x % R;
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / R;
    const bool active = row < p.D;
    const int64_t r = active ? row : p.D - 1;
    uint64_t key[W];
#pragma unroll
    for (int w = 0; w < W; ++w) key[w] = __ldg(p.keys + (size_t)w * p.D + r);
    const uint64_t hr = prehash<W>(key, p.nib);
    const TIO *__restrict__ x = static_cast<const TIO *>(p.x);
    double acc[KB];
#pragma unroll
    for (int j = 0; j < KB; ++j) acc[j] = 0.0;
    if (active) {
        for (int64_t g = sub; g < p.G; g += R) {
            int32_t b, e;
            const int L = __ldg(p.gL + g);
            if (L) {
                const uint64_t pos = __ldg(p.gpos + g);
                int l = 0;
                for (int i = 0; i < L; ++i) {
                    const int q = (int)((pos >> (16 * i)) & 0xffff);
                    l |= (int)((word_of<W>(key, q) >> (q & 63)) & 1) << i;
                }
                b = __ldg(p.gptr + g * 17 + l);
                e = __ldg(p.gptr + g * 17 + l + 1);
            } else {
                b = __ldg(p.grange + g);
                e = __ldg(p.grange + g + 1);
            }
            if (b >= e) continue;
            double amp = 0.0;
            bool any = false;
            for (int32_t t = b; t < e; ++t) {
                const uint8_t f = __ldg(p.tflag + t);
                bool ok = true;
                if (f & 1) {
#pragma unroll
                    for (int w = 0; w < W; ++w)
                        ok &= (key[w] & __ldg(p.tP + (size_t)w * p.T + t)) == __ldg(p.tV + (size_t)w * p.T + t);
                }
                if (!ok) continue;
                any = true;
                double ph = __ldg(p.tphi + t);
                if (f & 2) {
                    int par = 0;
#pragma unroll
                    for (int w = 0; w < W; ++w) par ^= __popcll(key[w] & __ldg(p.tZ + (size_t)w * p.T + t));
                    if (par & 1) ph = -ph;
                }
                amp += ph;
            }
            if (!any) continue;
            uint64_t c[W];
#pragma unroll
            for (int w = 0; w < W; ++w) c[w] = key[w] ^ __ldg(p.gF + (size_t)w * p.G + g);
            const int64_t idx = probe<W>(c, hr ^ __ldg(p.ghash + g), p.slots, p.keys, p.D, p.bmask, p.err);
            if (idx < 0) continue;
            const TIO *xc = x + idx * p.ld + p.col0;
#pragma unroll
            for (int j = 0; j < KB; ++j) acc[j] = fma(amp, (double)__ldg(xc + j), acc[j]);
        }
    }
    if (R > 1) {
#pragma unroll
        for (int j = 0; j < KB; ++j)
#pragma unroll
            for (int o = R / 2; o >= 1; o >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
    }
    if (active && sub == 0) {
        const double d = __ldg(p.diag + row);
        const TIO *xr = x + row * p.ld + p.col0;
        TIO *yr = static_cast<TIO *>(p.y) + row * p.ld + p.col0;
#pragma unroll
        for (int j = 0; j < KB; ++j) yr[j] = (TIO)fma(d, (double)__ldg(xr + j), acc[j]);
    }
}

// Run-time W (W > kMaxWordsStatic): a lane per row, keys in local memory.
template <int KB, typename TIO>
__global__ void __launch_bounds__(256) k_apply_dyn(const ApplyParams p, int W) {
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= p.D) return;
    uint64_t key[kMaxWordsDyn], c[kMaxWordsDyn];
    for (int w = 0; w < W; ++w) key[w] = p.keys[(size_t)w * p.D + row];
    const uint64_t hr = prehash_dyn(key, W, p.nib);
    const TIO *__restrict__ x = static_cast<const TIO *>(p.x);
    double acc[KB];
#pragma unroll
    for (int j = 0; j < KB; ++j) acc[j] = 0.0;
    for (int64_t g = 0; g < p.G; ++g) {
        int32_t b, e;
        const int L = p.gL[g];
        if (L) {
            const uint64_t pos = p.gpos[g];
            int l = 0;
            for (int i = 0; i < L; ++i) {
                const int q = (int)((pos >> (16 * i)) & 0xffff);
                l |= (int)((key[q >> 6] >> (q & 63)) & 1) << i;
            }
            b = p.gptr[g * 17 + l];
            e = p.gptr[g * 17 + l + 1];
        } else {
            b = p.grange[g];
            e = p.grange[g + 1];
        }
        double amp = 0.0;
        bool any = false;
        for (int32_t t = b; t < e; ++t) {
            bool ok = true;
            int par = 0;
            for (int w = 0; w < W; ++w) {
                ok &= (key[w] & p.tP[(size_t)w * p.T + t]) == p.tV[(size_t)w * p.T + t];
                par ^= __popcll(key[w] & p.tZ[(size_t)w * p.T + t]);
            }
            if (!ok) continue;
            any = true;
            amp += (par & 1) ? -p.tphi[t] : p.tphi[t];
        }
        if (!any) continue;
        for (int w = 0; w < W; ++w) c[w] = key[w] ^ p.gF[(size_t)w * p.G + g];
        const int64_t idx = probe_dyn(c, W, hr ^ p.ghash[g], p.slots, p.keys, p.D, p.bmask, p.err);
        if (idx < 0) continue;
        const TIO *xc = x + idx * p.ld + p.col0;
#pragma unroll
        for (int j = 0; j < KB; ++j) acc[j] = fma(amp, (double)xc[j], acc[j]);
    }
    const double d = p.diag[row];
    const TIO *xr = x + row * p.ld + p.col0;
    TIO *yr = static_cast<TIO *>(p.y) + row * p.ld + p.col0;
#pragma unroll
    for (int j = 0; j < KB; ++j) yr[j] = (TIO)fma(d, (double)xr[j], acc[j]);
}

// Launch one (W, R, KB) variant for storage type TIO.
template <typename TIO>
void launch_apply(const ApplyParams &p, int W, int R, int KB, cudaStream_t s);

}  // namespace qsd
