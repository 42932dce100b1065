// Warp-per-row excitation product (included by the apply_exc_p*.cu units).
//
// Per row (one warp): the occupied and empty qubits of each sector are listed
// in shared memory; for every shape of the operator's ladder terms, the lanes
// split the product of combinations "k occupied of sector 0 x l empty of
// sector 0 x ..." (k, l <= 2).  Each candidate flip mask F is looked up in the
// group hash table; a group found contributes its matrix element at the row
// (ladder-integer term range, projector tests, Jordan-Wigner signs), and a
// nonzero element costs one subspace lookup of r xor F.  The row's pattern on
// F fixes the shape, so each (row, group) pair is visited at most once.
// Groups outside the index (letters X, Y, or more than two excitations per
// sector) are scanned by the lanes.  Lanes accumulate their own candidates in
// a fixed order and the warp reduces with shuffles: deterministic.
#pragma once

#include "excite.cuh"

namespace qsd {

__device__ __forceinline__ int choose(int m, int k) { return k == 0 ? 1 : (k == 1 ? m : m * (m - 1) / 2); }

// The i-th k-subset (k <= 2) of list[0..m) as qubit positions.
__device__ __forceinline__ void unrank(int i, int k, const uint8_t *list, int &q0, int &q1) {
    if (k == 1) {
        q0 = list[i];
    } else if (k == 2) {
        int y = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)i)) * 0.5f);
        while (y * (y - 1) / 2 > i) --y;
        while ((y + 1) * y / 2 <= i) ++y;
        const int x = i - y * (y - 1) / 2;
        q0 = list[x];
        q1 = list[y];
    }
}

// Rank of a set of at most four positions (two picks of each of two lists,
// -1 = none) in the combinatorial number system: sum over its elements x of
// C(x, j) with j the element's 1-based place in ascending order (as unsigned,
// -1 is never below an element).
template <int W>
__device__ __forceinline__ uint32_t sector_rank(int a0, int a1, int b0, int b1, const uint32_t (*binom)[64 * W]) {
    const int v[4] = {a0, a1, b0, b1};
    uint32_t r = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (v[i] < 0) continue;
        int j = 1;
#pragma unroll
        for (int m = 0; m < 4; ++m) j += (m != i && (unsigned)v[m] < (unsigned)v[i]) ? 1 : 0;
        r += binom[j][v[i]];
    }
    return r;
}

template <int W>
__device__ __forceinline__ void set_bit(uint64_t (&F)[W], int q) {
#pragma unroll
    for (int w = 0; w < W; ++w)
        if ((q >> 6) == w) F[w] |= 1ull << (q & 63);
}

template <int W, int KB, int PREC>
__global__ void __launch_bounds__(256) k_apply_exc(const ApplyParams p, const ExcParams e) {
    using TIO = typename std::conditional<PREC == QSD_FP64, double, float>::type;
    __shared__ uint8_t lists[8][4][64 * W];
    __shared__ int cnt[8][4];
    __shared__ uint64_t bh[64 * W];  // h of each single qubit (the hash is linear)
    __shared__ uint32_t binom[5][64 * W];  // C(x, j) for the rank index
    for (int q = threadIdx.x; q < 64 * W; q += blockDim.x) bh[q] = bit_hash(q, p.nib);
    if (e.dense) {
        for (int i = threadIdx.x; i < 5 * 64 * W; i += blockDim.x) {
            const int j = i / (64 * W), x = i % (64 * W);
            uint64_t c = 1;
            for (int t = 0; t < j; ++t) c = c * (uint64_t)(x - t) / (uint64_t)(t + 1);
            binom[j][x] = x >= j ? (uint32_t)c : 0u;
        }
    }
    __syncthreads();
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= p.D) return;  // warp-uniform
    uint64_t key[W];
#pragma unroll
    for (int w = 0; w < W; ++w) key[w] = __ldg(p.keys + (size_t)w * p.D + row);
    const uint64_t hr = key_hash<W>(key, p.nib);
    // occupied / empty lists per sector
    for (int sct = 0; sct < 2; ++sct) {
        const int lo = sct ? e.split : 0, hi = sct ? e.n_qubits : e.split;
        int no = 0, nv = 0;
        for (int base = lo; base < hi; base += 32) {
            const int q = base + lane;
            const bool in = q < hi;
            const bool occ = in && ((word_of<W>(key, q) >> (q & 63)) & 1);
            const uint32_t bo = __ballot_sync(0xffffffffu, occ), bv = __ballot_sync(0xffffffffu, in && !occ);
            const uint32_t lt = (1u << lane) - 1u;
            if (occ) lists[wib][2 * sct][no + __popc(bo & lt)] = (uint8_t)q;
            if (in && !occ) lists[wib][2 * sct + 1][nv + __popc(bv & lt)] = (uint8_t)q;
            no += __popc(bo);
            nv += __popc(bv);
        }
        if (lane == 0) {
            cnt[wib][2 * sct] = no;
            cnt[wib][2 * sct + 1] = nv;
        }
    }
    __syncwarp();
    const TIO *__restrict__ x = static_cast<const TIO *>(p.x);
    double acc[KB];
    float as[KB], ae[KB];
#pragma unroll
    for (int j = 0; j < KB; ++j) { acc[j] = 0.0; as[j] = 0.f; ae[j] = 0.f; }

    auto contribute = [&](double amp, const uint64_t (&F)[W], uint64_t hF) {
        uint64_t c[W];
#pragma unroll
        for (int w = 0; w < W; ++w) c[w] = key[w] ^ F[w];
        const int64_t idx = probe<W>(c, hr ^ hF, p.hv, p.err);
        if (idx < 0) return;
        const TIO *xc = x + idx * p.ld + p.col0;
        if (PREC == QSD_FP32_DOT2) {
            const float h = (float)amp, l = (float)(amp - (double)h);
#pragma unroll
            for (int j = 0; j < KB; ++j) dot2_add(as[j], ae[j], h, l, (float)__ldg(xc + j));
        } else {
#pragma unroll
            for (int j = 0; j < KB; ++j) acc[j] = fma(amp, (double)__ldg(xc + j), acc[j]);
        }
    };

    for (int si = 0; si < e.n_shapes; ++si) {
        const uint32_t sh = e.shapes[si];
        const int k[4] = {(int)(sh & 15), (int)((sh >> 4) & 15), (int)((sh >> 8) & 15), (int)((sh >> 12) & 15)};
        int f[4];
        int64_t N = 1;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            f[i] = choose(cnt[wib][i], k[i]);
            N *= f[i];
        }
        // candidate t of the shape: mixed-radix digits (one per list) by
        // division, in 32-bit arithmetic whenever the count allows
        auto candidate = [&](auto t) {
            using I = decltype(t);
            I rest = t;
            uint64_t F[W];
#pragma unroll
            for (int w = 0; w < W; ++w) F[w] = 0;
            uint64_t hF = 0;  // h(F) by linearity: the xor of its bits' hashes
            int qs[4][2];     // the picks of each list (-1: none), positions within the sector
#pragma unroll
            for (int i = 3; i >= 0; --i) {
                const I fi = (I)f[i];
                const I qt = rest / fi;
                const int id = (int)(rest - qt * fi);
                rest = qt;
                int q0 = -1, q1 = -1;
                unrank(id, k[i], lists[wib][i], q0, q1);
                const int off = i >= 2 ? e.split : 0;
                qs[i][0] = q0 >= 0 ? q0 - off : -1;
                qs[i][1] = q1 >= 0 ? q1 - off : -1;
                if (q0 >= 0) {
                    set_bit<W>(F, q0);
                    hF ^= bh[q0];
                }
                if (q1 >= 0) {
                    set_bit<W>(F, q1);
                    hF ^= bh[q1];
                }
            }
            int64_t g;
            if (e.dense) {
                const uint32_t r0 = sector_rank<W>(qs[0][0], qs[0][1], qs[1][0], qs[1][1], binom);
                const uint32_t r1 = sector_rank<W>(qs[2][0], qs[2][1], qs[3][0], qs[3][1], binom);
                g = __ldg(e.dense + e.dbase[si] + r0 * e.dstride[si] + r1);
                if (g < 0) return;
            } else {
                const int64_t ge = probe<W>(F, hF, e.ght, p.err);
                if (ge < 0) return;
                g = __ldg(e.exc_gid + ge);
            }
            const double amp = scan_amp<W>(p, g, key);
            if (((uint64_t)__double_as_longlong(amp) << 1) == 0ull) return;
            contribute(amp, F, hF);
        };
        if (N <= (int64_t)0xffffffffLL) {
            for (uint32_t t = lane; t < (uint32_t)N; t += 32) candidate(t);
        } else {
            for (int64_t t = lane; t < N; t += 32) candidate(t);
        }
    }
    for (int64_t i = lane; i < e.n_rest; i += 32) {
        const int64_t g = __ldg(e.rest_gid + i);
        const double amp = scan_amp<W>(p, g, key);
        if (((uint64_t)__double_as_longlong(amp) << 1) == 0ull) continue;
        uint64_t F[W];
        F[0] = __ldg(p.gF + g);
#pragma unroll
        for (int w = 1; w < W; ++w) F[w] = __ldg(p.gF + (size_t)w * p.G + g);
        contribute(amp, F, __ldg(&p.grec[g].hF));
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

}  // namespace qsd
