// Filter/verify product for operators whose groups are all table groups
// (every term tests and signs only qubits of a support of <= 5, e.g. all
// spin models), one lane per row, rows in the subspace's hash order, one
// right-hand side (included by the apply_fv_inst.cu units).
//
// The per-row group loop of the gather product (Methods, "Matrix evaluation")
// is split in two passes so that the rare work of a lookup runs at full warp
// width:
//   filter  the warp walks the groups together (group records and amplitude
//           tables staged in shared memory once per block); each lane takes
//           its row's pattern on the group's support, skips a zero element
//           (the paper's rejection of null terms before the query), and tests
//           the bit of h(r xor F) in the subspace's occupancy filter (128 bits
//           per bucket, at most 1/64 set: the paper's occupancy bit-set).  A
//           clear bit is a miss -- the common case -- and costs nothing more.
//           Otherwise (row, group, bucket, tag) goes to a per-warp ring of
//           candidates in shared memory.
//   verify  whenever 32 candidates are queued, each lane takes one: the
//           bucket's tags, the owner's key (by shuffle) xor F, the row
//           indices of the matching slots, the full-key check, x of the found
//           column, and the probe's continuation into the next buckets when
//           the bucket overflowed.  The found (element, x) pairs go back to
//           their owners in queue order by shuffles.
// Candidates enter the ring in group order and leave it in that order, so
// each row accumulates its elements in group order with the same operations
// as the one-pass scan: the result is bitwise that of QSD_PATH_SCAN_HASH.
// The grid is persistent (the resident blocks of every SM) so that the
// staging is paid once per block; blocks take 256-row tiles in a grid-stride
// loop.
#pragma once

#include "apply_kernel.cuh"

namespace qsd {

constexpr int kFvMaxGroups = 1024;  // group records staged per block (G < 2^18 for the meta word)
constexpr int kFvMaxAmps = 2048;    // amplitudes staged per block (index < 2^24)
constexpr int kFvRing = 64;         // candidates per warp (at most 31 + 32 queued)
constexpr int kFvThreads = 256;
constexpr int kFvWarps = kFvThreads / 32;
constexpr int kFvU = 4;             // groups per filter batch (bucket loads in flight per lane)
constexpr int kFvWideX = 3;         // internal mode: the FP32-mixed block on an FP64 copy of x

__host__ __device__ inline int64_t fv_padded_groups(int64_t G) { return (G + kFvU - 1) / kFvU * kFvU; }

// Shared memory: per (padded) group a 16-byte record {high word of h(F), low
// byte of h(F), nonzero-pattern mask, first amplitude} and its 8-byte support
// (qubits, 12 bits each); the amplitudes (8 bytes each: FP64, or the FP32
// (hi, lo) pair of DOT2); then per warp a ring of kFvRing candidates as three
// uint32 arrays: bucket; meta = owner lane (bits 0-4), group (bits 14-31);
// amplitude index (bits 0-23) and tag (bits 24-31); and per warp the
// delivery area of a verify batch: the found elements and x values by queue
// slot (8 bytes each) and each owner lane's mask of its found slots.  Padding
// groups have an empty mask.
constexpr int kFvDeliverBytes = 32 * 8 * 2 + 32 * 4;
inline size_t fv_smem_bytes(int64_t G, int64_t n_amp) {
    return (size_t)fv_padded_groups(G) * 24 + (size_t)n_amp * 8 + (size_t)kFvWarps * (kFvRing * 12 + kFvDeliverBytes);
}

struct FvRing {
    uint32_t *b, *m, *a;
    uint64_t *va, *vx;  // [32]: element (FP64, or the DOT2 (hi, lo) pair) and x of each found slot
    uint32_t *own;      // [32]: per owner lane, the mask of its found slots
};

// Verify the n (1..32) oldest queued candidates of the warp (one per lane)
// and deliver the found (element, x) pairs to their owner lanes in queue
// order; the same operations as the one-pass scan's accumulation.  Delivery:
// the verifier lanes of each owner (one __match_any_sync) post their mask to
// the owner, and every owner walks its own found slots in order, so the
// accumulation takes as many rounds as the busiest owner has candidates
// (one or two), not one round per candidate.
// KB > 1 (a block of columns): the verifier posts the found column's index
// and the owner gathers its KB values of x itself.
template <int W, int PREC, typename TIO, int KB>
__device__ __forceinline__ void fv_verify(const ApplyParams &p, const FvRing &q, uint32_t head, int n, int lane,
                                          const uint64_t (&key)[W], const double *amp, const float2 *ampf,
                                          const TIO *__restrict__ x, double (&acc)[KB], float (&as)[KB],
                                          float (&ae)[KB]) {
    const uint32_t slot = (head + (uint32_t)lane) & (kFvRing - 1);
    const bool mine = lane < n;
    const uint32_t meta = mine ? q.m[slot] : 0u;
    const uint32_t b = mine ? q.b[slot] : 0u;
    const uint32_t at = mine ? q.a[slot] : 0u;
    const int o = (int)(meta & 31u);
    // the bucket's tags (the filter read only its occupancy bit)
    const uint2 tb = mine ? __ldg(reinterpret_cast<const uint2 *>(p.hv.tags) + b) : make_uint2(0u, 0u);
    uint64_t c[W];
#pragma unroll
    for (int w = 0; w < W; ++w) c[w] = __shfl_sync(0xffffffffu, key[w], o);
    bool found = false;
    int64_t fidx = -1;  // KB > 1: the found column
    TIO xv = TIO(0);
    double a = 0.0;
    float ah = 0.f, al = 0.f;
    if (mine) {
        const int64_t g = (int64_t)(meta >> 14);
#pragma unroll
        for (int w = 0; w < W; ++w) c[w] ^= __ldg(p.gF + (size_t)w * p.G + g);
        int64_t idx = KB == 1 ? verify_matches_x<W, TIO>(p.hv, b, tag_match(tb, at >> 24), c, x + p.col0, p.ld, xv)
                              : verify_matches<W>(p.hv, b, tag_match(tb, at >> 24), c);
        if (idx < 0 && bucket_full(tb)) {
            idx = probe_from<W>(p.hv, b, at >> 24, c, p.err);
            if (KB == 1 && idx >= 0) xv = __ldg(x + idx * p.ld + p.col0);
        }
        found = idx >= 0;
        fidx = idx;
        const uint32_t ai = at & 0xffffffu;
        if (PREC == QSD_FP32_DOT2) {
            const float2 f = ampf[ai];
            ah = f.x;
            al = f.y;
        } else {
            a = amp[ai];
        }
    }
    // post: each owner's found slots (the lowest verifier lane of each owner
    // writes the owner's mask), the elements and x values by slot
    q.own[lane] = 0u;
    __syncwarp();
    const uint32_t grp = __match_any_sync(0xffffffffu, found ? (uint32_t)o : 32u + (uint32_t)lane);
    if (found) {
        if ((grp & ((1u << lane) - 1u)) == 0u) q.own[o] = grp;
        if (PREC == QSD_FP32_DOT2) {
            q.va[lane] = ((uint64_t)__float_as_uint(al) << 32) | __float_as_uint(ah);
        } else {
            q.va[lane] = (uint64_t)__double_as_longlong(a);
        }
        if (KB > 1) q.vx[lane] = (uint64_t)fidx;  // the owner gathers the block's columns
        else if (sizeof(TIO) == 8) q.vx[lane] = (uint64_t)__double_as_longlong((double)xv);
        else q.vx[lane] = (uint64_t)__float_as_uint((float)xv);
    }
    __syncwarp();
    // walk: every owner its own found slots, in queue order
    uint32_t mine_m = q.own[lane];
    while (__any_sync(0xffffffffu, mine_m != 0u)) {
        if (mine_m) {
            const int t = __ffs(mine_m) - 1;
            mine_m &= mine_m - 1u;
            const uint64_t ev = q.va[t], xb = q.vx[t];
            if (KB > 1) {
                const TIO *xc = x + (int64_t)xb * p.ld + p.col0;
                if (PREC == QSD_FP32_DOT2) {
                    const float h = __uint_as_float((uint32_t)ev), l = __uint_as_float((uint32_t)(ev >> 32));
#pragma unroll
                    for (int j = 0; j < KB; ++j) dot2_add(as[j], ae[j], h, l, (float)__ldg(xc + j));
                } else {
                    const double av = __longlong_as_double((long long)ev);
#pragma unroll
                    for (int j = 0; j < KB; ++j) acc[j] = fma(av, (double)__ldg(xc + j), acc[j]);
                }
            } else {
                const TIO xt = sizeof(TIO) == 8 ? (TIO)__longlong_as_double((long long)xb)
                                                : (TIO)__uint_as_float((uint32_t)xb);
                if (PREC == QSD_FP32_DOT2) {
                    dot2_add(as[0], ae[0], __uint_as_float((uint32_t)ev), __uint_as_float((uint32_t)(ev >> 32)),
                             (float)xt);
                } else {
                    acc[0] = fma(__longlong_as_double((long long)ev), (double)xt, acc[0]);
                }
            }
        }
    }
    __syncwarp();
}

// The row's bits on a group's support (nb <= 5 qubits, 12 bits each in pos).
template <int W>
__device__ __forceinline__ uint32_t fv_pattern(uint64_t pos, uint32_t nb, const uint64_t (&key)[W]) {
    uint32_t l = 0;
    for (uint32_t i = 0; i < nb; ++i) l |= bit_of<W>(key, (int)((pos >> (12 * i)) & 0xfff)) << i;
    return l;
}

// The row's bits on a two-qubit support whose qubits sit in bits 16-23 and
// 24-31 of y.
template <int W>
__device__ __forceinline__ uint32_t fv_pattern2(uint32_t y, const uint64_t (&key)[W]) {
    return bit_of<W>(key, (int)((y >> 16) & 0xffu)) | (bit_of<W>(key, (int)(y >> 24)) << 1);
}

// NB: the support size of every group when fixed (0: one constant element,
// e.g. X flips, so the filter reads no row bits; 2: e.g. flip-flop bonds),
// or -1 (read per group).  KB: columns of the block (1 or 16); the filter and
// verify passes are shared by the block's columns, every found column
// gathers KB values of x.
template <int W, int PREC, int NB, int KB = 1>
__global__ void __launch_bounds__(kFvThreads) k_apply_fv(const ApplyParams p, int n_amp, int64_t tiles) {
    // PREC, or kFvWideX: FP64 arithmetic on an exact FP64 copy of FP32 x with
    // FP32 y (bitwise the FP32-mixed product)
    constexpr int AP = PREC == kFvWideX ? QSD_FP64 : PREC;
    using TIO = typename std::conditional<AP == QSD_FP64, double, float>::type;  // x
    using TY = typename std::conditional<PREC == QSD_FP64, double, float>::type;  // y
    extern __shared__ __align__(16) unsigned char fv_smem[];
    const int G = (int)p.G;
    const int Gp = (int)fv_padded_groups(p.G);
    uint4 *recA = reinterpret_cast<uint4 *>(fv_smem);
    uint64_t *recB = reinterpret_cast<uint64_t *>(fv_smem + (size_t)Gp * 16);
    double *amp = reinterpret_cast<double *>(fv_smem + (size_t)Gp * 24);
    float2 *ampf = reinterpret_cast<float2 *>(amp);
    uint32_t *ring = reinterpret_cast<uint32_t *>(fv_smem + (size_t)Gp * 24 + (size_t)n_amp * 8);
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    FvRing q;
    q.b = ring + (size_t)wib * kFvRing * 3;
    q.m = q.b + kFvRing;
    q.a = q.m + kFvRing;
    unsigned char *dl = reinterpret_cast<unsigned char *>(ring + (size_t)kFvWarps * kFvRing * 3) +
                        (size_t)wib * kFvDeliverBytes;
    q.va = reinterpret_cast<uint64_t *>(dl);
    q.vx = q.va + 32;
    q.own = reinterpret_cast<uint32_t *>(q.vx + 32);

    for (int g = threadIdx.x; g < Gp; g += blockDim.x) {
        uint4 A = make_uint4(0u, 0u, 0u, 0u);
        uint64_t B = 0;
        if (g < G) {
            const ulonglong2 r0 = __ldg(reinterpret_cast<const ulonglong2 *>(p.grec + g));
            const uint4 r1 = __ldg(reinterpret_cast<const uint4 *>(p.grec + g) + 1);
            // y: tag byte, support size (bits 8-10), first two support qubits
            // (bits 16-23, 24-31; n <= 256)
            A = make_uint4((uint32_t)(r0.x >> 32),
                           ((uint32_t)r0.x & 0xffu) | ((r1.y & 7u) << 8) | (((uint32_t)r0.y & 0xffu) << 16) |
                               ((((uint32_t)(r0.y >> 12)) & 0xffu) << 24),
                           r1.z, r1.x);
            B = r0.y;
        }
        recA[g] = A;
        recB[g] = B;
    }
    if (AP == QSD_FP32_DOT2) {
        for (int i = threadIdx.x; i < n_amp; i += blockDim.x) ampf[i] = __ldg(p.ampf + i);
    } else {
        for (int i = threadIdx.x; i < n_amp; i += blockDim.x) amp[i] = __ldg(p.amp + i);
    }
    __syncthreads();

    const TIO *__restrict__ x = static_cast<const TIO *>(p.x);
    const uint32_t *__restrict__ occ = p.hv.occ;
    const uint32_t oshift = (uint32_t)p.hv.occ_shift;
    const uint32_t bshift = (uint32_t)p.hv.shift - 32u;
    const uint32_t lt = (1u << lane) - 1u;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t pos = tile * kFvThreads + threadIdx.x;
        const bool active = pos < p.D;
        const int64_t pc = active ? pos : p.D - 1;
        uint64_t key[W];
#pragma unroll
        for (int w = 0; w < W; ++w) key[w] = __ldg(p.hkeys + (size_t)w * p.D + pc);
        const uint64_t hr = __ldg(p.hhash + pc);
        const uint32_t hr_hi = (uint32_t)(hr >> 32), hr_lo = (uint32_t)hr & 0xffu;
        // an inactive lane (past the last row) needs no group: its mask bit
        // is taken from an empty pattern range
        const uint32_t live = active ? 0xffffffffu : 0u;
        double acc[KB];
        float as[KB], ae[KB];
#pragma unroll
        for (int j = 0; j < KB; ++j) {
            acc[j] = 0.0;
            as[j] = ae[j] = 0.f;
        }
        uint32_t head = 0, tail = 0;  // warp-uniform ring positions

        for (int g0 = 0; g0 < Gp; g0 += kFvU) {
            // phase 1: every group's filter word in flight (the word and the
            // bit position kept; bucket, tag, pattern and amplitude index are
            // recomputed for the rare candidates)
            uint32_t wd[kFvU], bit[kFvU];
            uint32_t needm = 0;
#pragma unroll
            for (int u = 0; u < kFvU; ++u) {
                const uint4 R = recA[g0 + u];
                uint32_t l = 0;
                if (NB == 2) l = fv_pattern2<W>(R.y, key);
                else if (NB < 0) l = fv_pattern<W>(recB[g0 + u], (R.y >> 8) & 7u, key);
                const uint32_t need = ((R.z & live) >> l) & 1u;
                const uint32_t bi = (hr_hi ^ R.x) >> oshift;
                bit[u] = bi & 31u;
                wd[u] = need ? __ldg(occ + (bi >> 5)) : 0u;
                needm |= need << u;
            }
            // phase 2: misses end here; candidates enter the ring in group order
#pragma unroll
            for (int u = 0; u < kFvU; ++u) {
                const bool cand = ((needm >> u) & (wd[u] >> bit[u])) & 1u;
                const uint32_t bal = __ballot_sync(0xffffffffu, cand);
                if (bal == 0u) continue;  // warp-uniform: every lookup of the group missed
                if (cand) {
                    const uint4 R = recA[g0 + u];
                    const uint32_t l = NB == 0 ? 0u
                                       : NB == 2 ? fv_pattern2<W>(R.y, key)
                                                 : fv_pattern<W>(recB[g0 + u], (R.y >> 8) & 7u, key);
                    const uint32_t t = (hr_lo ^ R.y) & 0xffu;
                    const uint32_t slot = (tail + (uint32_t)__popc(bal & lt)) & (kFvRing - 1);
                    q.b[slot] = (hr_hi ^ R.x) >> bshift;
                    q.m[slot] = (uint32_t)lane | ((uint32_t)(g0 + u) << 14);
                    q.a[slot] = (R.w + l) | ((t ? t : 1u) << 24);
                }
                tail += (uint32_t)__popc(bal);
                __syncwarp();
                if (tail - head >= 32u) {
                    fv_verify<W, AP, TIO, KB>(p, q, head, 32, lane, key, amp, ampf, x, acc, as, ae);
                    head += 32u;
                    __syncwarp();
                }
            }
        }
        __syncwarp();
        if (tail != head)
            fv_verify<W, AP, TIO, KB>(p, q, head, (int)(tail - head), lane, key, amp, ampf, x, acc, as, ae);
        __syncwarp();
        if (active) {
            const int64_t r = (int64_t)__ldg(p.hperm + pc);
            const double d = __ldg(p.diag + r);
            const TIO *xr = x + r * p.ld + p.col0;
            TY *yr = static_cast<TY *>(p.y) + r * p.ld + p.col0;
            if (AP == QSD_FP32_DOT2) {
                const float dh = (float)d, dl = (float)(d - (double)dh);
#pragma unroll
                for (int j = 0; j < KB; ++j) {
                    dot2_add(as[j], ae[j], dh, dl, (float)__ldg(xr + j));
                    yr[j] = (TY)(as[j] + ae[j]);
                }
            } else {
#pragma unroll
                for (int j = 0; j < KB; ++j) yr[j] = (TY)fma(d, (double)__ldg(xr + j), acc[j]);
            }
        }
    }
}

// Launch the filter/verify product for precision mode PREC (W <= 4, KB = 1
// or 16 columns, hash order, every group a table group, G <= kFvMaxGroups,
// n_amp <= kFvMaxAmps); nb: the support size of every group when fixed (0 or
// 2), else -1.
template <int PREC>
void launch_apply_fv(const ApplyParams &p, int n_amp, int W, int nb, int KB, int num_sms, cudaStream_t s);

}  // namespace qsd
