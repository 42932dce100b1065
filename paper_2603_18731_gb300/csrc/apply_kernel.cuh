// The matrix-free product y = H_S x (Methods, "Matrix evaluation").
//
// Gather form: R lanes own one output row (R = 1: a lane per row, every group
// broadcast to the warp; R = 8: the groups of a row split over 8 lanes and
// reduced by shuffles).  Per row and group:
//   1. table groups (every term tests and signs only bits inside a support
//      of <= 5 qubits, e.g. all spin models): the row's bits on the support
//      index a precomputed table of the group's matrix element, which is
//      exactly zero when no term survives -- the group is then skipped with
//      no lookup (the paper's rejection of null terms before the subspace
//      query);
//      scan groups (fermionic terms with Jordan-Wigner strings): the ladder
//      integer of the row selects the int_ptrs term range (Fig. 3b) and each
//      term passes its projector test and adds phi (-1)^popc(r & Z);
//   2. the column r xor F is looked up once for the whole group (property 3);
//   3. the element times x[column] is accumulated.
// Groups are processed U = 4 at a time: the four bucket loads are issued
// before any is inspected, so each lane keeps four lookups in flight.
//
// Accumulation: QSD_FP64 and QSD_FP32_MIXED accumulate in FP64 (DFMA);
// QSD_FP32_DOT2 accumulates FP32 products with error-free transformations
// (TwoProduct by FMA and TwoSum, Ogita-Rump-Oishi "Dot2", SIAM J. Sci.
// Comput. 2005): the sum is as accurate as one computed in twice the FP32
// precision and rounded once, with no FP64 instruction in the loop.
#pragma once

#include "qsd_internal.cuh"

namespace qsd {

constexpr int kTableBitsMax = 5;
constexpr uint32_t kGroupScan = 0x80u;
constexpr int kMsobShift = 16;         // GroupRec::info bits 16..27: most significant flipped qubit
constexpr uint32_t kMsobMask = 0xfffu;
constexpr uint32_t kNoTable = 0xffffffffu;

// Groups per batch (bucket loads in flight per lane) and the minimum resident
// blocks of 256 threads per SM asked of the compiler, per key width W, for the
// k = 1 kernels (measured on GB300: one-word keys run best at full occupancy
// with one lookup in flight per lane; four-word keys, whose rows hold more
// registers, with two lookups in flight at half occupancy).  k > 1 kernels
// keep two lookups in flight and their register budget.
template <int W, int KB> struct ApplyShape {
    static constexpr int U = (KB == 1 && W == 1) ? 1 : 2;
    static constexpr int MINB = KB == 1 ? (W == 1 ? 8 : 4) : 1;
};

// 32-byte group record, one per off-diagonal group
struct __align__(16) GroupRec {
    uint64_t hF;    // hash h of the flip mask F
    uint64_t pos;   // table groups: support qubits, 12 bits each, ascending
    uint32_t off;   // table groups: offset of the 2^nb amplitudes
    uint32_t info;  // bits 0..2: nb; kGroupScan: scan group; bits 16..27: MSOB
    uint32_t nzmask;  // table groups: bit l set iff the amplitude of pattern l is nonzero
    uint32_t pad;
};

struct ApplyParams {
    const uint64_t *keys;   // [W][D]
    int64_t D;
    HashView hv;
    const uint64_t *nib;
    int64_t G;
    const GroupRec *grec;    // [G]
    const double *amp;       // table amplitudes
    const float2 *ampf;      // the same split into FP32 (hi, lo)
    int64_t n_amp;           // number of table amplitudes
    int table_nb;            // support size shared by every group (0: constant elements), or -1
    const uint64_t *gF;      // [W][G]
    const int32_t *grange;   // [G+1]
    const uint8_t *gL;       // [G]
    const uint64_t *gpos;    // [G]
    const int32_t *gptr;     // [G][17]
    int64_t T;
    const uint64_t *tP, *tV, *tZ;  // [W][T]
    const double *tphi;      // [T]
    const uint8_t *tflag;    // [T]
    const double *diag;      // [D]
    const uint64_t *rhash;   // [D] hash h of each row
    const uint32_t *hperm;   // [D] hash order: row at each position
    const uint64_t *hkeys;   // [W][D] hash order: keys at the positions
    const uint64_t *hhash;   // [D] hash order: h at the positions
    const void *x;
    void *y;
    int64_t ld;              // row stride of x and y (= k)
    int64_t col0;            // first column handled by this launch
    uint32_t *err;
    int num_sms;
};

template <int W>
__device__ __forceinline__ uint64_t word_of(const uint64_t (&x)[W], int q) {
    uint64_t v = x[0];
#pragma unroll
    for (int w = 1; w < W; ++w)
        if ((q >> 6) == w) v = x[w];
    return v;
}

// Bit q of a multi-word key with 32-bit operations only (the word's high or
// low half, then a 32-bit shift).
template <int W>
__device__ __forceinline__ uint32_t bit_of(const uint64_t (&x)[W], int q) {
    const uint64_t v = word_of<W>(x, q);
    const uint32_t h = (q & 32) ? (uint32_t)(v >> 32) : (uint32_t)v;
    return (h >> (q & 31)) & 1u;
}

// a != 0 (either sign of zero counts as zero), on the two 32-bit halves.
__device__ __forceinline__ bool nonzero_f64(double a) {
    return ((uint32_t)(__double2hiint(a) & 0x7fffffff) | (uint32_t)__double2loint(a)) != 0u;
}

// Matrix element of a scan group at the row (0 when no term survives).
template <int W>
__device__ __noinline__ double scan_amp(const ApplyParams &p, int64_t g, const uint64_t (&key)[W]) {
    int32_t b, e;
    const int L = __ldg(p.gL + g);
    if (L) {
        const uint64_t pos = __ldg(p.gpos + g);
        int l = 0;
        for (int i = 0; i < L; ++i) {
            const int q = (int)((pos >> (16 * i)) & 0xffff);
            l |= (int)bit_of<W>(key, q) << i;
        }
        b = __ldg(p.gptr + g * 17 + l);
        e = __ldg(p.gptr + g * 17 + l + 1);
    } else {
        b = __ldg(p.grange + g);
        e = __ldg(p.grange + g + 1);
    }
    double amp = 0.0;
    for (int32_t t = b; t < e; ++t) {
        const uint8_t f = __ldg(p.tflag + t);
        bool ok = true;
        if (f & 1) {
#pragma unroll
            for (int w = 0; w < W; ++w)
                ok &= (key[w] & __ldg(p.tP + (size_t)w * p.T + t)) == __ldg(p.tV + (size_t)w * p.T + t);
        }
        if (!ok) continue;
        double ph = __ldg(p.tphi + t);
        if (f & 2) {
            int par = 0;
#pragma unroll
            for (int w = 0; w < W; ++w) par ^= __popcll(key[w] & __ldg(p.tZ + (size_t)w * p.T + t));
            if (par & 1) ph = -ph;
        }
        amp += ph;
    }
    return amp;
}

// The double of a float, exactly, by integer operations on the IEEE-754
// encodings: sign kept, 8-bit exponent rebiased by 1023 - 127 = 896, the 23
// mantissa bits moved up by 29 (a float's value fits a double exactly).
// Zeros map to zeros; subnormal, infinite and NaN inputs (exponent field 0
// with a nonzero mantissa, or 255) take the hardware conversion.  Cheaper
// than the conversion instruction where FP64 work is the bottleneck.
__device__ __forceinline__ double f32_to_f64(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t ex = (u >> 23) & 0xffu;
    const uint32_t sign_hi = u & 0x80000000u;
    if (ex - 1u < 254u) {  // normal: exponent 1..254
        const uint32_t hi = sign_hi | ((ex + 896u) << 20) | ((u & 0x7fffffu) >> 3);
        const uint32_t lo = u << 29;
        return __hiloint2double((int)hi, (int)lo);
    }
    if ((u & 0x7fffffffu) == 0u) return __hiloint2double((int)sign_hi, 0);
    return (double)f;
}

// Error-free accumulation of hi*x + lo*x into (s, e).
__device__ __forceinline__ void dot2_add(float &s, float &e, float hi, float lo, float xv) {
    const float p = hi * xv;
    float pe = fmaf(hi, xv, -p);
    pe = fmaf(lo, xv, pe);
    const float t = s + p;
    const float bp = t - s;
    const float te = (s - (t - bp)) + (p - bp);
    s = t;
    e += te + pe;
}

// Merge (s2, e2) into (s, e) (shuffle reduction of the DOT2 accumulators).
__device__ __forceinline__ void dot2_merge(float &s, float &e, float s2, float e2) {
    const float t = s + s2;
    const float bp = t - s;
    const float te = (s - (t - bp)) + (s2 - bp);
    s = t;
    e += te + e2;
}

// One output row; the R lanes of a row call this together.
//
// HO (hash order, R = 1): `row` is a position in the subspace's bucket order;
// the lane handles row hperm[row] with the key copy hkeys at that position
// (coalesced), so that for each group the warp's 32 lookups fall in a few
// consecutive buckets; diagonal, own x and y are then per-row gathers.
//
// SYM (Hermitian real operators, FP64 only): the row evaluates only the
// groups whose most significant flipped qubit is set in it -- its
// lower-triangle elements (Supplementary, "Lower / upper triangle
// evaluation") -- and each element h found at (r, c) adds h x[c] to row r and
// h x[r] to row c.  Both go to y by FP64 atomic adds into a zeroed y, so
// every element is evaluated and looked up once instead of twice, at the
// price of a summation order that varies from run to run.
template <int W, int R, int KB, int PREC, bool SYM = false, bool HO = false>
__device__ __forceinline__ void apply_row(const ApplyParams &p, const int64_t row) {
    using TIO = typename std::conditional<PREC == QSD_FP64, double, float>::type;
    constexpr int U = ApplyShape<W, KB>::U;
    static_assert(!HO || R == 1, "hash order: one lane per row");
    const int sub = threadIdx.x % R;
    const bool active = row < p.D;
    const int64_t pos = active ? row : p.D - 1;
    const int64_t r = HO ? (int64_t)__ldg(p.hperm + pos) : pos;
    const uint64_t *__restrict__ kp = HO ? p.hkeys : p.keys;
    uint64_t key[W];
#pragma unroll
    for (int w = 0; w < W; ++w) key[w] = __ldg(kp + (size_t)w * p.D + pos);
    const uint64_t hr = __ldg((HO ? p.hhash : p.rhash) + pos);
    const TIO *__restrict__ x = static_cast<const TIO *>(p.x);
    static_assert(!SYM || PREC == QSD_FP64, "half evaluation is FP64 only");
    // accumulators: FP64 (modes 0, 1) or FP32 (s, e) pairs (DOT2)
    double acc[KB];
    float as[KB], ae[KB];
#pragma unroll
    for (int j = 0; j < KB; ++j) { acc[j] = 0.0; as[j] = 0.f; ae[j] = 0.f; }
    double xr_own[SYM ? KB : 1];
    if (SYM) {
#pragma unroll
        for (int j = 0; j < KB; ++j) xr_own[j] = (double)__ldg(x + r * p.ld + p.col0 + j);
    }

    const int64_t G = p.G;
    for (int64_t g0 = (int64_t)sub * U; g0 < G; g0 += (int64_t)R * U) {
        // phase 1: element of each of U groups, and its bucket load in flight
        double a[U];
        float ah[U], al[U];
        uint2 tb[U];
        uint32_t bidx[U];
        uint32_t tag[U];
        uint32_t aidx[U];  // table groups: amplitude index; kNoTable: a[u] holds the element
        bool need[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t g = g0 + u;
            bool nz = false;
            aidx[u] = kNoTable;
            a[u] = 0.0;
            ah[u] = al[u] = 0.f;
            uint64_t hF = 0;
            if (g < G) {
                const ulonglong2 *rp = reinterpret_cast<const ulonglong2 *>(p.grec + g);
                const ulonglong2 r0 = __ldg(rp);
                const uint4 r1 = __ldg(reinterpret_cast<const uint4 *>(rp + 1));
                hF = r0.x;
                const uint32_t off = r1.x, info = r1.y, nzm = r1.z;
                bool lower = true;
                if (SYM) {
                    const int qm = (int)((info >> kMsobShift) & kMsobMask);
                    lower = bit_of<W>(key, qm);
                }
                if (!lower) {
                    // upper-triangle element: reached from its column's row
                } else if (!(info & kGroupScan)) {
                    // nb is uniform across the warp (lane per row): a real loop
                    const int nb = (int)(info & 7u);
                    int l = 0;
                    if (nb > 0) {
                        const int q0 = (int)(r0.y & 0xfff);
                        l = (int)bit_of<W>(key, q0);
                        if (nb > 1) {
                            const int q1 = (int)((r0.y >> 12) & 0xfff);
                            l |= (int)bit_of<W>(key, q1) << 1;
                            for (int i = 2; i < nb; ++i) {
                                const int q = (int)((r0.y >> (12 * i)) & 0xfff);
                                l |= (int)bit_of<W>(key, q) << i;
                            }
                        }
                    }
                    if (KB > 1) {
                        // block products: the pattern's nonzero bit decides
                        // the lookup and the amplitude is read only for a hit
                        // (k = 1 keeps the load here: fewer live registers)
                        nz = (nzm >> l) & 1u;
                        aidx[u] = off + (uint32_t)l;
                    } else if (PREC == QSD_FP32_DOT2) {
                        const float2 f = __ldg(p.ampf + off + l);
                        ah[u] = f.x;
                        al[u] = f.y;
                        nz = (nzm >> l) & 1u;
                    } else {
                        a[u] = __ldg(p.amp + off + l);
                        nz = nonzero_f64(a[u]);
                    }
                } else if (active) {
                    a[u] = scan_amp<W>(p, g, key);
                    nz = nonzero_f64(a[u]);
                    if (PREC == QSD_FP32_DOT2) {
                        ah[u] = (float)a[u];
                        al[u] = (float)(a[u] - (double)ah[u]);
                    }
                }
            }            need[u] = active && nz;
            if (need[u]) {
                bidx[u] = hash_bucket(hr ^ hF, p.hv.shift, tag[u]);
                tb[u] = __ldg(reinterpret_cast<const uint2 *>(p.hv.tags) + bidx[u]);
            }
        }
        // phase 2: resolve the lookups and accumulate
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (!need[u]) continue;
            const int64_t g = g0 + u;
            const bool full = bucket_full(tb[u]);
            if (!tag_any(tb[u], tag[u]) && !full) continue;  // absent: the common case
            const uint32_t match = tag_match(tb[u], tag[u]);
            uint64_t c[W];
            c[0] = key[0] ^ __ldg(p.gF + g);
#pragma unroll
            for (int w = 1; w < W; ++w) c[w] = key[w] ^ __ldg(p.gF + (size_t)w * p.G + g);
            // k = 1 and multi-word keys: x of the candidate row is loaded with
            // its key words (one-word keys at their 32-register budget spill
            // more than the shorter chain saves: measured)
            constexpr bool XSPEC = KB == 1 && W > 1;
            TIO xv = TIO(0);
            int64_t idx = XSPEC ? verify_matches_x<W, TIO>(p.hv, bidx[u], match, c, x + p.col0, p.ld, xv)
                                : verify_matches<W>(p.hv, bidx[u], match, c);
            if (idx < 0 && full) {
                idx = probe_from<W>(p.hv, bidx[u], tag[u], c, p.err);
                if (XSPEC && idx >= 0) xv = __ldg(x + idx * p.ld + p.col0);
            }
            if (idx < 0) continue;
            if (KB > 1 && aidx[u] != kNoTable) {
                if (PREC == QSD_FP32_DOT2) {
                    const float2 f = __ldg(p.ampf + aidx[u]);
                    ah[u] = f.x;
                    al[u] = f.y;
                } else {
                    a[u] = __ldg(p.amp + aidx[u]);
                }
            }
            const TIO *xc = x + idx * p.ld + p.col0;
            if (PREC == QSD_FP32_DOT2) {
#pragma unroll
                for (int j = 0; j < KB; ++j) dot2_add(as[j], ae[j], ah[u], al[u], (float)(XSPEC ? xv : __ldg(xc + j)));
            } else {
#pragma unroll
                for (int j = 0; j < KB; ++j) acc[j] = fma(a[u], (double)(XSPEC ? xv : __ldg(xc + j)), acc[j]);
                if (SYM) {
                    double *yc = static_cast<double *>(p.y) + idx * p.ld + p.col0;
#pragma unroll
                    for (int j = 0; j < KB; ++j) atomicAdd(yc + j, a[u] * xr_own[j]);
                }
            }
        }
    }
    if (R > 1) {
#pragma unroll
        for (int j = 0; j < KB; ++j) {
#pragma unroll
            for (int o = R / 2; o >= 1; o >>= 1) {
                if (PREC == QSD_FP32_DOT2) {
                    const float s2 = __shfl_xor_sync(0xffffffffu, as[j], o);
                    const float e2 = __shfl_xor_sync(0xffffffffu, ae[j], o);
                    dot2_merge(as[j], ae[j], s2, e2);
                } else {
                    acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
                }
            }
        }
    }
    if (active && sub == 0) {
        const double d = __ldg(p.diag + r);
        const TIO *xr = x + r * p.ld + p.col0;
        TIO *yr = static_cast<TIO *>(p.y) + r * p.ld + p.col0;
        if (PREC == QSD_FP32_DOT2) {
            const float dh = (float)d, dl = (float)(d - (double)dh);
#pragma unroll
            for (int j = 0; j < KB; ++j) {
                dot2_add(as[j], ae[j], dh, dl, (float)__ldg(xr + j));
                yr[j] = (TIO)(as[j] + ae[j]);
            }
        } else if (SYM) {
#pragma unroll
            for (int j = 0; j < KB; ++j) atomicAdd(reinterpret_cast<double *>(yr) + j, fma(d, xr_own[j], acc[j]));
        } else {
#pragma unroll
            for (int j = 0; j < KB; ++j) yr[j] = (TIO)fma(d, (double)__ldg(xr + j), acc[j]);
        }
    }
}

// One launch covers all rows: R lanes per row, rows past D inactive; HO:
// rows in hash order.
template <int W, int R, int KB, int PREC, bool SYM = false, bool HO = false>
__global__ void __launch_bounds__(256, (ApplyShape<W, KB>::MINB)) k_apply(const ApplyParams p) {
    apply_row<W, R, KB, PREC, SYM, HO>(p, ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / R);
}

// Run-time W (W > kMaxWordsStatic): a lane per row, keys in local memory,
// every group evaluated term by term, FP64 accumulation in all modes.
template <int KB, typename TIO>
__global__ void __launch_bounds__(256) k_apply_dyn(const ApplyParams p, int W) {
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= p.D) return;
    uint64_t key[kMaxWordsDyn], c[kMaxWordsDyn];
    for (int w = 0; w < W; ++w) key[w] = p.keys[(size_t)w * p.D + row];
    const uint64_t hr = key_hash_dyn(key, W, p.nib);
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
        const int64_t idx = probe_dyn(c, W, hr ^ p.grec[g].hF, p.hv, p.err);
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

// Launch one (W, R, KB) variant of precision mode PREC; hash_order (W <= 4,
// R = 1) takes the rows in the subspace's bucket order.
template <int PREC>
void launch_apply(const ApplyParams &p, int W, int R, int KB, cudaStream_t s, bool hash_order = false);
// Product parameters of one (operator, subspace) pair with x, y of row
// stride k (column 0 first).
ApplyParams product_params(qsd_ctx ctx, qsd_op op, qsd_sub sub, const double *diag, int k, const void *x, void *y);
// Packed group-scan products (W <= 4, R = 1 or 8 lanes per row; R = 8 takes
// KB = 1) served from a device tile queue (tile_queue.cuh): params [n] and
// tile0 [n] (first tile of 256 / R rows of each pair, ascending, tile0[0] =
// 0) and the queue in device memory.  The grid is the resident grid of the
// variant, capped at max_tiles (pass the queue's tile count, or a bound when
// the count is written later, as in a captured graph).
struct TileQueue;
void launch_apply_queue(const ApplyParams *params, const int64_t *tile0, TileQueue *q, int64_t max_tiles, int W,
                        int R, int KB, int precision, int num_sms, cudaStream_t s);
// Half-evaluation product (FP64, Hermitian real operators, W <= 4); zeroes
// the launch's columns of y first.
void launch_apply_sym(const ApplyParams &p, int W, int R, int KB, cudaStream_t s, bool hash_order = false);

}  // namespace qsd
