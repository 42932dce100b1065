// Warp-per-row product over a sector-factored product subspace (included by
// the apply_fac_inst.cu units).
//
// Row r = ib |A| + ia holds the string (a, b) = (A[ia], B[ib]).  For every
// shape of the operator's ladder terms -- (dOcc, dEmp) changes in sector 0
// and in sector 1 (see excite.cuh) -- the columns the row can reach inside S
// are the products of ia's neighbours of the sector-0 type and ib's
// neighbours of the sector-1 type (a type (0, 0) keeps the half).  Each
// neighbour entry carries the rank of its flipped positions and the row's
// bits on them, so a candidate column (a', b') finds its group in the dense
// rank index with one load (-1: no group has that flip mask) and its ladder
// integer -- the row's pattern on F, low sector first -- without touching
// the strings.  The group's terms with that ladder integer (int_ptrs, Fig.
// 3b) pass their remaining projector tests and add phi (-1)^popc(r & Z): the
// same element as every other path.  A nonzero element multiplies x at
// column ib' |A| + ia': no lookup.  Groups outside the excitation index are
// evaluated and looked up per row.
//
// Work split: the warp evaluates 32 candidates at a time, one per lane; the
// found (element, column) pairs are compacted in shared memory in candidate
// order, and the block's KB columns of x are gathered by KB lanes per
// candidate (32 / KB candidates per load instruction: one coalesced row of x
// each), each lane accumulating one column.  Lanes holding the same column
// are reduced with shuffles at the end.  Every order is fixed: the result is
// deterministic.  Element sums and their conversion run on the integer
// pipes: the FP64 pipe (1/64 of the FP32 rate on GB300) is left to the
// accumulation's FMAs, k per found column.
#pragma once

#include "excite.cuh"
#include "tile_queue.cuh"

namespace qsd {

struct FacParams {
    const uint64_t *A, *B;        // distinct halves
    const uint32_t *ptrA, *ptrB;  // [8 n + 1] neighbour list starts by (string, type)
    const uint2 *nbrA, *nbrB;     // (neighbour index, rank | pattern << 20 | bits << 24)
    const void *trec;             // TermRec<W> [T], fixed-point phases
    double qscale;                // value of one fixed-point unit of the term phases, 2^-qexp
    int qexp;
    // linear ranges: first row per group (-1: none), per row Zref [W], K and
    // d [nq] in fixed point
    const int32_t *lin_base;
    const uint64_t *lin_z;
    const int64_t *lin_kq, *lin_dq;
    int nq;
    // range index [rank entry][16] (nullptr: rank index then group tables)
    const uint32_t *rix;
    // half sums of the linear ranges, [nA][nlr] (K included) and [nB][nlr]
    // (nullptr: sum the row's occupied qubits' coefficients)
    const int64_t *lsA, *lsB;
    int64_t nlr;
    uint32_t nA, nB;
    int split;
};

// Internal precision mode of the factored block products: FP64 arithmetic on
// an FP64 copy of an FP32 x (widened exactly, once per product), FP32 y --
// the FP32-mixed product, bitwise, with the per-value conversion out of the
// gather loop.
constexpr int kPrecWideX = 3;

// The parameters of one pair of a packed factored product.
struct FacPair {
    ApplyParams p;
    ExcParams e;
    FacParams f;
};

// Neighbour type of (dOcc, dEmp) in the low (sector 0) or high (sector 1)
// fields of a shape; -1 for (0, 0): the half is kept.
__device__ __forceinline__ int shape_type(uint32_t occ, uint32_t emp) {
    return (occ | emp) ? (int)(3 * occ + emp) - 1 : -1;
}

constexpr uint32_t kKeepHalf = 0xffffffffu;

// Element of group g at the row from the terms [b, e) of its ladder range:
// each term's projector test (the ladder bits already match) and sign, the
// phases in 64-bit fixed point, summed exactly in integers and converted once
// by integer operations -- exact to within the rounding of each phase to a
// multiple of 2^-e.  The element thus never touches the FP64 pipe (1/64 of
// the FP32 rate on GB300), which is left to the accumulation's FMAs; a sum of
// FP64 adds instead kept that pipe 73 % busy in the single-column product.
template <int W>
__device__ __forceinline__ int64_t ladder_terms_fixed(const TermRec<W> *__restrict__ tr, int32_t b, int32_t e,
                                                      const uint64_t (&key)[W]) {
    int64_t sum = 0;
    for (int32_t t = b; t < e; ++t) {
        const TermRec<W> r = load_term<W>(tr + t);
        bool ok = true;
        int par = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            ok &= (key[w] & r.P[w]) == r.V[w];
            par ^= __popcll(key[w] & r.Z[w]);
        }
        const int64_t v = (par & 1) ? -r.q : r.q;
        sum += ok ? v : 0;
    }
    return sum;
}

// v * 2^-ex rounded to the nearest double (ties to even), by integer
// operations on the IEEE-754 encoding: the 53 leading bits of |v| become the
// significand (the bits below decide the rounding), the exponent is the
// position of the leading bit minus ex.  The operator's fixed-point exponent
// is at most 1000 and |v| >= 1, so the result is always a normal number.
// Keeps the conversion off the FP64 pipe, which the accumulation of the
// found columns saturates.
__device__ __forceinline__ double scaled_i64_to_f64(int64_t v, int ex) {
    if (v == 0) return 0.0;
    const uint64_t sign = v < 0 ? (1ull << 63) : 0ull;
    const uint64_t u = v < 0 ? (uint64_t)0 - (uint64_t)v : (uint64_t)v;
    const int lz = __clzll((long long)u);
    const int e = 63 - lz - ex;  // |v| 2^-ex lies in [2^e, 2^(e+1)), e >= -1000
    const uint64_t m = u << lz;  // leading one at bit 63
    uint64_t mant = (m >> 11) & ((1ull << 52) - 1);
    const uint64_t rest = m & 0x7ffull;
    const uint64_t up = (rest > 0x400ull || (rest == 0x400ull && (mant & 1ull))) ? 1ull : 0ull;
    mant += up;
    int eb = e + 1023;
    if (mant >> 52) {  // the rounding carried into the next binade
        mant = 0;
        ++eb;
    }
    return __longlong_as_double((long long)(sign | ((uint64_t)eb << 52) | mant));
}

// Row `row` of the product (one warp; rows past D return at once).
template <int W, int KB, int PREC>
__device__ __forceinline__ void fac_row(const ApplyParams &p, const ExcParams &e, const FacParams &f,
                                        const int64_t row) {
    // x and y storage, and the arithmetic: PREC, or for kPrecWideX FP64
    // arithmetic on an exact FP64 copy of FP32 x with FP32 y (bitwise the
    // FP32-mixed product, without a conversion per gathered value)
    constexpr bool kWideX = PREC == kPrecWideX;
    constexpr int AP = kWideX ? QSD_FP64 : PREC;
    using TIO = typename std::conditional<AP == QSD_FP64, double, float>::type;  // x
    using TY = typename std::conditional<PREC == QSD_FP64, double, float>::type;  // y
    static_assert(32 % KB == 0, "KB divides the warp");
    constexpr int NC = 32 / KB;  // candidates per gather instruction
    __shared__ uint32_t pre[8][kMaxShapes + 1];  // per warp: first candidate of each shape
    __shared__ uint32_t sa[8][kMaxShapes], sb[8][kMaxShapes], lb[8][kMaxShapes];
    // per warp: the found candidates of the current pass, compacted
    // (the pending found candidates of earlier passes, fewer than 32 / KB, first)
    __shared__ double camp[8][64];
    __shared__ uint32_t ccol[8][64];
    __shared__ uint8_t occ[8][64 * W];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (row >= p.D) return;  // warp-uniform
    // D = |A| |B| <= 2^32: 32-bit division (a 64-bit one runs on the FP64 pipe)
    const uint32_t r32 = (uint32_t)row;
    const uint32_t ib = r32 / f.nA, ia = r32 - ib * f.nA;
    uint64_t key[W];
#pragma unroll
    for (int w = 0; w < W; ++w) key[w] = __ldg(p.keys + (size_t)w * p.D + row);
    const TermRec<W> *__restrict__ trec = static_cast<const TermRec<W> *>(f.trec);
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
    const uint32_t n_exc = pre[wib][e.n_shapes];
    const uint32_t total = n_exc + (uint32_t)e.n_rest;
    const uint64_t hr = e.n_rest > 0 ? key_hash<W>(key, p.nib) : 0ull;

    // the row's occupied qubits, ascending (linear ranges sum their coefficients)
    int nocc = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t bits = (uint32_t)(key[w] >> (32 * h));
            const bool on = (bits >> lane) & 1u;
            const uint32_t m = __ballot_sync(0xffffffffu, on);
            if (on) occ[wib][nocc + __popc(m & ((1u << lane) - 1u))] = (uint8_t)(64 * w + 32 * h + lane);
            nocc += __popc(m);
        }
    }
    __syncwarp();
    const TIO *__restrict__ x = static_cast<const TIO *>(p.x) + p.col0 + (lane % KB);
    double acc = 0.0;
    float as = 0.f, ae = 0.f;
    int si = 0;
    int pend = 0;  // FP64 accumulation: found candidates not yet gathered (warp-uniform)
    for (uint32_t base = 0; base < total; base += 32) {
        // 1. one candidate per lane: its element (0: none) and column
        const uint32_t t = base + (uint32_t)lane;
        double amp = 0.0;
        uint32_t col = 0;
        if (t < n_exc) {
            while (pre[wib][si + 1] <= t) ++si;  // t ascends: the shape only moves forward
            const uint32_t u = t - pre[wib][si];
            const uint32_t l1 = lb[wib][si];
            const uint32_t ua = u / l1, ub = u - ua * l1;
            const uint32_t s0 = sa[wib][si], s1 = sb[wib][si];
            const uint2 nA = s0 == kKeepHalf ? make_uint2(ia, 0u) : __ldg(f.nbrA + s0 + ua);
            const uint2 nB = s1 == kKeepHalf ? make_uint2(ib, 0u) : __ldg(f.nbrB + s1 + ub);
            const uint32_t di = e.dbase[si] + (nA.y & 0xfffffu) * e.dstride[si] + (nB.y & 0xfffffu);
            const uint32_t na = (nA.y >> 24) & 7u;
            const uint32_t l = ((nA.y >> 20) & 15u) | (((nB.y >> 20) & 15u) << na);
            // what to evaluate: a linear-table row (lr >= 0) or a term range [tb, te)
            int64_t lr = -1;
            int32_t tb = 0, te = 0;
            bool found = false;
            if (f.rix) {
                const uint32_t v = __ldg(f.rix + (size_t)di * 16 + l);
                if (v & 0x80000000u) {
                    lr = (int64_t)(v & 0x7fffffffu);
                    found = true;
                } else {
                    tb = (int32_t)(v & 0x1fffffu);
                    te = tb + (int32_t)(v >> 21);
                    found = te > tb;
                }
            } else {
                const int32_t g = __ldg(e.dense + di);
                if (g >= 0) {
                    const uint32_t nb = (nB.y >> 24) & 7u;
                    // the linear-table row and the ladder range, loaded together
                    const bool table = na + nb <= 4;  // ladder table (every indexed group is ladder-only on F)
                    const int32_t lb = table ? __ldg(f.lin_base + g) : -1;
                    tb = table ? __ldg(p.gptr + (size_t)g * 17 + l) : __ldg(p.grange + g);
                    te = table ? __ldg(p.gptr + (size_t)g * 17 + l + 1) : __ldg(p.grange + g + 1);
                    if (lb >= 0) lr = (int64_t)lb + l;
                    found = true;
                }
            }
            if (found) {
                if (lr >= 0) {
                    // a linear range: sign of the common string, K plus the
                    // coefficients of the row's occupied qubits
                    int par = 0;
#pragma unroll
                    for (int w = 0; w < W; ++w) par ^= __popcll(key[w] & __ldg(f.lin_z + lr * W + w));
                    // (sums modulo 2^64, exact when the element fits)
                    uint64_t sum;
                    if (f.lsA) {
                        sum = (uint64_t)__ldg(f.lsA + (size_t)ia * f.nlr + lr) +
                              (uint64_t)__ldg(f.lsB + (size_t)ib * f.nlr + lr);
                    } else {
                        const int64_t *__restrict__ dr = f.lin_dq + lr * f.nq;
                        sum = (uint64_t)__ldg(f.lin_kq + lr);
                        for (int i = 0; i < nocc; ++i) sum += (uint64_t)__ldg(dr + occ[wib][i]);
                    }
                    const int64_t v = (int64_t)sum;
                    amp = scaled_i64_to_f64((par & 1) ? -v : v, f.qexp);
                } else {
                    amp = scaled_i64_to_f64(ladder_terms_fixed<W>(trec, tb, te, key), f.qexp);
                }
                col = nB.x * f.nA + nA.x;
            }
        } else if (t < total) {
            const int64_t g = __ldg(e.rest_gid + (t - n_exc));
            const double a = scan_amp<W>(p, g, key);
            if (((uint64_t)__double_as_longlong(a) << 1) != 0ull) {
                uint64_t c[W];
#pragma unroll
                for (int w = 0; w < W; ++w) c[w] = key[w] ^ __ldg(p.gF + (size_t)w * p.G + g);
                const int64_t idx = probe<W>(c, hr ^ __ldg(&p.grec[g].hF), p.hv, p.err);
                if (idx >= 0) {
                    amp = a;
                    col = (uint32_t)idx;
                }
            }
        }
        // 2. gather
        const bool nz = ((uint64_t)__double_as_longlong(amp) << 1) != 0ull;
        if (KB == 1) {
            // each lane its own candidate
            if (nz) {
                const TIO xv = __ldg(x + (size_t)col * p.ld);
                if (AP == QSD_FP32_DOT2) {
                    const float ah = (float)amp, al = (float)(amp - (double)ah);
                    dot2_add(as, ae, ah, al, (float)xv);
                } else if (AP == QSD_FP32_MIXED) {
                    acc = fma(amp, f32_to_f64((float)xv), acc);
                } else {
                    acc = fma(amp, (double)xv, acc);
                }
            }
            continue;
        }
        const uint32_t found = __ballot_sync(0xffffffffu, nz);
        if (!found) continue;
        if (AP == QSD_FP32_DOT2) {
            // KB lanes per candidate, NC candidates per load instruction: the
            // element's FP32 (hi, lo) split once, in the candidate's lane, and
            // broadcast by shuffles
            const float ah = (float)amp, al = (float)(amp - (double)ah);
#pragma unroll
            for (int i = 0; i < KB; ++i) {
                const int src = i * NC + lane / KB;
                const float h = __shfl_sync(0xffffffffu, ah, src);
                const float l = __shfl_sync(0xffffffffu, al, src);
                const uint32_t c = __shfl_sync(0xffffffffu, col, src);
                if (h != 0.f || l != 0.f) dot2_add(as, ae, h, l, (float)__ldg(x + (size_t)c * p.ld));
            }
            continue;
        }
        // FP64 accumulation: the found candidates appended, in candidate
        // order, behind those pending from earlier passes; whole groups of
        // NC are gathered (KB lanes per candidate, NC candidates per load
        // instruction), so every FP64 FMA runs at full lanes, and the rest
        // (fewer than NC) moves to the front for the next pass
        if (nz) {
            const int slot = pend + __popc(found & ((1u << lane) - 1u));
            camp[wib][slot] = amp;
            ccol[wib][slot] = col;
        }
        __syncwarp();
        const int tot = pend + __popc(found), full = tot - tot % NC;
        for (int i0 = 0; i0 < full; i0 += NC) {
            const int src = i0 + lane / KB;
            const TIO xv = __ldg(x + (size_t)ccol[wib][src] * p.ld);
            if (AP == QSD_FP32_MIXED) acc = fma(camp[wib][src], f32_to_f64((float)xv), acc);
            else acc = fma(camp[wib][src], (double)xv, acc);
        }
        pend = tot - full;
        if (pend > 0 && full > 0) {
            double a = 0.0;
            uint32_t c = 0;
            if (lane < pend) {
                a = camp[wib][full + lane];
                c = ccol[wib][full + lane];
            }
            __syncwarp();
            if (lane < pend) {
                camp[wib][lane] = a;
                ccol[wib][lane] = c;
            }
        }
        __syncwarp();
    }
    if (KB > 1 && AP != QSD_FP32_DOT2 && pend > 0) {
        // the last pending candidates: one partial gather
        const int src = lane / KB;
        if (src < pend) {
            const TIO xv = __ldg(x + (size_t)ccol[wib][src] * p.ld);
            if (AP == QSD_FP32_MIXED) acc = fma(camp[wib][src], f32_to_f64((float)xv), acc);
            else acc = fma(camp[wib][src], (double)xv, acc);
        }
    }
    // lanes with the same column (lane % KB) hold parts of its sum
#pragma unroll
    for (int o = KB; o < 32; o <<= 1) {
        if (AP == QSD_FP32_DOT2) {
            const float s2 = __shfl_xor_sync(0xffffffffu, as, o);
            const float e2 = __shfl_xor_sync(0xffffffffu, ae, o);
            dot2_merge(as, ae, s2, e2);
        } else {
            acc += __shfl_xor_sync(0xffffffffu, acc, o);
        }
    }
    if (lane < KB) {
        const double d = __ldg(p.diag + row);
        const TIO xr = __ldg(x + row * p.ld);
        TY *yr = static_cast<TY *>(p.y) + row * p.ld + p.col0 + lane;
        if (AP == QSD_FP32_DOT2) {
            const float dh = (float)d, dl = (float)(d - (double)dh);
            dot2_add(as, ae, dh, dl, (float)xr);
            *yr = (TY)(as + ae);
        } else {
            *yr = (TY)fma(d, (double)xr, acc);
        }
    }
}

template <int W, int KB, int PREC>
__global__ void __launch_bounds__(256) k_apply_fac(const ApplyParams p, const ExcParams e, const FacParams f) {
    fac_row<W, KB, PREC>(p, e, f, ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
}

// Packed factored products: tiles of 8 rows (a warp per row) of many pairs
// from a device tile queue; each row is evaluated as by k_apply_fac.
template <int W, int KB, int PREC>
__global__ void __launch_bounds__(256)
    k_apply_fac_queue(const FacPair *__restrict__ params, const int64_t *__restrict__ tile0, TileQueue *q) {
    __shared__ FacPair sp;
    run_tile_queue(params, tile0, q, sp, [](const FacPair &r, int, int64_t t) {
        fac_row<W, KB, PREC>(r.p, r.e, r.f, t * 8 + (threadIdx.x >> 5));
    });
}

// Launch the factored product for precision mode PREC (W <= 2).
template <int PREC>
void launch_apply_fac(const ApplyParams &p, const ExcParams &e, const FacParams &f, int W, int KB, cudaStream_t s);
// Packed product classes: 0..3 the group scan with one lane per row of key
// width W = class + 1 (256-row tiles), 4..7 the group scan with eight lanes
// per row, W = class - 3 (32-row tiles; single columns), 8..9 the factored
// product of key width W = class - 7 (8-row tiles, a warp per row).  A pair
// takes the factored product where it applies (the path the single product
// takes), else the scan; eight lanes per row only where asked for and where
// the single product would take them (small subspaces, many groups).
constexpr int kPackScan8Class = 4, kPackFacClass = 8, kPackClasses = 10;
int pack_class(qsd_ctx ctx, qsd_op op, qsd_sub sub, bool lanes8);
inline int pack_class_width(int c) {
    return c >= kPackFacClass ? c - kPackFacClass + 1 : (c >= kPackScan8Class ? c - kPackScan8Class + 1 : c + 1);
}
inline int pack_class_lanes(int c) { return c >= kPackFacClass ? 32 : (c >= kPackScan8Class ? 8 : 1); }
inline int pack_class_rows(int c) { return 256 / pack_class_lanes(c); }
// The factored-product parameters of one pair with x, y of row stride k.
FacPair factored_params(qsd_ctx ctx, qsd_op op, qsd_sub sub, const double *diag, int k, const void *x, void *y);

// Packed factored products (W <= 2) of the pairs of a device tile queue
// (8-row tiles); grid as launch_apply_queue.
template <int PREC>
void launch_apply_fac_queue(const FacPair *params, const int64_t *tile0, TileQueue *q, int64_t max_tiles, int W,
                            int KB, int num_sms, cudaStream_t s);

}  // namespace qsd
