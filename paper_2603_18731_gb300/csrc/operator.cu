// Operator loading and grouping (Methods, "Hamiltonian representations"),
// the cached diagonal, and the target / term tables used for integer-exact
// checks.
//
// Mask form of a word.  For a row bit-string r, a word over the extended
// alphabet has one candidate column r xor F, and
//     <r|W|r xor F> = phi * (-1)^popc(r & Z) * [(r & P) == V]
// with, per qubit q of the word:
//     Z: Z        0: P          1: P, V          X: F
//     Y: F, Z, phi *= -i        -: F, P          +: F, P, V
// (Y = [[0,-i],[i,0]] has <r|Y|1-r> = -i (-1)^r;  + = |1><0| needs r = 1;
//  - = |0><1| needs r = 0; the projectors fix the bit.)  F is the paper's
// off-diagonal structure (properties 1-3), P/V are the constraints of the
// projector and ladder letters (the 1/2^m rule), and the Z mask carries the
// Jordan-Wigner strings.
#include <algorithm>
#include <cmath>
#include <complex>

#include "apply_kernel.cuh"
#include "qsd_internal.cuh"

namespace qsd {

namespace {

constexpr int kLadderMax = 4;             // int_ptrs of 2^4+1 entries (Methods, Fig. 3b)
constexpr int kLadderPtrs = (1 << kLadderMax) + 1;

__global__ void k_gather_phi(const uint32_t *__restrict__ perm, const double *__restrict__ re,
                             const double *__restrict__ im, int64_t n, double *ore, double *oim) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    ore[i] = re[perm[i]];
    oim[i] = im[perm[i]];
}

__global__ void k_run_starts(const uint32_t *__restrict__ flags, const uint32_t *__restrict__ pos, int64_t n,
                             int64_t n_out, int32_t *starts) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && flags[i]) starts[pos[i]] = (int32_t)i;
    if (i == 0) starts[n_out] = (int32_t)n;
}

// Sum the coefficients of each run of equal words in input order.
__global__ void k_combine(const int32_t *__restrict__ starts, int64_t m, const double *__restrict__ re,
                          const double *__restrict__ im, double *ore, double *oim) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= m) return;
    double a = 0.0, b = 0.0;
    for (int32_t i = starts[u]; i < starts[u + 1]; ++i) { a += re[i]; b += im[i]; }
    ore[u] = a;
    oim[u] = b;
}

__global__ void k_count_zero(const uint64_t *__restrict__ v, int64_t n, unsigned long long *cnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && v[i] == 0) atomicAdd(cnt, 1ull);
}

// out[w][j] = src[(row0 + w) * ld + col0 + j]
__global__ void k_slice_rows(const uint64_t *__restrict__ src, int64_t ld, int row0, int rows, int64_t col0,
                             int64_t cnt, uint64_t *out) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cnt) return;
    for (int w = 0; w < rows; ++w) out[(size_t)w * cnt + j] = src[(size_t)(row0 + w) * ld + col0 + j];
}

__global__ void k_group_flags(const uint64_t *__restrict__ keysF /*[W] rows, stride ld*/, int64_t ld, int W,
                              int64_t off, int64_t T, uint32_t *flags) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= T) return;
    uint32_t f = 1;
    if (i > 0) {
        f = 0;
        for (int w = 0; w < W; ++w) f |= keysF[(size_t)w * ld + off + i] != keysF[(size_t)w * ld + off + i - 1];
    }
    flags[i] = f;
}

__global__ void k_group_starts(const uint32_t *__restrict__ flags, const uint32_t *__restrict__ pos, int64_t T,
                               int64_t G, int32_t *grange) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < T && flags[i]) grange[pos[i]] = (int32_t)i;
    if (i == 0) grange[G] = (int32_t)T;
}

__global__ void k_group_tables(int W, int64_t G, const int32_t *__restrict__ grange, const uint64_t *__restrict__ tF,
                               int64_t T, const uint64_t *__restrict__ tP, const uint64_t *__restrict__ tV,
                               const uint64_t *__restrict__ nib, uint64_t *gF, uint64_t *ghash, uint8_t *gL,
                               uint64_t *gpos, int32_t *gptr, unsigned long long *max_terms,
                               unsigned long long *n_ladder) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    const int32_t b = grange[g], e = grange[g + 1];
    uint64_t F[kMaxWordsDyn];
    int L = 0;
    for (int w = 0; w < W; ++w) {
        F[w] = tF[(size_t)w * T + b];
        gF[(size_t)w * G + g] = F[w];
        L += __popcll(F[w]);
    }
    ghash[g] = key_hash_dyn(F, W, nib);
    atomicMax(max_terms, (unsigned long long)(e - b));
    // flipped-qubit positions, ascending (first four)
    uint64_t pos = 0;
    int found = 0;
    for (int w = 0; w < W && found < kLadderMax; ++w) {
        uint64_t f = F[w];
        while (f && found < kLadderMax) {
            const int bit = __ffsll((long long)f) - 1;
            pos |= (uint64_t)(64 * w + bit) << (16 * found);
            ++found;
            f &= f - 1;
        }
    }
    gpos[g] = pos;
    bool ladder = L <= kLadderMax;
    for (int32_t t = b; t < e && ladder; ++t)
        for (int w = 0; w < W; ++w) ladder &= (tP[(size_t)w * T + t] & F[w]) == F[w];
    gL[g] = ladder ? (uint8_t)L : 0;
    if (!ladder) return;
    atomicAdd(n_ladder, 1ull);
    // terms are sorted by (V & F): the ladder integer is non-decreasing
    int32_t t = b;
    for (int l = 0; l < kLadderPtrs; ++l) {
        while (t < e) {
            int lt = 0;
            for (int i = 0; i < L; ++i) {
                const int q = (int)((pos >> (16 * i)) & 0xffff);
                lt |= (int)((tV[(size_t)(q >> 6) * T + t] >> (q & 63)) & 1) << i;
            }
            if (lt >= l) break;
            ++t;
        }
        gptr[g * kLadderPtrs + l] = t;
    }
}

// Support of a group: every qubit any of its terms tests (projector and
// ladder letters) or signs (Z, Y, Jordan-Wigner strings).  The flipped qubits
// of pure X letters do not change the element and stay outside.  Groups with
// a support of <= kTableBitsMax qubits get an amplitude table (a group of
// X letters only has an empty support: one constant element).
__global__ void k_group_support(int W, int64_t G, const int32_t *__restrict__ grange, const uint64_t *__restrict__ gF,
                                int64_t T, const uint64_t *__restrict__ tP, const uint64_t *__restrict__ tZ,
                                uint32_t *size, uint64_t *spos) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    int nb = 0;
    uint64_t pos = 0;
    for (int w = 0; w < W && nb <= kTableBitsMax; ++w) {
        uint64_t u = 0;
        for (int32_t t = grange[g]; t < grange[g + 1]; ++t) u |= tP[(size_t)w * T + t] | tZ[(size_t)w * T + t];
        while (u) {
            const int bit = __ffsll((long long)u) - 1;
            if (nb < kTableBitsMax) pos |= (uint64_t)(64 * w + bit) << (12 * nb);
            ++nb;
            u &= u - 1;
        }
    }
    size[g] = nb <= kTableBitsMax ? (1u << nb) : 0u;
    spos[g] = nb <= kTableBitsMax ? pos | ((uint64_t)nb << 60) : 0;
}

// Amplitude tables and the 32-byte group records.
__global__ void k_group_records(int W, int64_t G, const int32_t *__restrict__ grange, const uint64_t *__restrict__ gF,
                                const uint64_t *__restrict__ ghash, int64_t T, const uint64_t *__restrict__ tP,
                                const uint64_t *__restrict__ tV, const uint64_t *__restrict__ tZ,
                                const double *__restrict__ tphi, const uint32_t *__restrict__ size,
                                const uint32_t *__restrict__ off, const uint64_t *__restrict__ spos, double *amp,
                                float2 *ampf, GroupRec *rec) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    GroupRec R;
    R.hF = ghash[g];
    R.nzmask = 0;
    R.pad = 0;
    // most significant flipped qubit (the half-evaluation product's filter)
    uint32_t msob = 0;
    for (int w = 0; w < W; ++w)
        if (gF[(size_t)w * G + g]) msob = (uint32_t)(64 * w + 63 - __clzll((long long)gF[(size_t)w * G + g]));
    const uint32_t hi_info = (msob & kMsobMask) << kMsobShift;
    if (size[g] == 0) {
        R.pos = 0;
        R.off = 0;
        R.info = kGroupScan | hi_info;
        rec[g] = R;
        return;
    }
    const int nb = (int)(spos[g] >> 60);
    const uint64_t pos = spos[g] & ((1ull << 60) - 1);
    R.pos = pos;
    R.off = off[g];
    R.info = (uint32_t)nb | hi_info;
    uint64_t rs[kMaxWordsDyn];
    for (uint32_t l = 0; l < size[g]; ++l) {
        for (int w = 0; w < W; ++w) rs[w] = 0;
        for (int i = 0; i < nb; ++i) {
            const int q = (int)((pos >> (12 * i)) & 0xfff);
            if ((l >> i) & 1u) rs[q >> 6] |= 1ull << (q & 63);
        }
        double a = 0.0;
        for (int32_t t = grange[g]; t < grange[g + 1]; ++t) {
            bool ok = true;
            int par = 0;
            for (int w = 0; w < W; ++w) {
                ok &= (rs[w] & tP[(size_t)w * T + t]) == tV[(size_t)w * T + t];
                par ^= __popcll(rs[w] & tZ[(size_t)w * T + t]);
            }
            if (ok) a += (par & 1) ? -tphi[t] : tphi[t];
        }
        amp[R.off + l] = a;
        if (((uint64_t)__double_as_longlong(a) << 1) != 0ull) R.nzmask |= 1u << l;
        const float hi = (float)a;
        ampf[R.off + l] = make_float2(hi, (float)(a - (double)hi));
    }
    rec[g] = R;
}

__global__ void k_term_flags(int W, int64_t T, const uint64_t *__restrict__ tP, const uint64_t *__restrict__ tZ,
                             uint8_t *flag) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    uint64_t p = 0, z = 0;
    for (int w = 0; w < W; ++w) { p |= tP[(size_t)w * T + t]; z |= tZ[(size_t)w * T + t]; }
    flag[t] = (uint8_t)((p ? 1 : 0) | (z ? 2 : 0));
}

// Sorted unique word keys, K = 5W+1 rows: [Z | V | P | V&F | F | popc F].
__device__ int key_cmp_col(const uint64_t *keys, int K, int64_t ld, int64_t i, const uint64_t *k) {
    for (int w = K - 1; w >= 0; --w) {
        const uint64_t a = keys[(size_t)w * ld + i];
        if (a < k[w]) return -1;
        if (a > k[w]) return 1;
    }
    return 0;
}

// Hermiticity: the adjoint of (F, P, V, Z, phi) is (F, P, V xor (P & F), Z,
// conj(phi) (-1)^nY) with nY = popc(F & Z) (the Y letters), since + and -
// swap and c -> c* while the (-i)^nY factor of phi is kept.
__global__ void k_hermitian(int W, int64_t m, const uint64_t *__restrict__ keys, const double *__restrict__ re,
                            const double *__restrict__ im, double tol, uint32_t *bad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int K = 5 * W + 1;
    uint64_t k[5 * kMaxWordsDyn + 1];
    int ny = 0;
    for (int w = 0; w < W; ++w) {
        const uint64_t Z = keys[(size_t)w * m + i], V = keys[(size_t)(W + w) * m + i];
        const uint64_t P = keys[(size_t)(2 * W + w) * m + i], F = keys[(size_t)(4 * W + w) * m + i];
        const uint64_t Va = V ^ (P & F);
        k[w] = Z;
        k[W + w] = Va;
        k[2 * W + w] = P;
        k[3 * W + w] = Va & F;
        k[4 * W + w] = F;
        ny += __popcll(F & Z);
    }
    k[5 * W] = keys[(size_t)(5 * W) * m + i];
    const double sre = re[i], sim = (ny & 1) ? im[i] : -im[i];
    const double are = (ny & 1) ? -sre : sre;  // conj(phi) * (-1)^nY
    const double aim = sim;
    int64_t lo = 0, hi = m - 1, found = -1;
    while (lo <= hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        const int c = key_cmp_col(keys, K, m, mid, k);
        if (c == 0) { found = mid; break; }
        if (c < 0) lo = mid + 1; else hi = mid - 1;
    }
    if (found < 0) {
        if (fabs(sre) + fabs(sim) > tol) atomicOr(bad, 1u);
    } else if (fabs(re[found] - are) + fabs(im[found] - aim) > tol) {
        atomicOr(bad, 1u);
    }
}

__global__ void k_absmax(const double *__restrict__ re, const double *__restrict__ im, int64_t n,
                         unsigned long long *out /* [0]: max|phi|, [1]: max|im| as ordered bits */) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double a = fabs(re[i]) + fabs(im[i]), b = fabs(im[i]);
    atomicMax(out, (unsigned long long)__double_as_longlong(a));
    atomicMax(out + 1, (unsigned long long)__double_as_longlong(b));
}

// ------------------------------------------------------------ diagonal
template <int W>
__global__ void k_diagonal(const uint64_t *__restrict__ keys, int64_t D, double c0, int64_t Td,
                           const uint64_t *__restrict__ P, const uint64_t *__restrict__ V,
                           const uint64_t *__restrict__ Z, const double *__restrict__ phi, double *d) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= D) return;
    uint64_t x[W];
#pragma unroll
    for (int w = 0; w < W; ++w) x[w] = keys[(size_t)w * D + r];
    double s = c0;
    for (int64_t t = 0; t < Td; ++t) {
        bool ok = true;
        int par = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            ok &= (x[w] & __ldg(P + (size_t)w * Td + t)) == __ldg(V + (size_t)w * Td + t);
            par ^= __popcll(x[w] & __ldg(Z + (size_t)w * Td + t));
        }
        if (ok) s += (par & 1) ? -__ldg(phi + t) : __ldg(phi + t);
    }
    d[r] = s;
}

__global__ void k_diagonal_dyn(const uint64_t *__restrict__ keys, int W, int64_t D, double c0, int64_t Td,
                               const uint64_t *__restrict__ P, const uint64_t *__restrict__ V,
                               const uint64_t *__restrict__ Z, const double *__restrict__ phi, double *d) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= D) return;
    double s = c0;
    for (int64_t t = 0; t < Td; ++t) {
        bool ok = true;
        int par = 0;
        for (int w = 0; w < W; ++w) {
            const uint64_t x = keys[(size_t)w * D + r];
            ok &= (x & P[(size_t)w * Td + t]) == V[(size_t)w * Td + t];
            par ^= __popcll(x & Z[(size_t)w * Td + t]);
        }
        if (ok) s += (par & 1) ? -phi[t] : phi[t];
    }
    d[r] = s;
}

// --------------------------------------------------------- integer tables
// One thread per (row, input term): the unit factor of <r|W_t|r xor F_t>.
__global__ void k_term_table(const uint64_t *__restrict__ keys, int W, int64_t D, int64_t row0, int64_t nrows,
                             int64_t Ti, const uint64_t *__restrict__ iP, const uint64_t *__restrict__ iV,
                             const uint64_t *__restrict__ iZ, const uint8_t *__restrict__ iY, int8_t *out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nrows * Ti) return;
    const int64_t i = idx / Ti, t = idx % Ti, r = row0 + i;
    bool ok = true;
    int par = 0;
    for (int w = 0; w < W; ++w) {
        const uint64_t x = keys[(size_t)w * D + r];
        ok &= (x & iP[(size_t)w * Ti + t]) == iV[(size_t)w * Ti + t];
        par ^= __popcll(x & iZ[(size_t)w * Ti + t]);
    }
    // element = (-i)^nY (-1)^par = i^(3 nY + 2 par)
    const int p = (3 * iY[t] + 2 * (par & 1)) & 3;
    out[idx] = ok ? (int8_t)(1 + p) : (int8_t)0;
}

// One thread per (row, group), with the same skip rule as the product.
template <int W>
__global__ void k_target_table(const uint64_t *__restrict__ keys, int64_t D, const HashView hv,
                               const uint64_t *__restrict__ nib, int64_t G,
                               const uint64_t *__restrict__ gF, const uint64_t *__restrict__ ghash,
                               const int32_t *__restrict__ grange, const uint8_t *__restrict__ gL,
                               const uint64_t *__restrict__ gpos, const int32_t *__restrict__ gptr, int64_t T,
                               const uint64_t *__restrict__ tP, const uint64_t *__restrict__ tV,
                               int64_t row0, int64_t nrows, int64_t *out, uint32_t *err) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nrows * G) return;
    const int64_t i = idx / G, g = idx % G, r = row0 + i;
    uint64_t x[W];
#pragma unroll
    for (int w = 0; w < W; ++w) x[w] = keys[(size_t)w * D + r];
    int32_t b, e;
    const int L = gL[g];
    if (L) {
        const uint64_t pos = gpos[g];
        int l = 0;
        for (int j = 0; j < L; ++j) {
            const int q = (int)((pos >> (16 * j)) & 0xffff);
            uint64_t v = x[0];
#pragma unroll
            for (int w = 1; w < W; ++w) if ((q >> 6) == w) v = x[w];
            l |= (int)((v >> (q & 63)) & 1) << j;
        }
        b = gptr[g * kLadderPtrs + l];
        e = gptr[g * kLadderPtrs + l + 1];
    } else {
        b = grange[g];
        e = grange[g + 1];
    }
    bool any = false;
    for (int32_t t = b; t < e && !any; ++t) {
        bool ok = true;
#pragma unroll
        for (int w = 0; w < W; ++w) ok &= (x[w] & tP[(size_t)w * T + t]) == tV[(size_t)w * T + t];
        any |= ok;
    }
    if (!any) { out[idx] = -2; return; }
    uint64_t c[W];
#pragma unroll
    for (int w = 0; w < W; ++w) c[w] = x[w] ^ gF[(size_t)w * G + g];
    uint64_t hr = key_hash<W>(x, nib);
    out[idx] = probe<W>(c, hr ^ ghash[g], hv, err);
}

__global__ void k_target_table_dyn(const uint64_t *__restrict__ keys, int W, int64_t D, const HashView hv,
                                   const uint64_t *__restrict__ nib, int64_t G, const uint64_t *__restrict__ gF,
                                   const uint64_t *__restrict__ ghash, const int32_t *__restrict__ grange,
                                   int64_t T, const uint64_t *__restrict__ tP, const uint64_t *__restrict__ tV,
                                   int64_t row0, int64_t nrows, int64_t *out, uint32_t *err) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nrows * G) return;
    const int64_t i = idx / G, g = idx % G, r = row0 + i;
    uint64_t x[kMaxWordsDyn], c[kMaxWordsDyn];
    for (int w = 0; w < W; ++w) x[w] = keys[(size_t)w * D + r];
    bool any = false;
    for (int32_t t = grange[g]; t < grange[g + 1] && !any; ++t) {
        bool ok = true;
        for (int w = 0; w < W; ++w) ok &= (x[w] & tP[(size_t)w * T + t]) == tV[(size_t)w * T + t];
        any |= ok;
    }
    if (!any) { out[idx] = -2; return; }
    for (int w = 0; w < W; ++w) c[w] = x[w] ^ gF[(size_t)w * G + g];
    out[idx] = probe_dyn(c, W, key_hash_dyn(x, W, nib) ^ ghash[g], hv, err);
}

struct HostWord {
    std::vector<uint64_t> F, P, V, Z;
    int ny = 0;
};

}  // namespace

void load_operator(qsd_ctx ctx, qsd_op op, int64_t n_terms, const int64_t *term_ptr, const int32_t *op_qubit,
                   const uint8_t *op_code, const double *coef_re, const double *coef_im) {
    cudaStream_t s = ctx->stream;
    const int W = op->W, n = op->n_qubits;
    ensure_nibble_tables(ctx, W);
    if (n_terms < 0 || !term_ptr || (n_terms > 0 && !coef_re)) fail(QSD_ERR_INVALID_ARG, "load_operator: bad term arrays");
    if (term_ptr[0] != 0) fail(QSD_ERR_INVALID_ARG, "load_operator: term_ptr[0] must be 0");
    for (int64_t t = 0; t < n_terms; ++t)
        if (term_ptr[t + 1] < term_ptr[t]) fail(QSD_ERR_INVALID_ARG, "load_operator: term_ptr not non-decreasing");
    if (term_ptr[n_terms] > 0 && (!op_qubit || !op_code)) fail(QSD_ERR_INVALID_ARG, "load_operator: missing factors");
    if (n_terms >= (int64_t)0x7fffffff) fail(QSD_ERR_CAPACITY, "load_operator: too many terms");
    {
        // keep the input words for operators derived from this one (trimming)
        const int64_t nf = term_ptr[n_terms];
        op->in_term_ptr.assign(term_ptr, term_ptr + n_terms + 1);
        op->in_qubit.assign(op_qubit, op_qubit + (nf > 0 ? nf : 0));
        op->in_code.assign(op_code, op_code + (nf > 0 ? nf : 0));
        op->in_re.assign(coef_re, coef_re + n_terms);
        if (coef_im) op->in_im.assign(coef_im, coef_im + n_terms);
        else op->in_im.assign((size_t)n_terms, 0.0);
    }

    // ---- host: words -> masks (input order), validation
    const int64_t Ti = n_terms;
    std::vector<uint64_t> iF((size_t)W * Ti, 0), iP((size_t)W * Ti, 0), iV((size_t)W * Ti, 0), iZ((size_t)W * Ti, 0);
    std::vector<uint8_t> iY(Ti, 0);
    std::vector<uint64_t> seen(W);
    double id_re = 0.0, id_im = 0.0;
    std::vector<int64_t> canon;  // input index of each non-identity nonzero term
    std::vector<double> phre, phim;
    for (int64_t t = 0; t < Ti; ++t) {
        std::fill(seen.begin(), seen.end(), 0);
        int ny = 0;
        for (int64_t a = term_ptr[t]; a < term_ptr[t + 1]; ++a) {
            const int q = op_qubit[a];
            const int c = op_code[a];
            if (q < 0 || q >= n || c > 6)
                fail(QSD_ERR_QUBIT_RANGE, "load_operator: term " + std::to_string(t) + " has qubit " +
                                              std::to_string(q) + " / letter " + std::to_string(c) + " out of range");
            const int w = q >> 6;
            const uint64_t bit = 1ull << (q & 63);
            if (seen[w] & bit)
                fail(QSD_ERR_REPEATED_INDEX, "load_operator: term " + std::to_string(t) + " repeats qubit " + std::to_string(q));
            seen[w] |= bit;
            const size_t o = (size_t)w * Ti + t;
            switch (c) {
            case 0: iZ[o] |= bit; break;                          // Z
            case 1: iP[o] |= bit; break;                          // 0
            case 2: iP[o] |= bit; iV[o] |= bit; break;            // 1
            case 3: iF[o] |= bit; break;                          // X
            case 4: iF[o] |= bit; iZ[o] |= bit; ++ny; break;      // Y
            case 5: iF[o] |= bit; iP[o] |= bit; break;            // -
            default: iF[o] |= bit; iP[o] |= bit; iV[o] |= bit;    // +
            }
        }
        iY[t] = (uint8_t)(ny & 3);
        const double cr = coef_re[t], ci = coef_im ? coef_im[t] : 0.0;
        if (cr == 0.0 && ci == 0.0) continue;
        if (term_ptr[t + 1] == term_ptr[t]) { id_re += cr; id_im += ci; continue; }
        // phi = c * (-i)^nY = c * i^(3 nY)
        std::complex<double> ph(cr, ci);
        for (int k = 0; k < (3 * ny) % 4; ++k) ph *= std::complex<double>(0.0, 1.0);
        canon.push_back(t);
        phre.push_back(ph.real());
        phim.push_back(ph.imag());
    }
    op->T_in = Ti;
    op->identity = id_re;
    op->identity_im = id_im;
    if (Ti > 0) {
        op->iF.alloc(iF.size() * 8); op->iP.alloc(iP.size() * 8); op->iV.alloc(iV.size() * 8); op->iZ.alloc(iZ.size() * 8);
        op->iY.alloc(Ti);
        QSD_CUDA(cudaMemcpyAsync(op->iF.p, iF.data(), iF.size() * 8, cudaMemcpyHostToDevice, s));
        QSD_CUDA(cudaMemcpyAsync(op->iP.p, iP.data(), iP.size() * 8, cudaMemcpyHostToDevice, s));
        QSD_CUDA(cudaMemcpyAsync(op->iV.p, iV.data(), iV.size() * 8, cudaMemcpyHostToDevice, s));
        QSD_CUDA(cudaMemcpyAsync(op->iZ.p, iZ.data(), iZ.size() * 8, cudaMemcpyHostToDevice, s));
        QSD_CUDA(cudaMemcpyAsync(op->iY.p, iY.data(), Ti, cudaMemcpyHostToDevice, s));
    }

    // ---- device: sort by [Z | V | P | V&F | F | popc F] (last most significant)
    const int64_t Tc = (int64_t)canon.size();
    const int K = 5 * W + 1;
    int64_t Tu = 0, Td = 0;
    DevBuf ukeys, ure, uim;
    bool hermitian = std::abs(id_im) == 0.0;
    double maxphi = std::abs(id_re), maxim = std::abs(id_im);
    if (Tc > 0) {
        std::vector<uint64_t> hk((size_t)K * Tc);
        for (int64_t j = 0; j < Tc; ++j) {
            const int64_t t = canon[j];
            int pc = 0;
            for (int w = 0; w < W; ++w) {
                const size_t o = (size_t)w * Ti + t;
                hk[(size_t)w * Tc + j] = iZ[o];
                hk[(size_t)(W + w) * Tc + j] = iV[o];
                hk[(size_t)(2 * W + w) * Tc + j] = iP[o];
                hk[(size_t)(3 * W + w) * Tc + j] = iV[o] & iF[o];
                hk[(size_t)(4 * W + w) * Tc + j] = iF[o];
                pc += __builtin_popcountll(iF[o]);
            }
            hk[(size_t)(5 * W) * Tc + j] = (uint64_t)pc;
        }
        std::vector<uint32_t> perm(Tc);
        for (int64_t j = 0; j < Tc; ++j) perm[j] = (uint32_t)j;
        DevBuf dk((size_t)K * Tc * 8), dperm((size_t)Tc * 4), dre((size_t)Tc * 8), dim_((size_t)Tc * 8);
        DevBuf sre((size_t)Tc * 8), sim((size_t)Tc * 8);
        QSD_CUDA(cudaMemcpyAsync(dk.p, hk.data(), hk.size() * 8, cudaMemcpyHostToDevice, s));
        QSD_CUDA(cudaMemcpyAsync(dperm.p, perm.data(), (size_t)Tc * 4, cudaMemcpyHostToDevice, s));
        QSD_CUDA(cudaMemcpyAsync(dre.p, phre.data(), (size_t)Tc * 8, cudaMemcpyHostToDevice, s));
        QSD_CUDA(cudaMemcpyAsync(dim_.p, phim.data(), (size_t)Tc * 8, cudaMemcpyHostToDevice, s));
        radix_sort(ctx, dk.as<uint64_t>(), K, Tc, dperm.as<uint32_t>());
        k_gather_phi<<<blocks_for(Tc, 256), 256, 0, s>>>(dperm.as<uint32_t>(), dre.as<double>(), dim_.as<double>(), Tc,
                                                        sre.as<double>(), sim.as<double>());
        QSD_LAUNCH_CHECK();
        // combine equal words: runs of equal keys, summed in input order
        DevBuf flags((size_t)Tc * 4), pos((size_t)Tc * 4);
        Tu = unique_sorted(ctx, dk.as<uint64_t>(), K, Tc, nullptr, 0);
        ukeys.alloc((size_t)K * Tu * 8);
        unique_sorted(ctx, dk.as<uint64_t>(), K, Tc, ukeys.as<uint64_t>(), Tu);
        DevBuf starts((size_t)(Tu + 1) * 4);
        diff_flags(ctx, dk.as<uint64_t>(), K, Tc, flags.as<uint32_t>());
        exclusive_scan_u32(ctx, flags.as<uint32_t>(), pos.as<uint32_t>(), Tc, false);
        k_run_starts<<<blocks_for(Tc, 256), 256, 0, s>>>(flags.as<uint32_t>(), pos.as<uint32_t>(), Tc, Tu,
                                                         starts.as<int32_t>());
        QSD_LAUNCH_CHECK();
        ure.alloc((size_t)Tu * 8);
        uim.alloc((size_t)Tu * 8);
        k_combine<<<blocks_for(Tu, 256), 256, 0, s>>>(starts.as<int32_t>(), Tu, sre.as<double>(), sim.as<double>(),
                                                      ure.as<double>(), uim.as<double>());
        QSD_LAUNCH_CHECK();
        // diagonal terms (popc F == 0) come first
        DevBuf cnt(8);
        QSD_CUDA(cudaMemsetAsync(cnt.p, 0, 8, s));
        k_count_zero<<<blocks_for(Tu, 256), 256, 0, s>>>(ukeys.as<uint64_t>() + (size_t)(5 * W) * Tu, Tu,
                                                         cnt.as<unsigned long long>());
        QSD_LAUNCH_CHECK();
        unsigned long long h_cnt = 0;
        QSD_CUDA(cudaMemcpyAsync(&h_cnt, cnt.p, 8, cudaMemcpyDeviceToHost, s));
        // coefficient magnitudes and Hermiticity over all unique terms
        DevBuf mx(16);
        QSD_CUDA(cudaMemsetAsync(mx.p, 0, 16, s));
        k_absmax<<<blocks_for(Tu, 256), 256, 0, s>>>(ure.as<double>(), uim.as<double>(), Tu, mx.as<unsigned long long>());
        QSD_LAUNCH_CHECK();
        unsigned long long h_mx[2];
        QSD_CUDA(cudaMemcpyAsync(h_mx, mx.p, 16, cudaMemcpyDeviceToHost, s));
        QSD_CUDA(cudaStreamSynchronize(s));
        Td = (int64_t)h_cnt;
        double m0, m1;
        memcpy(&m0, &h_mx[0], 8);
        memcpy(&m1, &h_mx[1], 8);
        maxphi = std::max(maxphi, m0);
        maxim = std::max(maxim, m1);
        const double tol = 1e-14 * std::max(maxphi, 1e-300);
        QSD_CUDA(cudaMemsetAsync(ctx->d_err, 0, 4, s));
        k_hermitian<<<blocks_for(Tu, 128), 128, 0, s>>>(W, Tu, ukeys.as<uint64_t>(), ure.as<double>(), uim.as<double>(),
                                                        tol, ctx->d_err);
        QSD_LAUNCH_CHECK();
        hermitian = hermitian && take_device_error(ctx) == 0;
    }
    const double imag_tol = 1e-14 * std::max(maxphi, 1e-300);
    op->info.is_real = maxim <= imag_tol ? 1 : 0;
    op->info.is_hermitian = hermitian ? 1 : 0;

    // ---- diagonal terms
    op->Td = Td;
    if (Td > 0) {
        op->dP.alloc((size_t)W * Td * 8); op->dV.alloc((size_t)W * Td * 8); op->dZ.alloc((size_t)W * Td * 8);
        op->dphi.alloc((size_t)Td * 8);
        op->dphi_im.alloc((size_t)Td * 8);
        const int nb = blocks_for(Td, 256);
        k_slice_rows<<<nb, 256, 0, s>>>(ukeys.as<uint64_t>(), Tu, 2 * W, W, 0, Td, op->dP.as<uint64_t>());
        k_slice_rows<<<nb, 256, 0, s>>>(ukeys.as<uint64_t>(), Tu, W, W, 0, Td, op->dV.as<uint64_t>());
        k_slice_rows<<<nb, 256, 0, s>>>(ukeys.as<uint64_t>(), Tu, 0, W, 0, Td, op->dZ.as<uint64_t>());
        QSD_CUDA(cudaMemcpyAsync(op->dphi.p, ure.p, (size_t)Td * 8, cudaMemcpyDeviceToDevice, s));
        QSD_CUDA(cudaMemcpyAsync(op->dphi_im.p, uim.p, (size_t)Td * 8, cudaMemcpyDeviceToDevice, s));
        QSD_LAUNCH_CHECK();
    }

    // ---- off-diagonal terms and groups
    const int64_t T = Tu - Td;
    op->T = T;
    int64_t G = 0;
    unsigned long long h_stats[2] = {0, 0};
    if (T > 0) {
        op->tP.alloc((size_t)W * T * 8); op->tV.alloc((size_t)W * T * 8); op->tZ.alloc((size_t)W * T * 8);
        DevBuf tF((size_t)W * T * 8);
        op->tphi.alloc((size_t)T * 8);
        op->tphi_im.alloc((size_t)T * 8);
        op->tflag.alloc((size_t)T);
        const int nb = blocks_for(T, 256);
        k_slice_rows<<<nb, 256, 0, s>>>(ukeys.as<uint64_t>(), Tu, 2 * W, W, Td, T, op->tP.as<uint64_t>());
        k_slice_rows<<<nb, 256, 0, s>>>(ukeys.as<uint64_t>(), Tu, W, W, Td, T, op->tV.as<uint64_t>());
        k_slice_rows<<<nb, 256, 0, s>>>(ukeys.as<uint64_t>(), Tu, 0, W, Td, T, op->tZ.as<uint64_t>());
        k_slice_rows<<<nb, 256, 0, s>>>(ukeys.as<uint64_t>(), Tu, 4 * W, W, Td, T, tF.as<uint64_t>());
        QSD_LAUNCH_CHECK();
        QSD_CUDA(cudaMemcpyAsync(op->tphi.p, ure.as<double>() + Td, (size_t)T * 8, cudaMemcpyDeviceToDevice, s));
        QSD_CUDA(cudaMemcpyAsync(op->tphi_im.p, uim.as<double>() + Td, (size_t)T * 8, cudaMemcpyDeviceToDevice, s));
        k_term_flags<<<nb, 256, 0, s>>>(W, T, op->tP.as<uint64_t>(), op->tZ.as<uint64_t>(), op->tflag.as<uint8_t>());
        QSD_LAUNCH_CHECK();
        // group boundaries: F changes
        DevBuf gfl((size_t)T * 4), gpo((size_t)T * 4);
        k_group_flags<<<nb, 256, 0, s>>>(tF.as<uint64_t>(), T, W, 0, T, gfl.as<uint32_t>());
        QSD_LAUNCH_CHECK();
        G = (int64_t)exclusive_scan_u32(ctx, gfl.as<uint32_t>(), gpo.as<uint32_t>(), T, true);
        op->grange.alloc((size_t)(G + 1) * 4);
        k_group_starts<<<nb, 256, 0, s>>>(gfl.as<uint32_t>(), gpo.as<uint32_t>(), T, G, op->grange.as<int32_t>());
        QSD_LAUNCH_CHECK();
        op->gF.alloc((size_t)W * G * 8);
        op->ghash.alloc((size_t)G * 8);
        op->gL.alloc((size_t)G);
        op->gpos.alloc((size_t)G * 8);
        op->gptr.alloc((size_t)G * kLadderPtrs * 4);
        DevBuf stats(16);
        QSD_CUDA(cudaMemsetAsync(stats.p, 0, 16, s));
        k_group_tables<<<blocks_for(G, 128), 128, 0, s>>>(
            W, G, op->grange.as<int32_t>(), tF.as<uint64_t>(), T, op->tP.as<uint64_t>(), op->tV.as<uint64_t>(),
            ctx->nib.as<uint64_t>(), op->gF.as<uint64_t>(), op->ghash.as<uint64_t>(), op->gL.as<uint8_t>(),
            op->gpos.as<uint64_t>(), op->gptr.as<int32_t>(), stats.as<unsigned long long>(),
            stats.as<unsigned long long>() + 1);
        QSD_LAUNCH_CHECK();
        QSD_CUDA(cudaMemcpyAsync(h_stats, stats.p, 16, cudaMemcpyDeviceToHost, s));
        // amplitude tables for small-support groups, and the group records
        {
            DevBuf size((size_t)G * 4), off((size_t)G * 4), spos((size_t)G * 8);
            k_group_support<<<blocks_for(G, 128), 128, 0, s>>>(W, G, op->grange.as<int32_t>(), op->gF.as<uint64_t>(),
                                                               T, op->tP.as<uint64_t>(), op->tZ.as<uint64_t>(),
                                                               size.as<uint32_t>(), spos.as<uint64_t>());
            QSD_LAUNCH_CHECK();
            op->n_amp = (int64_t)exclusive_scan_u32(ctx, size.as<uint32_t>(), off.as<uint32_t>(), G, true);
            op->amp.alloc((size_t)std::max<int64_t>(op->n_amp, 1) * 8);
            op->ampf.alloc((size_t)std::max<int64_t>(op->n_amp, 1) * 8);
            op->grec.alloc((size_t)G * sizeof(GroupRec));
            k_group_records<<<blocks_for(G, 128), 128, 0, s>>>(
                W, G, op->grange.as<int32_t>(), op->gF.as<uint64_t>(), op->ghash.as<uint64_t>(), T,
                op->tP.as<uint64_t>(), op->tV.as<uint64_t>(), op->tZ.as<uint64_t>(), op->tphi.as<double>(),
                size.as<uint32_t>(), off.as<uint32_t>(), spos.as<uint64_t>(), op->amp.as<double>(),
                op->ampf.as<float2>(), op->grec.as<GroupRec>());
            QSD_LAUNCH_CHECK();
            std::vector<uint32_t> hsz(G);
            QSD_CUDA(cudaMemcpyAsync(hsz.data(), size.p, (size_t)G * 4, cudaMemcpyDeviceToHost, s));
            QSD_CUDA(cudaStreamSynchronize(s));
            op->n_table_groups = 0;
            op->max_table_size = 0;
            op->min_table_size = G > 0 ? (int64_t)1 << 62 : 0;
            for (auto v : hsz) {
                op->n_table_groups += v > 0;
                op->max_table_size = std::max<int64_t>(op->max_table_size, v);
                op->min_table_size = std::min<int64_t>(op->min_table_size, v);
            }
        }
        op->host_groups.resize((size_t)G * W);
        std::vector<uint64_t> gsoa((size_t)G * W);
        QSD_CUDA(cudaMemcpyAsync(gsoa.data(), op->gF.p, (size_t)G * W * 8, cudaMemcpyDeviceToHost, s));
        QSD_CUDA(cudaStreamSynchronize(s));
        for (int64_t g = 0; g < G; ++g)
            for (int w = 0; w < W; ++w) op->host_groups[(size_t)g * W + w] = gsoa[(size_t)w * G + g];
    }
    op->G = G;
    build_excitation_index(ctx, op);
    qsd_op_info &I = op->info;
    I.n_qubits = n;
    I.n_words = W;
    I.n_terms_in = Ti;
    I.n_terms = T;
    I.n_diag_terms = Td;
    I.n_groups = G;
    I.max_group_terms = (int64_t)h_stats[0];
    I.n_ladder_groups = (int64_t)h_stats[1];
    I.identity_coef = id_re;
    I.n_excitation_groups = op->exc_ok ? op->G_exc : 0;
    I.n_excitation_shapes = op->exc_ok ? op->n_shapes : 0;
    I.excitation_rank_index = (op->exc_ok && op->dense_ok) ? 1 : 0;
    I.n_linear_ranges = op->n_lin_rows;
    QSD_CUDA(cudaStreamSynchronize(s));
}

void compute_diagonal(qsd_ctx ctx, qsd_op op, qsd_sub sub, double *d) {
    compute_diagonal_on(ctx, op, sub, d, ctx->stream);
}

void compute_diagonal_on(qsd_ctx ctx, qsd_op op, qsd_sub sub, double *d, cudaStream_t s) {
    (void)ctx;
    const int64_t D = sub->D;
    if (D <= 0) return;
    const int nb = blocks_for(D, 256);
    const uint64_t *P = op->dP.as<uint64_t>(), *V = op->dV.as<uint64_t>(), *Z = op->dZ.as<uint64_t>();
    const double *phi = op->dphi.as<double>();
    const uint64_t *keys = sub->keys.as<uint64_t>();
    switch (op->W) {
    case 1: k_diagonal<1><<<nb, 256, 0, s>>>(keys, D, op->identity, op->Td, P, V, Z, phi, d); break;
    case 2: k_diagonal<2><<<nb, 256, 0, s>>>(keys, D, op->identity, op->Td, P, V, Z, phi, d); break;
    case 3: k_diagonal<3><<<nb, 256, 0, s>>>(keys, D, op->identity, op->Td, P, V, Z, phi, d); break;
    case 4: k_diagonal<4><<<nb, 256, 0, s>>>(keys, D, op->identity, op->Td, P, V, Z, phi, d); break;
    default: k_diagonal_dyn<<<nb, 256, 0, s>>>(keys, op->W, D, op->identity, op->Td, P, V, Z, phi, d);
    }
    QSD_LAUNCH_CHECK();
}

void target_table(qsd_ctx ctx, qsd_op op, qsd_sub sub, int64_t row0, int64_t nrows, int64_t *out) {
    const int64_t G = op->G;
    if (nrows <= 0 || G <= 0) return;
    cudaStream_t s = ctx->stream;
    const int64_t total = nrows * G;
    const int nb = blocks_for(total, 256);
    const HashView hv = hash_view(sub);
    const uint64_t *keys = sub->keys.as<uint64_t>(), *nib = ctx->nib.as<uint64_t>();
#define QSD_TT(WW)                                                                                             \
    k_target_table<WW><<<nb, 256, 0, s>>>(keys, sub->D, hv, nib, G, op->gF.as<uint64_t>(),                 \
                                          op->ghash.as<uint64_t>(), op->grange.as<int32_t>(), op->gL.as<uint8_t>(), \
                                          op->gpos.as<uint64_t>(), op->gptr.as<int32_t>(), op->T,              \
                                          op->tP.as<uint64_t>(), op->tV.as<uint64_t>(), row0, nrows, out, ctx->d_err)
    switch (op->W) {
    case 1: QSD_TT(1); break;
    case 2: QSD_TT(2); break;
    case 3: QSD_TT(3); break;
    case 4: QSD_TT(4); break;
    default:
        k_target_table_dyn<<<nb, 256, 0, s>>>(keys, op->W, sub->D, hv, nib, G, op->gF.as<uint64_t>(),
                                              op->ghash.as<uint64_t>(), op->grange.as<int32_t>(), op->T,
                                              op->tP.as<uint64_t>(), op->tV.as<uint64_t>(), row0, nrows, out,
                                              ctx->d_err);
    }
#undef QSD_TT
    QSD_LAUNCH_CHECK();
}

void term_table(qsd_ctx ctx, qsd_op op, qsd_sub sub, int64_t row0, int64_t nrows, int8_t *out) {
    const int64_t Ti = op->T_in;
    if (nrows <= 0 || Ti <= 0) return;
    const int64_t total = nrows * Ti;
    k_term_table<<<blocks_for(total, 256), 256, 0, ctx->stream>>>(
        sub->keys.as<uint64_t>(), op->W, sub->D, row0, nrows, Ti, op->iP.as<uint64_t>(), op->iV.as<uint64_t>(),
        op->iZ.as<uint64_t>(), op->iY.as<uint8_t>(), out);
    QSD_LAUNCH_CHECK();
}

}  // namespace qsd
