// Explicit CSR form of H_S (Methods, "Matrix evaluation", two-pass build;
// Supplementary "Lower / upper triangle evaluation" and "Most-significant
// off-diagonal bit").
//
// Pass 1 counts, per row, the off-diagonal entries the row evaluates; pass 2
// evaluates them again and writes (row, column, value).  With the triangle
// option a row r evaluates only the groups whose most significant flipped
// qubit (MSOB) is set in r: the column r xor F then has that bit cleared and
// every higher bit equal, so it is a smaller integer, hence (the subspace is
// indexed in integer order) a smaller index -- a lower-triangle entry, found
// without forming the column.  Each lower entry (r, c, h) also gives the
// upper entry (c, r, conj h) of the Hermitian matrix.
//
// Entries are written as 64-bit keys (row << 32 | column) in any order and
// then radix sorted on the device; keys are unique, so the result does not
// depend on the order the rows wrote them.  A row's structure is its diagonal
// (always stored) plus every column in S reached by at least one term that
// passes its projector test; values are kept even when the terms cancel.
#include "qsd_internal.cuh"

namespace qsd {

namespace {

struct CsrParams {
    const uint64_t *keys;  // [W][D]
    int64_t D;
    int W;
    HashView hv;
    const uint64_t *nib;
    int64_t G;
    const uint64_t *gF;     // [W][G]
    const uint64_t *ghash;  // [G]
    const int32_t *grange;  // [G+1]
    const uint8_t *gL;
    const uint64_t *gpos;
    const int32_t *gptr;
    const uint16_t *msob;   // [G]
    int64_t T;
    const uint64_t *tP, *tV, *tZ;
    const double *tphi, *tphi_im;
    const uint8_t *tflag;
    uint32_t *cnt;          // pass 1 writes, pass 2 reads: entries per row
    const uint32_t *off;    // pass 2: first entry of the row
    int64_t L;              // pass 2: total lower entries (mirror offset)
    uint64_t *ekey;
    double *ere, *eim;
    uint32_t *err;
};

// Most significant set bit of each group's flip mask.
__global__ void k_group_msob(int W, int64_t G, const uint64_t *__restrict__ gF, uint16_t *msob) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    int m = 0;
    for (int w = 0; w < W; ++w) {
        const uint64_t f = gF[(size_t)w * G + g];
        if (f) m = 64 * w + 63 - __clzll((long long)f);
    }
    msob[g] = (uint16_t)m;
}

// One thread per row.  W > 0: unrolled keys; W == 0: run-time c.W.
template <int W, bool LOWER, bool FILL>
__global__ void __launch_bounds__(256) k_csr_rows(const CsrParams c) {
    constexpr int NW = W ? W : kMaxWordsDyn;
    const int nw = W ? W : c.W;
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= c.D) return;
    uint64_t key[NW], col[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w)
        if (w < nw) key[w] = __ldg(c.keys + (size_t)w * c.D + row);
    const uint64_t hr = prehash_dyn(key, nw, c.nib);
    uint32_t n = 0;
    const int64_t base = FILL ? (int64_t)c.off[row] : 0;
    for (int64_t g = 0; g < c.G; ++g) {
        if (LOWER) {
            const int q = __ldg(c.msob + g);
            uint64_t kw = key[0];
#pragma unroll
            for (int w = 1; w < NW; ++w)
                if (w < nw && (q >> 6) == w) kw = key[w];
            if (!((kw >> (q & 63)) & 1)) continue;
        }
        int32_t b, e;
        const int Lb = __ldg(c.gL + g);
        if (Lb) {
            const uint64_t pos = __ldg(c.gpos + g);
            int l = 0;
            for (int i = 0; i < Lb; ++i) {
                const int q = (int)((pos >> (16 * i)) & 0xffff);
                uint64_t kw = key[0];
#pragma unroll
                for (int w = 1; w < NW; ++w)
                    if (w < nw && (q >> 6) == w) kw = key[w];
                l |= (int)((kw >> (q & 63)) & 1) << i;
            }
            b = __ldg(c.gptr + g * 17 + l);
            e = __ldg(c.gptr + g * 17 + l + 1);
        } else {
            b = __ldg(c.grange + g);
            e = __ldg(c.grange + g + 1);
        }
        bool pass = false;
        double re = 0.0, im = 0.0;
        for (int32_t t = b; t < e; ++t) {
            const uint8_t f = __ldg(c.tflag + t);
            bool ok = true;
            int par = 0;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                if (w >= nw) break;
                if (f & 1) ok &= (key[w] & __ldg(c.tP + (size_t)w * c.T + t)) == __ldg(c.tV + (size_t)w * c.T + t);
                if (f & 2) par ^= __popcll(key[w] & __ldg(c.tZ + (size_t)w * c.T + t));
            }
            if (!ok) continue;
            pass = true;
            const double s = (par & 1) ? -1.0 : 1.0;
            re += s * __ldg(c.tphi + t);
            if (FILL && c.eim) im += s * __ldg(c.tphi_im + t);
        }
        if (!pass) continue;
#pragma unroll
        for (int w = 0; w < NW; ++w)
            if (w < nw) col[w] = key[w] ^ __ldg(c.gF + (size_t)w * c.G + g);
        int64_t idx;
        if constexpr (W > 0) {
            uint64_t cc[W];
#pragma unroll
            for (int w = 0; w < W; ++w) cc[w] = col[w];
            idx = probe<W>(cc, hr ^ __ldg(c.ghash + g), c.hv, c.err);
        } else {
            idx = probe_dyn(col, nw, hr ^ __ldg(c.ghash + g), c.hv, c.err);
        }
        if (idx < 0) continue;
        if (FILL) {
            // pass 2 reaches the entries pass 1 counted; never write past them
            if (n >= __ldg(c.cnt + row)) {
                atomicOr(c.err, 2u);
                break;
            }
            const int64_t at = base + n;
            c.ekey[at] = ((uint64_t)row << 32) | (uint64_t)idx;
            c.ere[at] = re;
            if (c.eim) c.eim[at] = im;
            if (LOWER) {
                c.ekey[c.L + at] = ((uint64_t)idx << 32) | (uint64_t)row;
                c.ere[c.L + at] = re;
                if (c.eim) c.eim[c.L + at] = -im;
            }
        }
        ++n;
    }
    if (!FILL) c.cnt[row] = n;
}

__global__ void k_csr_diag(int64_t D, const double *__restrict__ diag, int64_t at, uint64_t *ekey, double *ere,
                           double *eim, uint32_t *perm, int64_t nnz) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < D) {
        ekey[at + r] = ((uint64_t)r << 32) | (uint64_t)r;
        ere[at + r] = diag[r];
        if (eim) eim[at + r] = 0.0;
    }
    // the sort's payload: original positions
    for (int64_t i = r; i < nnz; i += (int64_t)gridDim.x * blockDim.x) perm[i] = (uint32_t)i;
}

template <typename IDX>
__global__ void k_csr_out(int64_t nnz, int64_t D, const uint64_t *__restrict__ ekey, const uint32_t *__restrict__ perm,
                          const double *__restrict__ ere, const double *__restrict__ eim, int64_t *indptr, IDX *indices,
                          double *data_re, double *data_im) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nnz) return;
    const uint64_t k = ekey[i];
    const int64_t r = (int64_t)(k >> 32);
    indices[i] = (IDX)(k & 0xffffffffull);
    const uint32_t src = perm[i];
    data_re[i] = ere[src];
    if (data_im) data_im[i] = eim ? eim[src] : 0.0;
    // every row holds its diagonal, so every row starts somewhere
    if (i == 0 || (ekey[i - 1] >> 32) != (uint64_t)r) indptr[r] = i;
    if (i == nnz - 1) indptr[D] = nnz;
}

template <bool LOWER, bool FILL>
void launch_rows(const CsrParams &c, cudaStream_t s) {
    const int blocks = blocks_for(c.D, 256);
    switch (c.W) {
    case 1: k_csr_rows<1, LOWER, FILL><<<blocks, 256, 0, s>>>(c); break;
    case 2: k_csr_rows<2, LOWER, FILL><<<blocks, 256, 0, s>>>(c); break;
    case 3: k_csr_rows<3, LOWER, FILL><<<blocks, 256, 0, s>>>(c); break;
    case 4: k_csr_rows<4, LOWER, FILL><<<blocks, 256, 0, s>>>(c); break;
    default: k_csr_rows<0, LOWER, FILL><<<blocks, 256, 0, s>>>(c); break;
    }
    QSD_LAUNCH_CHECK();
}

CsrParams make_csr_params(qsd_ctx ctx, qsd_op op, qsd_sub sub) {
    CsrParams c{};
    c.keys = sub->keys.as<uint64_t>();
    c.D = sub->D;
    c.W = op->W;
    c.hv = hash_view(sub);
    c.nib = ctx->nib.as<uint64_t>();
    c.G = op->G;
    c.gF = op->gF.as<uint64_t>();
    c.ghash = op->ghash.as<uint64_t>();
    c.grange = op->grange.as<int32_t>();
    c.gL = op->gL.as<uint8_t>();
    c.gpos = op->gpos.as<uint64_t>();
    c.gptr = op->gptr.as<int32_t>();
    c.msob = op->gmsob.as<uint16_t>();
    c.T = op->T;
    c.tP = op->tP.as<uint64_t>();
    c.tV = op->tV.as<uint64_t>();
    c.tZ = op->tZ.as<uint64_t>();
    c.tphi = op->tphi.as<double>();
    c.tphi_im = op->tphi_im.as<double>();
    c.tflag = op->tflag.as<uint8_t>();
    c.err = ctx->d_err;
    return c;
}

}  // namespace

// Pass 1: per-row counts into ctx->csr (kept for the filling call).
static void csr_count(qsd_ctx ctx, qsd_op op, qsd_sub sub, bool lower) {
    CsrState &st = ctx->csr;
    st.clear();
    cudaStream_t s = ctx->stream;
    const int64_t D = sub->D;
    if (op->G > 0 && !op->gmsob.p) {
        op->gmsob.alloc((size_t)op->G * 2);
        k_group_msob<<<blocks_for(op->G, 256), 256, 0, s>>>(op->W, op->G, op->gF.as<uint64_t>(),
                                                             op->gmsob.as<uint16_t>());
        QSD_LAUNCH_CHECK();
    }
    st.cnt.alloc((size_t)std::max<int64_t>(D, 1) * 4);
    st.off.alloc((size_t)std::max<int64_t>(D, 1) * 4);
    int64_t L = 0;
    if (D > 0 && op->G > 0) {
        CsrParams c = make_csr_params(ctx, op, sub);
        c.cnt = st.cnt.as<uint32_t>();
        if (lower) launch_rows<true, false>(c, s);
        else launch_rows<false, false>(c, s);
        L = (int64_t)exclusive_scan_u32(ctx, st.cnt.as<uint32_t>(), st.off.as<uint32_t>(), D, true);
    }
    if (take_device_error(ctx)) fail(QSD_ERR_INTERNAL, "qsd_to_csr: hash probe ran past the table");
    const int64_t nnz = D + (lower ? 2 * L : L);
    if (nnz >= (int64_t)0xffffffffLL)
        fail(QSD_ERR_CAPACITY, "qsd_to_csr: " + std::to_string(nnz) + " entries (limit 2^32 - 1)");
    st.op = op;
    st.sub = sub;
    st.lower = lower;
    st.L = L;
    st.nnz = nnz;
}

int64_t to_csr(qsd_ctx ctx, qsd_op op, qsd_sub sub, bool lower, int64_t *indptr, void *indices, int index_bits,
               double *data_re, double *data_im, const double *diag) {
    CsrState &st = ctx->csr;
    const bool sizing = !indptr && !indices && !data_re;
    if (!(st.op == op && st.sub == sub && st.lower == lower && st.nnz >= 0)) csr_count(ctx, op, sub, lower);
    const int64_t nnz = st.nnz, D = sub->D, L = st.L;
    if (sizing) return nnz;
    cudaStream_t s = ctx->stream;
    if (D == 0) {
        QSD_CUDA(cudaMemsetAsync(indptr, 0, 8, s));
        QSD_CUDA(cudaStreamSynchronize(s));
        st.clear();
        return 0;
    }
    DevBuf ekey((size_t)nnz * 8), ere((size_t)nnz * 8), eim(data_im ? (size_t)nnz * 8 : 0), perm((size_t)nnz * 4);
    if (L > 0) {
        CsrParams c = make_csr_params(ctx, op, sub);
        c.off = st.off.as<uint32_t>();
        c.cnt = st.cnt.as<uint32_t>();
        c.L = L;
        c.ekey = ekey.as<uint64_t>();
        c.ere = ere.as<double>();
        c.eim = data_im ? eim.as<double>() : nullptr;
        if (lower) launch_rows<true, true>(c, s);
        else launch_rows<false, true>(c, s);
    }
    const int64_t at = lower ? 2 * L : L;
    k_csr_diag<<<blocks_for(D, 256), 256, 0, s>>>(D, diag, at, ekey.as<uint64_t>(), ere.as<double>(),
                                                   data_im ? eim.as<double>() : nullptr, perm.as<uint32_t>(), nnz);
    QSD_LAUNCH_CHECK();
    radix_sort(ctx, ekey.as<uint64_t>(), 1, nnz, perm.as<uint32_t>());
    const int blocks = blocks_for(nnz, 256);
    if (index_bits == 32)
        k_csr_out<int32_t><<<blocks, 256, 0, s>>>(nnz, D, ekey.as<uint64_t>(), perm.as<uint32_t>(), ere.as<double>(),
                                                  data_im ? eim.as<double>() : nullptr, indptr,
                                                  static_cast<int32_t *>(indices), data_re, data_im);
    else
        k_csr_out<int64_t><<<blocks, 256, 0, s>>>(nnz, D, ekey.as<uint64_t>(), perm.as<uint32_t>(), ere.as<double>(),
                                                  data_im ? eim.as<double>() : nullptr, indptr,
                                                  static_cast<int64_t *>(indices), data_re, data_im);
    QSD_LAUNCH_CHECK();
    if (const uint32_t e = take_device_error(ctx))
        fail(QSD_ERR_INTERNAL, (e & 2u) ? "qsd_to_csr: pass 2 found more entries than pass 1"
                                        : "qsd_to_csr: hash probe ran past the table");
    st.clear();
    return nnz;
}

}  // namespace qsd
