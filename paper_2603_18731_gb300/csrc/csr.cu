// Explicit CSR form of H_S (Methods, "Matrix evaluation", two-pass build;
// Supplementary "Lower / upper triangle evaluation" and "Most-significant
// off-diagonal bit").
//
// Pass 1 counts, per row, the off-diagonal entries the row evaluates; pass 2
// evaluates them again and writes them straight into the caller's arrays.
// With the triangle option a row r evaluates only the groups whose most
// significant flipped qubit (MSOB) is set in r: the column r xor F then has
// that bit cleared and every higher bit equal, so it is a smaller integer,
// hence (the subspace is indexed in integer order) a smaller index -- a
// lower-triangle entry, found without forming the column.  Each lower entry
// (r, c, h) also gives the upper entry (c, r, conj h) of the Hermitian matrix;
// pass 1 counts those per receiving row too, so every row's segment is known
// before pass 2: [entries the row evaluated | diagonal | mirrored entries].
// Pass 3 sorts each segment by column (a thread per short row, a block per
// long row; rows longer than one block sorts fall back to a device radix sort
// of (row, column) keys).  Columns are unique within a row, so the result does
// not depend on the order in which rows wrote their entries.
//
// A row's structure is its diagonal (always stored) plus every column in S
// reached by at least one term that passes its projector test; values are
// kept even when the terms cancel.
#include "qsd_internal.cuh"

namespace qsd {

namespace {

constexpr int kShortRow = 32;    // rows up to this length: insertion sort by one thread
constexpr int kLongRow = 4096;   // rows up to this length: bitonic sort by one block

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
    const double *diag;     // [D]
    uint32_t *cnt;          // [D] entries the row evaluates (pass 1 writes)
    uint32_t *cnt_up;       // [D] mirrored entries the row receives (pass 1 counts)
    const uint32_t *off;    // [D] first entry of the row's segment (pass 2)
    uint32_t *cursor;       // [D] mirrored entries written so far (pass 2)
    void *indices;          // int32 or int64 [nnz]
    double *data_re, *data_im;
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
// FILL: 0 = pass 1 (count), 32 / 64 = pass 2 with that index width.
template <int W, bool LOWER, int FILL>
__global__ void __launch_bounds__(256) k_csr_rows(const CsrParams c) {
    using IDX = typename std::conditional<FILL == 64, int64_t, int32_t>::type;
    constexpr int NW = W ? W : kMaxWordsDyn;
    const int nw = W ? W : c.W;
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= c.D) return;
    uint64_t key[NW], col[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w)
        if (w < nw) key[w] = __ldg(c.keys + (size_t)w * c.D + row);
    const uint64_t hr = key_hash_dyn(key, nw, c.nib);
    IDX *ind = static_cast<IDX *>(c.indices);
    uint32_t n = 0;
    const uint32_t lim = FILL ? c.cnt[row] : 0u;
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
            if (FILL && c.data_im) im += s * __ldg(c.tphi_im + t);
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
            if (n >= lim) {
                atomicOr(c.err, 2u);
                break;
            }
            ind[base + n] = (IDX)idx;
            c.data_re[base + n] = re;
            if (c.data_im) c.data_im[base + n] = im;
            if (LOWER) {
                const uint32_t slot = atomicAdd(c.cursor + idx, 1u);
                if (slot < c.cnt_up[idx]) {
                    const int64_t at = (int64_t)c.off[idx] + c.cnt[idx] + 1 + slot;
                    ind[at] = (IDX)row;
                    c.data_re[at] = re;
                    if (c.data_im) c.data_im[at] = -im;
                } else {
                    atomicOr(c.err, 2u);
                }
            }
        } else if (LOWER) {
            atomicAdd(c.cnt_up + idx, 1u);
        }
        ++n;
    }
    if (!FILL) {
        c.cnt[row] = n;
    } else {
        const int64_t at = base + lim;
        ind[at] = (IDX)row;
        c.data_re[at] = c.diag[row];
        if (c.data_im) c.data_im[at] = 0.0;
    }
}

__global__ void k_row_len(int64_t D, const uint32_t *__restrict__ cnt, const uint32_t *__restrict__ cnt_up,
                          uint32_t *len) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < D) len[r] = cnt[r] + 1u + (cnt_up ? cnt_up[r] : 0u);
}

__global__ void k_indptr(int64_t D, const uint32_t *__restrict__ off, int64_t nnz, int64_t *indptr) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < D) indptr[r] = off[r];
    if (r == D) indptr[D] = nnz;
}

// Short rows: insertion sort by one thread; longer rows are listed.
template <typename IDX>
__global__ void k_sort_short(int64_t D, const uint32_t *__restrict__ off, const uint32_t *__restrict__ len,
                             IDX *ind, double *re, double *im, uint32_t *long_rows, uint32_t *n_long) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= D) return;
    const uint32_t L = len[r];
    if (L > (uint32_t)kShortRow) {
        long_rows[atomicAdd(n_long, 1u)] = (uint32_t)r;
        return;
    }
    const int64_t b = off[r];
    for (uint32_t i = 1; i < L; ++i) {
        const IDX k = ind[b + i];
        const double vr = re[b + i], vi = im ? im[b + i] : 0.0;
        int64_t j = (int64_t)i - 1;
        while (j >= 0 && ind[b + j] > k) {
            ind[b + j + 1] = ind[b + j];
            re[b + j + 1] = re[b + j];
            if (im) im[b + j + 1] = im[b + j];
            --j;
        }
        ind[b + j + 1] = k;
        re[b + j + 1] = vr;
        if (im) im[b + j + 1] = vi;
    }
}

// Long rows (up to kLongRow): one block per listed row, bitonic sort of
// (column << 16 | position) keys in shared memory, then a permuted write.
template <typename IDX>
__global__ void __launch_bounds__(512) k_sort_long(const uint32_t *__restrict__ rows, const uint32_t *__restrict__ off,
                                                   const uint32_t *__restrict__ len, IDX *ind, double *re,
                                                   double *im, uint32_t *err) {
    extern __shared__ uint64_t sm[];
    uint64_t *sk = sm;                                        // [kLongRow]
    double *sre = reinterpret_cast<double *>(sm + kLongRow);  // [kLongRow]
    double *sim = sre + kLongRow;                             // [kLongRow]
    const uint32_t r = rows[blockIdx.x];
    const uint32_t L = len[r];
    if (L > (uint32_t)kLongRow) {
        if (threadIdx.x == 0) atomicOr(err, 4u);
        return;  // block-uniform
    }
    const int64_t b = off[r];
    uint32_t P = 1;
    while (P < L) P <<= 1;
    for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
        if (i < L) {
            sk[i] = ((uint64_t)(uint32_t)ind[b + i] << 16) | i;
            sre[i] = re[b + i];
            sim[i] = im ? im[b + i] : 0.0;
        } else {
            sk[i] = ~0ull;
        }
    }
    __syncthreads();
    for (uint32_t k = 2; k <= P; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
                const uint32_t p = i ^ j;
                if (p > i) {
                    const uint64_t a = sk[i], c = sk[p];
                    const bool up = (i & k) == 0;
                    if ((a > c) == up) {
                        sk[i] = c;
                        sk[p] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (uint32_t i = threadIdx.x; i < L; i += blockDim.x) {
        const uint32_t src = (uint32_t)(sk[i] & 0xffffu);
        ind[b + i] = (IDX)(sk[i] >> 16);
        re[b + i] = sre[src];
        if (im) im[b + i] = sim[src];
    }
}

// Fallback for rows longer than kLongRow: (row << 32 | column) keys of every
// entry, sorted on the device; values follow through the permutation.
template <typename IDX>
__global__ void k_entry_keys(int64_t D, const uint32_t *__restrict__ off, const uint32_t *__restrict__ len,
                             const IDX *__restrict__ ind, uint64_t *keys, uint32_t *perm) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= D) return;
    const int64_t b = off[r];
    for (uint32_t i = 0; i < len[r]; ++i) {
        keys[b + i] = ((uint64_t)r << 32) | (uint64_t)(uint32_t)ind[b + i];
        perm[b + i] = (uint32_t)(b + i);
    }
}

template <typename IDX>
__global__ void k_entry_gather(int64_t nnz, const uint64_t *__restrict__ keys, const uint32_t *__restrict__ perm,
                               const double *__restrict__ re0, const double *__restrict__ im0, IDX *ind, double *re,
                               double *im) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nnz) return;
    ind[i] = (IDX)(keys[i] & 0xffffffffull);
    re[i] = re0[perm[i]];
    if (im) im[i] = im0[perm[i]];
}

template <bool LOWER, int FILL>
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

template <typename IDX>
void sort_rows(qsd_ctx ctx, int64_t D, int64_t nnz, const uint32_t *off, const uint32_t *len, IDX *ind, double *re,
               double *im) {
    cudaStream_t s = ctx->stream;
    DevBuf rows, n_long;
    rows.alloc_async((size_t)D * 4, s);
    n_long.alloc_async(4, s);
    QSD_CUDA(cudaMemsetAsync(n_long.p, 0, 4, s));
    k_sort_short<IDX><<<blocks_for(D, 256), 256, 0, s>>>(D, off, len, ind, re, im, rows.as<uint32_t>(),
                                                         n_long.as<uint32_t>());
    QSD_LAUNCH_CHECK();
    uint32_t h_long = 0;
    QSD_CUDA(cudaMemcpyAsync(&h_long, n_long.p, 4, cudaMemcpyDeviceToHost, s));
    QSD_CUDA(cudaStreamSynchronize(s));
    if (h_long == 0) return;
    const size_t smem = (size_t)kLongRow * 24;
    QSD_CUDA(cudaFuncSetAttribute(k_sort_long<IDX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    QSD_CUDA(cudaMemsetAsync(ctx->d_err, 0, 4, s));
    k_sort_long<IDX><<<h_long, 512, smem, s>>>(rows.as<uint32_t>(), off, len, ind, re, im, ctx->d_err);
    QSD_LAUNCH_CHECK();
    if (!(take_device_error(ctx) & 4u)) return;
    // some row is longer than one block sorts: sort all entries by (row, column)
    DevBuf keys((size_t)nnz * 8), perm((size_t)nnz * 4), re0((size_t)nnz * 8), im0(im ? (size_t)nnz * 8 : 0);
    k_entry_keys<IDX><<<blocks_for(D, 256), 256, 0, s>>>(D, off, len, ind, keys.as<uint64_t>(), perm.as<uint32_t>());
    QSD_LAUNCH_CHECK();
    QSD_CUDA(cudaMemcpyAsync(re0.p, re, (size_t)nnz * 8, cudaMemcpyDeviceToDevice, s));
    if (im) QSD_CUDA(cudaMemcpyAsync(im0.p, im, (size_t)nnz * 8, cudaMemcpyDeviceToDevice, s));
    radix_sort(ctx, keys.as<uint64_t>(), 1, nnz, perm.as<uint32_t>());
    k_entry_gather<IDX><<<blocks_for(nnz, 256), 256, 0, s>>>(nnz, keys.as<uint64_t>(), perm.as<uint32_t>(),
                                                             re0.as<double>(), im ? im0.as<double>() : nullptr, ind,
                                                             re, im);
    QSD_LAUNCH_CHECK();
    QSD_CUDA(cudaStreamSynchronize(s));
}

}  // namespace

// Pass 1: per-row counts and segment offsets into ctx->csr (kept for the
// filling call).
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
    const size_t n4 = (size_t)std::max<int64_t>(D, 1) * 4;
    // stream-ordered: no device-wide synchronisation for the temporaries
    st.cnt.alloc_async(n4, s);
    st.cnt_up.alloc_async(n4, s);
    st.len.alloc_async(n4, s);
    st.off.alloc_async(n4, s);
    int64_t nnz = 0;
    if (D > 0) {
        QSD_CUDA(cudaMemsetAsync(st.cnt.p, 0, n4, s));
        QSD_CUDA(cudaMemsetAsync(st.cnt_up.p, 0, n4, s));
        if (op->G > 0) {
            CsrParams c = make_csr_params(ctx, op, sub);
            c.cnt = st.cnt.as<uint32_t>();
            c.cnt_up = st.cnt_up.as<uint32_t>();
            if (lower) launch_rows<true, 0>(c, s);
            else launch_rows<false, 0>(c, s);
        }
        k_row_len<<<blocks_for(D, 256), 256, 0, s>>>(D, st.cnt.as<uint32_t>(), lower ? st.cnt_up.as<uint32_t>() : nullptr,
                                                     st.len.as<uint32_t>());
        QSD_LAUNCH_CHECK();
        nnz = (int64_t)exclusive_scan_u32(ctx, st.len.as<uint32_t>(), st.off.as<uint32_t>(), D, true);
    }
    if (take_device_error(ctx)) fail(QSD_ERR_INTERNAL, "qsd_to_csr: hash probe ran past the table");
    if (nnz >= (int64_t)0xffffffffLL)
        fail(QSD_ERR_CAPACITY, "qsd_to_csr: " + std::to_string(nnz) + " entries (limit 2^32 - 1)");
    st.op = op;
    st.sub = sub;
    st.lower = lower;
    st.nnz = nnz;
}

int64_t to_csr(qsd_ctx ctx, qsd_op op, qsd_sub sub, bool lower, int64_t *indptr, void *indices, int index_bits,
               double *data_re, double *data_im, const double *diag) {
    CsrState &st = ctx->csr;
    const bool sizing = !indptr && !indices && !data_re;
    if (!(st.op == op && st.sub == sub && st.lower == lower && st.nnz >= 0)) csr_count(ctx, op, sub, lower);
    const int64_t nnz = st.nnz, D = sub->D;
    if (sizing) return nnz;
    cudaStream_t s = ctx->stream;
    if (D == 0) {
        QSD_CUDA(cudaMemsetAsync(indptr, 0, 8, s));
        QSD_CUDA(cudaStreamSynchronize(s));
        st.clear();
        return 0;
    }
    CsrParams c = make_csr_params(ctx, op, sub);
    c.diag = diag;
    c.cnt = st.cnt.as<uint32_t>();
    c.cnt_up = st.cnt_up.as<uint32_t>();
    c.off = st.off.as<uint32_t>();
    DevBuf cursor;
    cursor.alloc_async((size_t)D * 4, s);
    QSD_CUDA(cudaMemsetAsync(cursor.p, 0, (size_t)D * 4, s));
    c.cursor = cursor.as<uint32_t>();
    c.indices = indices;
    c.data_re = data_re;
    c.data_im = data_im;
    if (index_bits == 32) {
        if (lower) launch_rows<true, 32>(c, s);
        else launch_rows<false, 32>(c, s);
    } else {
        if (lower) launch_rows<true, 64>(c, s);
        else launch_rows<false, 64>(c, s);
    }
    k_indptr<<<blocks_for(D + 1, 256), 256, 0, s>>>(D, st.off.as<uint32_t>(), nnz, indptr);
    QSD_LAUNCH_CHECK();
    if (const uint32_t e = take_device_error(ctx))
        fail(QSD_ERR_INTERNAL, (e & 2u) ? "qsd_to_csr: pass 2 found other entries than pass 1"
                                        : "qsd_to_csr: hash probe ran past the table");
    if (index_bits == 32)
        sort_rows<int32_t>(ctx, D, nnz, st.off.as<uint32_t>(), st.len.as<uint32_t>(), static_cast<int32_t *>(indices),
                           data_re, data_im);
    else
        sort_rows<int64_t>(ctx, D, nnz, st.off.as<uint32_t>(), st.len.as<uint32_t>(), static_cast<int64_t *>(indices),
                           data_re, data_im);
    st.clear();
    return nnz;
}

}  // namespace qsd
