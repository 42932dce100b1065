// Excitation index of an operator's ladder groups (built at load time).
//
// The paper rejects groups whose ladder integer has no term before any lookup
// (Methods, "Fermionic Hamiltonians", Fig. 3b) and names bulk rejection of
// groups as future work (Discussion).  Here a row does not visit the groups
// at all: a ladder term is nonzero only where its raising qubits are occupied
// and its lowering qubits empty, so a row enumerates exactly the flip masks of
// that form -- its single and double "excitations" per shape of the operator --
// and finds their groups in a hash table keyed by the flip mask.
#include <algorithm>
#include <cmath>
#include <map>
#include <set>
#include <vector>

#include "excite.cuh"

namespace qsd {

namespace {

// Shape of each term (0xffffffff: not indexable), see excite.cuh.
__global__ void k_term_shapes(int W, int64_t G, const int32_t *__restrict__ grange, const uint64_t *__restrict__ gF,
                              int64_t T, const uint64_t *__restrict__ tP, const uint64_t *__restrict__ tV, int split,
                              uint32_t *shape) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    for (int32_t t = grange[g]; t < grange[g + 1]; ++t) {
        int c[4] = {0, 0, 0, 0};
        bool ladder = true;
        for (int w = 0; w < W; ++w) {
            const uint64_t F = gF[(size_t)w * G + g], P = tP[(size_t)w * T + t], V = tV[(size_t)w * T + t];
            ladder &= (P & F) == F;
            // sector masks of this word
            uint64_t s0 = 0;
            const int lo = 64 * w;
            if (split >= lo + 64) s0 = ~0ull;
            else if (split > lo) s0 = (1ull << (split - lo)) - 1;
            c[0] += __popcll(V & F & s0);
            c[1] += __popcll(F & ~V & s0);
            c[2] += __popcll(V & F & ~s0);
            c[3] += __popcll(F & ~V & ~s0);
        }
        const bool ok = ladder && c[0] <= 2 && c[1] <= 2 && c[2] <= 2 && c[3] <= 2;
        shape[t] = ok ? (uint32_t)(c[0] | (c[1] << 4) | (c[2] << 8) | (c[3] << 12)) : 0xffffffffu;
    }
}

__global__ void k_gather_exc(int W, int64_t G, const int32_t *__restrict__ ids, int64_t n,
                             const uint64_t *__restrict__ gF, uint64_t *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t g = ids[i];
    for (int w = 0; w < W; ++w) out[(size_t)w * n + i] = gF[(size_t)w * G + g];
}

template <int W>
__global__ void k_term_records(int64_t T, const uint64_t *__restrict__ tP, const uint64_t *__restrict__ tV,
                               const uint64_t *__restrict__ tZ, const double *__restrict__ tphi, double scale,
                               TermRec<W> *out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    TermRec<W> r{};
    for (int w = 0; w < W; ++w) {
        r.P[w] = tP[(size_t)w * T + t];
        r.V[w] = tV[(size_t)w * T + t];
        r.Z[w] = tZ[(size_t)w * T + t];
    }
    // fixed point (scale a power of two: the product is exact)
    r.q = __double2ll_rn(tphi[t] * scale);
    out[t] = r;
}

// Fixed-point exponent e of an operator's term phases: the largest e with
// max over groups of sum |phi| * 2^e < 2^62 (at most 2^62 in magnitude for
// any sum of a group's terms), capped at 1000.
int fixed_point_exponent(const std::vector<double> &phi, const std::vector<int32_t> &grange) {
    double m = 0.0;
    for (size_t g = 0; g + 1 < grange.size(); ++g) {
        double s = 0.0;
        for (int32_t t = grange[g]; t < grange[g + 1]; ++t) s += std::fabs(phi[(size_t)t]);
        m = std::max(m, s);
    }
    if (!(m > 0.0)) return 0;
    int ex = 0;
    std::frexp(m, &ex);  // m < 2^ex
    return std::min(1000, 61 - ex);
}

int64_t choose_h(int64_t m, int k) { return k == 0 ? 1 : (k == 1 ? m : m * (m - 1) / 2); }

uint64_t binom_h(uint64_t n, int k) {
    if ((uint64_t)k > n) return 0;
    uint64_t c = 1;
    for (int i = 0; i < k; ++i) c = c * (n - (uint64_t)i) / (uint64_t)(i + 1);
    return c;
}

// Dense rank index: a group's flip mask F has b0 bits in sector 0 and b1 in
// sector 1 (at most 4 each, from at most two raised and two lowered qubits
// per sector); its entry is base(b0, b1) + rank0 * C(n1, b1) + rank1 with
// rank_s = sum_j C(pos_j, j + 1) over the ascending positions of F's bits
// within sector s (the combinatorial number system: a bijection between the
// b-subsets of n positions and [0, C(n, b))).  Built only when all
// signatures together stay within 2^24 entries; a row's candidate then finds
// its group with one load.
void build_dense_index(qsd_ctx ctx, qsd_op op, const std::vector<int32_t> &exc) {
    op->dense_ok = false;
    const int W = op->W, split = op->exc_split;
    const int n0 = split, n1 = op->n_qubits - split;
    std::map<std::pair<int, int>, uint64_t> base;
    uint64_t total = 0;
    for (int i = 0; i < op->n_shapes; ++i) {
        const uint32_t sh = op->shapes[i];
        const int b0 = (int)(sh & 15) + (int)((sh >> 4) & 15), b1 = (int)((sh >> 8) & 15) + (int)((sh >> 12) & 15);
        if (base.count({b0, b1})) continue;
        base[{b0, b1}] = total;
        total += binom_h((uint64_t)n0, b0) * binom_h((uint64_t)n1, b1);
        if (total > (1ull << 24)) return;
    }
    const int64_t n = op->G_exc;
    std::vector<uint64_t> F((size_t)W * n);
    QSD_CUDA(cudaMemcpyAsync(F.data(), op->excF.p, F.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
    QSD_CUDA(cudaStreamSynchronize(ctx->stream));
    std::vector<int32_t> table(std::max<uint64_t>(total, 1), -1);
    for (int64_t i = 0; i < n; ++i) {
        uint64_t rank[2] = {0, 0};
        int b[2] = {0, 0};
        for (int q = 0; q < op->n_qubits; ++q) {
            if (!((F[(size_t)(q >> 6) * n + i] >> (q & 63)) & 1)) continue;
            const int sct = q < split ? 0 : 1;
            const int pos = q - (sct ? split : 0);
            ++b[sct];
            rank[sct] += binom_h((uint64_t)pos, b[sct]);
        }
        auto it = base.find({b[0], b[1]});
        if (it == base.end()) return;  // not reachable from any shape: keep the hash table
        table[it->second + rank[0] * binom_h((uint64_t)n1, b[1]) + rank[1]] = exc[(size_t)i];
    }
    for (int i = 0; i < op->n_shapes; ++i) {
        const uint32_t sh = op->shapes[i];
        const int b0 = (int)(sh & 15) + (int)((sh >> 4) & 15), b1 = (int)((sh >> 8) & 15) + (int)((sh >> 12) & 15);
        op->dbase[i] = (uint32_t)base[{b0, b1}];
        op->dstride[i] = (uint32_t)binom_h((uint64_t)n1, b1);
    }
    op->dense.alloc(table.size() * 4);
    QSD_CUDA(cudaMemcpyAsync(op->dense.p, table.data(), table.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    QSD_CUDA(cudaStreamSynchronize(ctx->stream));
    op->dense_ok = true;
}

// Linear ranges.  A ladder range (group g, pattern l) whose terms each test at
// most one qubit r outside F (a projector, value v_t) and whose Z masks all
// equal one mask Zref except, for a term, at its own r, has an element of the
// form
//   s(row) * (K + sum over the row's occupied qubits r of d_r),
//   s(row) = (-1)^popc(row & Zref),
// with c_t = phi_t, negated when Z_t and Zref differ at r and v_t = 1 (the
// row's bit at r is then 1); K = sum of c_t over the terms without r and over
// those with v_t = 0; d_r = (sum of c_t with v_t = 1 at r) - (sum with
// v_t = 0 at r).
// Single-excitation groups of a two-body fermionic operator are of this kind:
// a constant plus one coefficient per occupied orbital, up to the sign of the
// Jordan-Wigner string.  Tabulated, in the fixed point of the term records,
// for the groups whose ranges are all linear and hold at least
// kLinearMinTerms terms somewhere; the table sums the same integers q_t as
// the term loop, so it gives the same element.
constexpr int kLinearMinTerms = 6;

void build_linear_ranges(qsd_ctx ctx, qsd_op op, const std::vector<int32_t> &exc, const std::vector<double> &phi,
                         double scale) {
    const int W = op->W, n = op->n_qubits;
    const int64_t G = op->G, T = op->T;
    cudaStream_t s = ctx->stream;
    std::vector<uint8_t> gL((size_t)G);
    std::vector<int32_t> gptr((size_t)G * 17);
    std::vector<uint64_t> gF((size_t)W * G), tP((size_t)W * T), tV((size_t)W * T), tZ((size_t)W * T);
    QSD_CUDA(cudaMemcpyAsync(gL.data(), op->gL.p, (size_t)G, cudaMemcpyDeviceToHost, s));
    QSD_CUDA(cudaMemcpyAsync(gptr.data(), op->gptr.p, (size_t)G * 17 * 4, cudaMemcpyDeviceToHost, s));
    QSD_CUDA(cudaMemcpyAsync(gF.data(), op->gF.p, (size_t)W * G * 8, cudaMemcpyDeviceToHost, s));
    QSD_CUDA(cudaMemcpyAsync(tP.data(), op->tP.p, (size_t)W * T * 8, cudaMemcpyDeviceToHost, s));
    QSD_CUDA(cudaMemcpyAsync(tV.data(), op->tV.p, (size_t)W * T * 8, cudaMemcpyDeviceToHost, s));
    QSD_CUDA(cudaMemcpyAsync(tZ.data(), op->tZ.p, (size_t)W * T * 8, cudaMemcpyDeviceToHost, s));
    QSD_CUDA(cudaStreamSynchronize(s));
    std::vector<int32_t> base((size_t)G, -1);
    std::vector<uint64_t> zref;
    std::vector<int64_t> kq, dq;
    int64_t rows = 0;
    auto word = [&](const std::vector<uint64_t> &a, int w, int64_t t) { return a[(size_t)w * T + t]; };
    for (int32_t g : exc) {
        const int L = gL[(size_t)g];
        if (L == 0) continue;
        const int npat = 1 << L;
        int maxlen = 0;
        bool linear = true;
        // per pattern: Zref, the Z mask of a term without a projector outside
        // F (else of the first term); every term's Z may differ from it only
        // on the term's own projector qubit
        std::vector<uint64_t> Z((size_t)npat * W, 0);
        for (int l = 0; l < npat && linear; ++l) {
            const int32_t b = gptr[(size_t)g * 17 + l], e = gptr[(size_t)g * 17 + l + 1];
            maxlen = std::max(maxlen, (int)(e - b));
            if (e <= b) continue;
            int32_t tref = b;
            for (int32_t t = b; t < e && linear; ++t) {
                int extra = 0;
                for (int w = 0; w < W; ++w) extra += __builtin_popcountll(word(tP, w, t) & ~gF[(size_t)w * G + g]);
                if (extra > 1) linear = false;
                if (extra == 0 && tref == b) tref = t;
            }
            for (int w = 0; w < W; ++w) Z[(size_t)l * W + w] = word(tZ, w, tref);
            for (int32_t t = b; t < e && linear; ++t)
                for (int w = 0; w < W; ++w) {
                    const uint64_t own = word(tP, w, t) & ~gF[(size_t)w * G + g];
                    if ((word(tZ, w, t) ^ Z[(size_t)l * W + w]) & ~own) linear = false;
                }
        }
        if (!linear || maxlen < kLinearMinTerms) continue;
        base[(size_t)g] = (int32_t)rows;
        for (int l = 0; l < npat; ++l) {
            const int32_t b = gptr[(size_t)g * 17 + l], e = gptr[(size_t)g * 17 + l + 1];
            int64_t Kq = 0;
            std::vector<int64_t> dqq((size_t)n, 0);
            for (int32_t t = b; t < e; ++t) {
                int r = -1;
                bool v = false, zdiff = false;
                for (int w = 0; w < W; ++w) {
                    const uint64_t own = word(tP, w, t) & ~gF[(size_t)w * G + g];
                    if (own) {
                        r = 64 * w + __builtin_ctzll(own);
                        v = (word(tV, w, t) & own) != 0;
                        zdiff = ((word(tZ, w, t) ^ Z[(size_t)l * W + w]) & own) != 0;
                    }
                }
                // popc(row & Z_t) = popc(row & Zref) + (Z_t xor Zref at r) * row_r, and
                // row_r = v where the term survives
                const bool neg = r >= 0 && v && zdiff;
                const int64_t q0 = std::llrint(phi[(size_t)t] * scale);
                const int64_t cq = neg ? -q0 : q0;
                if (r < 0) {
                    Kq += cq;
                } else if (v) {
                    dqq[(size_t)r] += cq;
                } else {
                    Kq += cq;
                    dqq[(size_t)r] -= cq;
                }
            }
            for (int w = 0; w < W; ++w) zref.push_back(Z[(size_t)l * W + w]);
            kq.push_back(Kq);
            dq.insert(dq.end(), dqq.begin(), dqq.end());
            ++rows;
        }
    }
    op->n_lin_rows = rows;
    // Range index: the rank index resolved by ladder integer, one 32-bit
    // entry per (flip mask, pattern): bit 31 set: the linear-table row in bits
    // 0-30; else the range's first term (bits 0-20) and its length (bits
    // 21-30; 0: no term, no group).  A candidate then finds what to evaluate
    // with one load.  Built when every indexed group has a ladder table, the
    // terms number below 2^21 and every range holds below 2^10 terms.
    op->range_ok = false;
    if (op->dense_ok && T < ((int64_t)1 << 21)) {
        const int64_t nd = (int64_t)(op->dense.bytes / 4);
        std::vector<int32_t> dense((size_t)nd);
        QSD_CUDA(cudaMemcpyAsync(dense.data(), op->dense.p, (size_t)nd * 4, cudaMemcpyDeviceToHost, s));
        QSD_CUDA(cudaStreamSynchronize(s));
        std::vector<uint32_t> rix((size_t)nd * 16, 0u);
        bool ok = true;
        for (int64_t i = 0; i < nd && ok; ++i) {
            const int32_t g = dense[(size_t)i];
            if (g < 0) continue;
            const int L = gL[(size_t)g];
            if (L == 0) { ok = false; break; }
            for (int l = 0; l < (1 << L); ++l) {
                uint32_t v;
                if (base[(size_t)g] >= 0) {
                    v = 0x80000000u | (uint32_t)(base[(size_t)g] + l);
                } else {
                    const int32_t b = gptr[(size_t)g * 17 + l], e = gptr[(size_t)g * 17 + l + 1];
                    if (e - b >= 1024) { ok = false; break; }
                    v = (uint32_t)b | ((uint32_t)(e - b) << 21);
                }
                rix[(size_t)i * 16 + l] = v;
            }
        }
        if (ok) {
            op->rix.alloc(rix.size() * 4);
            QSD_CUDA(cudaMemcpyAsync(op->rix.p, rix.data(), rix.size() * 4, cudaMemcpyHostToDevice, s));
            op->range_ok = true;
        }
    }
    op->lin_base.alloc((size_t)G * 4);
    QSD_CUDA(cudaMemcpyAsync(op->lin_base.p, base.data(), (size_t)G * 4, cudaMemcpyHostToDevice, s));
    if (rows > 0) {
        op->lin_z.alloc(zref.size() * 8);
        op->lin_kq.alloc(kq.size() * 8);
        op->lin_dq.alloc(dq.size() * 8);
        QSD_CUDA(cudaMemcpyAsync(op->lin_z.p, zref.data(), zref.size() * 8, cudaMemcpyHostToDevice, s));
        QSD_CUDA(cudaMemcpyAsync(op->lin_kq.p, kq.data(), kq.size() * 8, cudaMemcpyHostToDevice, s));
        QSD_CUDA(cudaMemcpyAsync(op->lin_dq.p, dq.data(), dq.size() * 8, cudaMemcpyHostToDevice, s));
    }
    QSD_CUDA(cudaStreamSynchronize(s));
}

}  // namespace

void build_excitation_index(qsd_ctx ctx, qsd_op op) {
    op->exc_ok = false;
    const int W = op->W;
    const int64_t G = op->G, T = op->T;
    if (G == 0 || W > kMaxWordsStatic) return;
    cudaStream_t s = ctx->stream;
    op->exc_split = op->n_qubits / 2;
    DevBuf shape((size_t)T * 4);
    k_term_shapes<<<blocks_for(G, 128), 128, 0, s>>>(W, G, op->grange.as<int32_t>(), op->gF.as<uint64_t>(), T,
                                                     op->tP.as<uint64_t>(), op->tV.as<uint64_t>(), op->exc_split,
                                                     shape.as<uint32_t>());
    QSD_LAUNCH_CHECK();
    std::vector<uint32_t> hs(T);
    std::vector<int32_t> gr(G + 1);
    QSD_CUDA(cudaMemcpyAsync(hs.data(), shape.p, (size_t)T * 4, cudaMemcpyDeviceToHost, s));
    QSD_CUDA(cudaMemcpyAsync(gr.data(), op->grange.p, (size_t)(G + 1) * 4, cudaMemcpyDeviceToHost, s));
    QSD_CUDA(cudaStreamSynchronize(s));
    std::vector<int32_t> exc, rest;
    std::set<uint32_t> shapes;
    for (int64_t g = 0; g < G; ++g) {
        bool ok = true;
        for (int32_t t = gr[g]; t < gr[g + 1] && ok; ++t) ok = hs[t] != 0xffffffffu;
        if (ok) {
            exc.push_back((int32_t)g);
            for (int32_t t = gr[g]; t < gr[g + 1]; ++t) shapes.insert(hs[t]);
        } else {
            rest.push_back((int32_t)g);
        }
    }
    if (exc.empty() || shapes.size() > (size_t)kMaxShapes) return;
    op->n_shapes = 0;
    for (uint32_t v : shapes) op->shapes[op->n_shapes++] = v;
    op->G_exc = (int64_t)exc.size();
    op->G_rest = (int64_t)rest.size();
    op->exc_gid.alloc(exc.size() * 4);
    op->rest_gid.alloc(std::max<size_t>(rest.size(), 1) * 4);
    QSD_CUDA(cudaMemcpyAsync(op->exc_gid.p, exc.data(), exc.size() * 4, cudaMemcpyHostToDevice, s));
    if (!rest.empty())
        QSD_CUDA(cudaMemcpyAsync(op->rest_gid.p, rest.data(), rest.size() * 4, cudaMemcpyHostToDevice, s));
    op->excF.alloc((size_t)W * op->G_exc * 8);
    k_gather_exc<<<blocks_for(op->G_exc, 256), 256, 0, s>>>(W, G, op->exc_gid.as<int32_t>(), op->G_exc,
                                                           op->gF.as<uint64_t>(), op->excF.as<uint64_t>());
    QSD_LAUNCH_CHECK();
    HashTable t = build_hash(ctx, op->excF.as<uint64_t>(), W, op->G_exc);
    op->gtags = std::move(t.tags);
    op->gsidx = std::move(t.sidx);
    op->g_nbuckets = t.n_buckets;
    op->g_shift = t.shift;
    QSD_CUDA(cudaStreamSynchronize(s));
    build_dense_index(ctx, op, exc);
    if (W <= 2) {
        const size_t rb = W == 1 ? sizeof(TermRec<1>) : sizeof(TermRec<2>);
        std::vector<double> phi((size_t)T);
        QSD_CUDA(cudaMemcpyAsync(phi.data(), op->tphi.p, (size_t)T * 8, cudaMemcpyDeviceToHost, s));
        QSD_CUDA(cudaStreamSynchronize(s));
        const int ex = fixed_point_exponent(phi, gr);
        const double scale = std::ldexp(1.0, ex);
        op->qscale = std::ldexp(1.0, -ex);
        op->qexp = ex;
        op->trec.alloc((size_t)T * rb);
        if (W == 1)
            k_term_records<1><<<blocks_for(T, 256), 256, 0, s>>>(T, op->tP.as<uint64_t>(), op->tV.as<uint64_t>(),
                                                                 op->tZ.as<uint64_t>(), op->tphi.as<double>(), scale,
                                                                 op->trec.as<TermRec<1>>());
        else
            k_term_records<2><<<blocks_for(T, 256), 256, 0, s>>>(T, op->tP.as<uint64_t>(), op->tV.as<uint64_t>(),
                                                                 op->tZ.as<uint64_t>(), op->tphi.as<double>(), scale,
                                                                 op->trec.as<TermRec<2>>());
        QSD_LAUNCH_CHECK();
        QSD_CUDA(cudaStreamSynchronize(s));
        build_linear_ranges(ctx, op, exc, phi, scale);
    }
    op->exc_ok = true;
}

double excitation_candidates(qsd_op op, qsd_sub sub) {
    if (!op->exc_ok || sub->key0.empty()) return -1.0;
    int64_t cnt[4] = {0, 0, 0, 0};
    for (int q = 0; q < op->n_qubits; ++q) {
        const bool occ = (sub->key0[q >> 6] >> (q & 63)) & 1;
        const int sct = q < op->exc_split ? 0 : 1;
        cnt[2 * sct + (occ ? 0 : 1)]++;
    }
    double total = 0.0;
    for (int i = 0; i < op->n_shapes; ++i) {
        const uint32_t sh = op->shapes[i];
        double n = 1.0;
        for (int j = 0; j < 4; ++j) n *= (double)choose_h(cnt[j], (int)((sh >> (4 * j)) & 15));
        total += n;
    }
    return total + (double)op->G_rest;
}

}  // namespace qsd
