// Subspace refinement RAMPS on the device (Supplementary, "Recursive
// algorithm for a minimal perturbative subspace", Algorithm S1, Eq. S2).
//
// The paper runs the recursion serially and names parallel evaluation of the
// rows as future work (Discussion).  Here each level is one grid over every
// (frontier row, off-diagonal group) pair: the group's terms give the element
// h = <row|H|row xor F> (zero when no term passes its projector test); a
// column not yet in the output (and inside the restriction subspace, when
// given) gets amp = pre |h|^2 / (E - H_kk), with H_kk evaluated from the
// diagonal terms for that bit-string; columns with |amp| > tau are appended
// to a candidate list.  The list is sorted by key on the device and every
// distinct column keeps its largest |amp| (ties: the larger amp), so the next
// level does not depend on the order of the appends.  Where the printed
// algorithm is silent: output rows are never revisited (the recursion would
// otherwise return to its start, where E - H_kk = 0); starting rows expand
// together; a column with H_kk = E is added but not expanded; `max_levels`
// ends the recursion.
#include <cstring>
#include <vector>

#include "qsd_internal.cuh"

namespace qsd {

namespace {

struct RampsParams {
    int W;
    const uint64_t *fkeys;  // [W][nF] frontier rows
    const double *fpre;     // [nF] prefactors
    int64_t nF;
    int64_t G;
    const uint64_t *gF, *ghash;
    const int32_t *grange;
    const uint8_t *gL;
    const uint64_t *gpos;
    const int32_t *gptr;
    int64_t T;
    const uint64_t *tP, *tV, *tZ;
    const double *tphi, *tphi_im;
    const uint8_t *tflag;
    int64_t Td;
    const uint64_t *dP, *dV, *dZ;
    const double *dphi;
    double identity;
    const uint64_t *nib;
    HashView out;           // rows already in the output
    HashView allowed;       // restriction subspace (tags == nullptr: none)
    double E, tau;
    uint64_t *ckeys;        // [W][cap] candidates
    double *camp, *cgap;    // [cap]
    unsigned long long *count;
    int64_t cap;
    uint32_t *err;
};

template <int W>
__device__ __forceinline__ uint64_t kword(const uint64_t (&k)[W], int q) {
    uint64_t v = k[0];
#pragma unroll
    for (int w = 1; w < W; ++w)
        if ((q >> 6) == w) v = k[w];
    return v;
}

// One thread per (frontier row, group).
template <int W>
__global__ void __launch_bounds__(256) k_ramps_expand(const RampsParams p) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= p.nF * p.G) return;
    const int64_t j = idx / p.G, g = idx % p.G;
    uint64_t key[W], col[W];
#pragma unroll
    for (int w = 0; w < W; ++w) key[w] = __ldg(p.fkeys + (size_t)w * p.nF + j);
    // the group's element at this row
    int32_t b, e;
    const int L = __ldg(p.gL + g);
    if (L) {
        const uint64_t pos = __ldg(p.gpos + g);
        int l = 0;
        for (int i = 0; i < L; ++i) {
            const int q = (int)((pos >> (16 * i)) & 0xffff);
            l |= (int)((kword<W>(key, q) >> (q & 63)) & 1) << i;
        }
        b = __ldg(p.gptr + g * 17 + l);
        e = __ldg(p.gptr + g * 17 + l + 1);
    } else {
        b = __ldg(p.grange + g);
        e = __ldg(p.grange + g + 1);
    }
    bool pass = false;
    double hre = 0.0, him = 0.0;
    for (int32_t t = b; t < e; ++t) {
        const uint8_t f = __ldg(p.tflag + t);
        bool ok = true;
        int par = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            if (f & 1) ok &= (key[w] & __ldg(p.tP + (size_t)w * p.T + t)) == __ldg(p.tV + (size_t)w * p.T + t);
            if (f & 2) par ^= __popcll(key[w] & __ldg(p.tZ + (size_t)w * p.T + t));
        }
        if (!ok) continue;
        pass = true;
        const double s = (par & 1) ? -1.0 : 1.0;
        hre += s * __ldg(p.tphi + t);
        him += s * __ldg(p.tphi_im + t);
    }
    if (!pass) return;
#pragma unroll
    for (int w = 0; w < W; ++w) col[w] = key[w] ^ __ldg(p.gF + (size_t)w * p.G + g);
    const uint64_t hk = key_hash<W>(col, p.nib);
    if (probe<W>(col, hk, p.out, p.err) >= 0) return;  // already in the output
    if (p.allowed.tags && probe<W>(col, hk, p.allowed, p.err) < 0) return;
    double hkk = p.identity;
    for (int64_t t = 0; t < p.Td; ++t) {
        bool ok = true;
        int par = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            ok &= (col[w] & __ldg(p.dP + (size_t)w * p.Td + t)) == __ldg(p.dV + (size_t)w * p.Td + t);
            par ^= __popcll(col[w] & __ldg(p.dZ + (size_t)w * p.Td + t));
        }
        if (ok) hkk += (par & 1) ? -__ldg(p.dphi + t) : __ldg(p.dphi + t);
    }
    const double gap = p.E - hkk;
    const double amp = gap == 0.0 ? __longlong_as_double(0x7ff0000000000000ll)  // +inf: unbounded
                                  : __ldg(p.fpre + j) * (hre * hre + him * him) / gap;
    if (!(fabs(amp) > p.tau)) return;
    const unsigned long long at = atomicAdd(p.count, 1ull);
    if ((int64_t)at >= p.cap) return;  // counted; the host grows the list and reruns the level
#pragma unroll
    for (int w = 0; w < W; ++w) p.ckeys[(size_t)w * p.cap + at] = col[w];
    p.camp[at] = amp;
    p.cgap[at] = gap;
}

// Runs of equal keys in the sorted candidates: the run start picks the best
// candidate and writes the next frontier row (prefactor amp / gap; 0 when
// the gap is 0: added, not expanded).
__global__ void k_ramps_best(int W, const uint64_t *__restrict__ skeys, int64_t n, const uint32_t *__restrict__ perm,
                             const uint32_t *__restrict__ flags, const uint32_t *__restrict__ pos,
                             const double *__restrict__ camp, const double *__restrict__ cgap, int64_t nR,
                             uint64_t *rkeys, double *rpre, double *ramp) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !flags[i]) return;
    uint32_t best = perm[i];
    for (int64_t k = i + 1; k < n && !flags[k]; ++k) {
        const uint32_t c = perm[k];
        const double a = camp[c], bb = camp[best];
        if (fabs(a) > fabs(bb) || (fabs(a) == fabs(bb) && a > bb)) best = c;
    }
    const int64_t r = pos[i];
    for (int w = 0; w < W; ++w) rkeys[(size_t)w * nR + r] = skeys[(size_t)w * n + i];
    const double g = cgap[best];
    rpre[r] = g == 0.0 ? 0.0 : camp[best] / g;
    ramp[r] = camp[best];
}

// dst[w][0..na) = a[w][..], dst[w][na..na+nb) = b[w][..] (SoA concatenation)
__global__ void k_concat(int W, const uint64_t *__restrict__ a, int64_t na, const uint64_t *__restrict__ b,
                         int64_t nb, uint64_t *dst) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n = na + nb;
    if (i >= n) return;
    for (int w = 0; w < W; ++w)
        dst[(size_t)w * n + i] = i < na ? a[(size_t)w * na + i] : b[(size_t)w * nb + (i - na)];
}

// SoA [W][n] -> row-major [n][W]
__global__ void k_to_rows(int W, const uint64_t *__restrict__ soa, int64_t n, uint64_t *rows) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int w = 0; w < W; ++w) rows[(size_t)i * W + w] = soa[(size_t)w * n + i];
}

__global__ void k_fill(double *x, int64_t n, double v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}

void launch_expand(const RampsParams &p, cudaStream_t s) {
    const int64_t total = p.nF * p.G;
    if (total <= 0) return;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    switch (p.W) {
    case 1: k_ramps_expand<1><<<blocks, 256, 0, s>>>(p); break;
    case 2: k_ramps_expand<2><<<blocks, 256, 0, s>>>(p); break;
    case 3: k_ramps_expand<3><<<blocks, 256, 0, s>>>(p); break;
    default: k_ramps_expand<4><<<blocks, 256, 0, s>>>(p); break;
    }
    QSD_LAUNCH_CHECK();
}

}  // namespace

void ramps(qsd_ctx ctx, qsd_op op, qsd_sub start, double E, double tau, int max_levels, qsd_sub allowed,
           int64_t max_rows, qsd_sub out, qsd_ramps_info *info) {
    cudaStream_t s = ctx->stream;
    const int W = op->W;
    std::memset(info, 0, sizeof(*info));
    // output rows so far (SoA) and their hash table; the frontier
    int64_t n_out = start->D;
    DevBuf okeys((size_t)std::max<int64_t>(n_out, 1) * W * 8);
    QSD_CUDA(cudaMemcpyAsync(okeys.p, start->keys.p, (size_t)n_out * W * 8, cudaMemcpyDeviceToDevice, s));
    DevBuf fkeys((size_t)std::max<int64_t>(n_out, 1) * W * 8), fpre((size_t)std::max<int64_t>(n_out, 1) * 8);
    QSD_CUDA(cudaMemcpyAsync(fkeys.p, start->keys.p, (size_t)n_out * W * 8, cudaMemcpyDeviceToDevice, s));
    if (n_out > 0) {
        k_fill<<<blocks_for(n_out, 256), 256, 0, s>>>(fpre.as<double>(), n_out, 1.0 / E);
        QSD_LAUNCH_CHECK();
    }
    int64_t nF = n_out;
    int64_t cap = std::max<int64_t>(1 << 16, 4 * nF);
    DevBuf cnt(8);
    RampsParams p{};
    p.W = W;
    p.G = op->G;
    p.gF = op->gF.as<uint64_t>();
    p.ghash = op->ghash.as<uint64_t>();
    p.grange = op->grange.as<int32_t>();
    p.gL = op->gL.as<uint8_t>();
    p.gpos = op->gpos.as<uint64_t>();
    p.gptr = op->gptr.as<int32_t>();
    p.T = op->T;
    p.tP = op->tP.as<uint64_t>();
    p.tV = op->tV.as<uint64_t>();
    p.tZ = op->tZ.as<uint64_t>();
    p.tphi = op->tphi.as<double>();
    p.tphi_im = op->tphi_im.as<double>();
    p.tflag = op->tflag.as<uint8_t>();
    p.Td = op->Td;
    p.dP = op->dP.as<uint64_t>();
    p.dV = op->dV.as<uint64_t>();
    p.dZ = op->dZ.as<uint64_t>();
    p.dphi = op->dphi.as<double>();
    p.identity = op->identity;
    p.nib = ctx->nib.as<uint64_t>();
    p.allowed = allowed ? hash_view(allowed) : HashView{};
    p.E = E;
    p.tau = tau;
    p.err = ctx->d_err;
    int level = 0;
    while (nF > 0 && level < max_levels && op->G > 0) {
        HashTable ht = build_hash(ctx, okeys.as<uint64_t>(), W, n_out);
        p.out = HashView{ht.tags.as<uint8_t>(), ht.sidx.as<uint32_t>(), okeys.as<uint64_t>(), n_out,
                         (uint64_t)ht.n_buckets - 1, ht.shift};
        p.fkeys = fkeys.as<uint64_t>();
        p.fpre = fpre.as<double>();
        p.nF = nF;
        unsigned long long n_cand = 0;
        DevBuf ckeys, camp, cgap;
        for (int attempt = 0; attempt < 2; ++attempt) {
            ckeys.alloc((size_t)cap * W * 8);
            camp.alloc((size_t)cap * 8);
            cgap.alloc((size_t)cap * 8);
            p.ckeys = ckeys.as<uint64_t>();
            p.camp = camp.as<double>();
            p.cgap = cgap.as<double>();
            p.cap = cap;
            p.count = cnt.as<unsigned long long>();
            QSD_CUDA(cudaMemsetAsync(cnt.p, 0, 8, s));
            launch_expand(p, s);
            QSD_CUDA(cudaMemcpyAsync(&n_cand, cnt.p, 8, cudaMemcpyDeviceToHost, s));
            QSD_CUDA(cudaStreamSynchronize(s));
            if ((int64_t)n_cand <= cap) break;
            cap = (int64_t)n_cand;  // grow to fit and rerun the level
        }
        if (take_device_error(ctx)) fail(QSD_ERR_INTERNAL, "qsd_ramps: hash probe ran past the table");
        info->candidates += (int64_t)n_cand;
        if (n_cand == 0) {
            nF = 0;
            break;
        }
        const int64_t n = (int64_t)n_cand;
        if (n >= (int64_t)0xffffffffLL) fail(QSD_ERR_CAPACITY, "qsd_ramps: more than 2^32 candidates in a level");
        // compact the candidate keys to stride n, sort them with their index
        DevBuf skeys((size_t)n * W * 8), perm((size_t)n * 4), flags((size_t)n * 4), pos((size_t)n * 4);
        for (int w = 0; w < W; ++w)
            QSD_CUDA(cudaMemcpyAsync(skeys.as<uint64_t>() + (size_t)w * n, ckeys.as<uint64_t>() + (size_t)w * cap,
                                     (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
        std::vector<uint32_t> iota(n);
        for (int64_t i = 0; i < n; ++i) iota[i] = (uint32_t)i;
        QSD_CUDA(cudaMemcpyAsync(perm.p, iota.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s));
        radix_sort(ctx, skeys.as<uint64_t>(), W, n, perm.as<uint32_t>());
        diff_flags(ctx, skeys.as<uint64_t>(), W, n, flags.as<uint32_t>());
        const int64_t nR = (int64_t)exclusive_scan_u32(ctx, flags.as<uint32_t>(), pos.as<uint32_t>(), n, true);
        DevBuf rkeys((size_t)nR * W * 8), rpre((size_t)nR * 8), ramp((size_t)nR * 8);
        k_ramps_best<<<blocks_for(n, 256), 256, 0, s>>>(W, skeys.as<uint64_t>(), n, perm.as<uint32_t>(),
                                                       flags.as<uint32_t>(), pos.as<uint32_t>(), camp.as<double>(),
                                                       cgap.as<double>(), nR, rkeys.as<uint64_t>(),
                                                       rpre.as<double>(), ramp.as<double>());
        QSD_LAUNCH_CHECK();
        // output += the level's rows (none of them was in the output)
        DevBuf nout((size_t)(n_out + nR) * W * 8);
        k_concat<<<blocks_for(n_out + nR, 256), 256, 0, s>>>(W, okeys.as<uint64_t>(), n_out, rkeys.as<uint64_t>(),
                                                            nR, nout.as<uint64_t>());
        QSD_LAUNCH_CHECK();
        QSD_CUDA(cudaStreamSynchronize(s));
        okeys = std::move(nout);
        n_out += nR;
        if (level < 64) info->level_rows[level] = nR;
        ++level;
        // next frontier: rows with a nonzero prefactor, in key order
        std::vector<double> hpre(nR);
        QSD_CUDA(cudaMemcpy(hpre.data(), rpre.p, (size_t)nR * 8, cudaMemcpyDeviceToHost));
        std::vector<uint32_t> keep;
        for (int64_t r = 0; r < nR; ++r)
            if (hpre[r] != 0.0) keep.push_back((uint32_t)r);
        if ((int64_t)keep.size() == nR) {
            fkeys = std::move(rkeys);
            fpre = std::move(rpre);
            nF = nR;
        } else {
            // rare (a diagonal equal to E): gather the expandable rows on the host
            std::vector<uint64_t> hk((size_t)nR * W), nk(keep.size() * W);
            QSD_CUDA(cudaMemcpy(hk.data(), rkeys.p, hk.size() * 8, cudaMemcpyDeviceToHost));
            std::vector<double> np(keep.size());
            for (size_t i = 0; i < keep.size(); ++i) {
                for (int w = 0; w < W; ++w) nk[(size_t)w * keep.size() + i] = hk[(size_t)w * nR + keep[i]];
                np[i] = hpre[keep[i]];
            }
            nF = (int64_t)keep.size();
            fkeys.alloc(std::max<size_t>(nk.size(), 1) * 8);
            fpre.alloc(std::max<size_t>(np.size(), 1) * 8);
            if (nF > 0) {
                QSD_CUDA(cudaMemcpy(fkeys.p, nk.data(), nk.size() * 8, cudaMemcpyHostToDevice));
                QSD_CUDA(cudaMemcpy(fpre.p, np.data(), np.size() * 8, cudaMemcpyHostToDevice));
            }
        }
        if (max_rows > 0 && n_out >= max_rows) {
            info->truncated = 1;
            break;
        }
    }
    info->levels = level;
    info->stopped_by_limit = (nF > 0 && level >= max_levels) ? 1 : 0;
    // the output subspace: sorted, deduplicated, hashed
    DevBuf rows((size_t)std::max<int64_t>(n_out, 1) * W * 8);
    if (n_out > 0) {
        k_to_rows<<<blocks_for(n_out, 256), 256, 0, s>>>(W, okeys.as<uint64_t>(), n_out, rows.as<uint64_t>());
        QSD_LAUNCH_CHECK();
    }
    build_subspace(ctx, out, rows.as<uint64_t>(), n_out, true);
    info->rows_out = out->D;
}

}  // namespace qsd
