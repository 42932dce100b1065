// Complex product y = H_S x for operators with complex matrix elements (the
// extended alphabet allows complex coefficients, Methods "Qubit
// Hamiltonians"), FP64, x and y complex128 [D][k] interleaved (re, im).
//
// A lane per row, every group evaluated term by term (ladder int_ptrs where
// the group has them): the element is the sum over the group's passing terms
// of phi_t (-1)^popc(r & Z_t) with complex phi_t; one lookup of r xor F per
// group with a passing term; the diagonal (complex for a non-Hermitian
// operator) from the diagonal terms.  Groups and terms in a fixed order:
// deterministic.
#include "qsd_internal.cuh"

namespace qsd {

namespace {

struct CplxParams {
    const uint64_t *keys;
    int64_t D;
    HashView hv;
    const uint64_t *nib;
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
    const double *dphi, *dphi_im;
    double id_re, id_im;
    const double2 *x;
    double2 *y;
    int k;
    uint32_t *err;
};

template <int W>
__device__ __forceinline__ uint32_t cbit(const uint64_t (&x)[W], int q) {
    uint64_t v = x[0];
#pragma unroll
    for (int w = 1; w < W; ++w)
        if ((q >> 6) == w) v = x[w];
    return (uint32_t)((v >> (q & 63)) & 1);
}

// KB columns starting at c0 (KB <= 16)
template <int W, int KB>
__global__ void __launch_bounds__(256) k_apply_complex(const CplxParams p, int c0) {
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= p.D) return;
    uint64_t key[W];
#pragma unroll
    for (int w = 0; w < W; ++w) key[w] = __ldg(p.keys + (size_t)w * p.D + row);
    const uint64_t hr = key_hash<W>(key, p.nib);
    double2 acc[KB];
#pragma unroll
    for (int j = 0; j < KB; ++j) acc[j] = make_double2(0.0, 0.0);
    // diagonal
    double dre = p.id_re, dim = p.id_im;
    for (int64_t t = 0; t < p.Td; ++t) {
        bool ok = true;
        int par = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            ok &= (key[w] & __ldg(p.dP + (size_t)w * p.Td + t)) == __ldg(p.dV + (size_t)w * p.Td + t);
            par ^= __popcll(key[w] & __ldg(p.dZ + (size_t)w * p.Td + t));
        }
        if (!ok) continue;
        const double s = (par & 1) ? -1.0 : 1.0;
        dre += s * __ldg(p.dphi + t);
        dim += s * __ldg(p.dphi_im + t);
    }
    for (int64_t g = 0; g < p.G; ++g) {
        int32_t b, e;
        const int L = __ldg(p.gL + g);
        if (L) {
            const uint64_t pos = __ldg(p.gpos + g);
            int l = 0;
            for (int i = 0; i < L; ++i) l |= (int)cbit<W>(key, (int)((pos >> (16 * i)) & 0xffff)) << i;
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
        if (!pass) continue;
        uint64_t c[W];
#pragma unroll
        for (int w = 0; w < W; ++w) c[w] = key[w] ^ __ldg(p.gF + (size_t)w * p.G + g);
        const int64_t idx = probe<W>(c, hr ^ __ldg(p.ghash + g), p.hv, p.err);
        if (idx < 0) continue;
        const double2 *xc = p.x + idx * p.k + c0;
#pragma unroll
        for (int j = 0; j < KB; ++j) {
            const double2 v = xc[j];
            acc[j].x = fma(hre, v.x, fma(-him, v.y, acc[j].x));
            acc[j].y = fma(hre, v.y, fma(him, v.x, acc[j].y));
        }
    }
    const double2 *xr = p.x + row * p.k + c0;
    double2 *yr = p.y + row * p.k + c0;
#pragma unroll
    for (int j = 0; j < KB; ++j) {
        const double2 v = xr[j];
        yr[j] = make_double2(fma(dre, v.x, fma(-dim, v.y, acc[j].x)), fma(dre, v.y, fma(dim, v.x, acc[j].y)));
    }
}

template <int W>
void launch_kb(const CplxParams &p, int KB, int c0, cudaStream_t s) {
    const int blocks = blocks_for(p.D, 256);
    switch (KB) {
    case 16: k_apply_complex<W, 16><<<blocks, 256, 0, s>>>(p, c0); break;
    case 4: k_apply_complex<W, 4><<<blocks, 256, 0, s>>>(p, c0); break;
    default: k_apply_complex<W, 1><<<blocks, 256, 0, s>>>(p, c0); break;
    }
}

}  // namespace

void apply_H_complex(qsd_ctx ctx, qsd_op op, qsd_sub sub, int k, const void *x, void *y) {
    if (sub->D <= 0) return;
    CplxParams p{};
    p.keys = sub->keys.as<uint64_t>();
    p.D = sub->D;
    p.hv = hash_view(sub);
    p.nib = ctx->nib.as<uint64_t>();
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
    p.dphi_im = op->dphi_im.as<double>();
    p.id_re = op->identity;
    p.id_im = op->identity_im;
    p.x = static_cast<const double2 *>(x);
    p.y = static_cast<double2 *>(y);
    p.k = k;
    p.err = ctx->d_err;
    cudaStream_t s = ctx->stream;
    for (int c = 0; c < k;) {
        const int KB = (k - c >= 16) ? 16 : (k - c >= 4 ? 4 : 1);
        switch (op->W) {
        case 1: launch_kb<1>(p, KB, c, s); break;
        case 2: launch_kb<2>(p, KB, c, s); break;
        case 3: launch_kb<3>(p, KB, c, s); break;
        case 4: launch_kb<4>(p, KB, c, s); break;
        default: fail(QSD_ERR_INVALID_ARG, "qsd_apply_H_complex: more than 256 qubits");
        }
        QSD_LAUNCH_CHECK();
        c += KB;
    }
}

}  // namespace qsd
