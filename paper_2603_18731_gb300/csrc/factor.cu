// Sector-factored index of a product subspace (built with the subspace).
//
// The paper's chemistry subspaces are products of alpha and beta strings
// (Results, "split into alpha and beta halves"), and its Discussion names
// rejecting groups in bulk as future work.  For such a subspace the columns a
// row reaches are exactly the products of the neighbours of its two halves
// inside the two half lists: a flip mask of a two-body fermionic operator
// changes at most two occupied and two empty qubits per sector, so the
// column (a', b') of row (a, b) is in S iff a' is in A and b' is in B.  The
// product kernel therefore enumerates only columns that are in S -- no lookup
// misses -- and computes their index as ib' |A| + ia' instead of probing the
// hash table.  This file builds what that needs: the two sorted half lists
// and, per string of each list, its neighbours in the same list by
// excitation type (see Factored in qsd_internal.cuh), each with what the
// product needs of its flip mask: the rank of the flipped positions (the
// group's entry in the operator's rank index) and the row's pattern on them
// (its ladder integer within the sector).
#include <algorithm>
#include <vector>

#include "qsd_internal.cuh"

namespace qsd {

namespace {

// Low half (qubits [0, split)) and high half (qubits [split, n)) of every
// row; split <= 64 and n - split <= 64.
template <int W>
__global__ void k_halves(const uint64_t *__restrict__ keys, int64_t D, int split, uint64_t *lo, uint64_t *hi) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= D) return;
    const uint64_t k0 = keys[r];
    const uint64_t k1 = W > 1 ? keys[D + r] : 0ull;
    if (split >= 64) {
        lo[r] = k0;
        hi[r] = k1;
    } else {
        lo[r] = k0 & ((1ull << split) - 1ull);
        hi[r] = (k0 >> split) | (W > 1 ? (k1 << (64 - split)) : 0ull);
    }
}

// Rank of the set of bits of F (positions below 64, at most four bits) in
// the combinatorial number system, sum over the ascending positions p_k of
// C(p_k, k), with the row's bits at those positions (bit k - 1 of the
// pattern = bit p_k of `row`) and the number of bits.  Packed as rank (bits
// 0-19; C(64, 4) < 2^20), pattern (bits 20-23) and count (bits 24-26).
__device__ __forceinline__ uint32_t neighbour_meta(uint64_t F, uint64_t row) {
    uint64_t rank = 0;
    uint32_t pat = 0;
    int k = 0;
    while (F) {
        const uint64_t p = (uint64_t)(__ffsll((long long)F) - 1);
        ++k;
        uint64_t c = p;  // C(p, k) by the multiplicative formula, exact in 64 bits
        for (int i = 1; i < k; ++i) c = c * (p - (uint64_t)i) / (uint64_t)(i + 1);
        rank += c;
        pat |= (uint32_t)((row >> p) & 1ull) << (k - 1);
        F &= F - 1;
    }
    return (uint32_t)rank | (pat << 20) | ((uint32_t)k << 24);
}

// One warp per string i of the list L[0..n): its neighbours j by type
// t = 3 dOcc + dEmp - 1 with dOcc = popc(L[i] & ~L[j]) and
// dEmp = popc(~L[i] & L[j]) both <= 2 (j = i has type -1).  Count mode
// (ptr == nullptr): cnt[8 i + t] = number of neighbours of type t.  Fill
// mode: writes (j, neighbour_meta(L[i] ^ L[j], L[i])) at ptr[8 i + t] in
// ascending j.
__global__ void k_neighbours(const uint64_t *__restrict__ L, uint32_t n, const uint32_t *__restrict__ ptr,
                             uint32_t *cnt, uint2 *out) {
    const uint32_t i = (uint32_t)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= n) return;  // warp-uniform
    const uint64_t a = L[i];
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t run[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (uint32_t j0 = 0; j0 < n; j0 += 32) {
        const uint32_t j = j0 + (uint32_t)lane;
        int t = -1;
        uint64_t b = 0;
        if (j < n) {
            b = L[j];
            const int dO = __popcll(a & ~b), dE = __popcll(~a & b);
            if (dO <= 2 && dE <= 2) t = 3 * dO + dE - 1;
        }
#pragma unroll
        for (int tt = 0; tt < 8; ++tt) {
            const uint32_t m = __ballot_sync(0xffffffffu, t == tt);
            if (ptr && t == tt)
                out[ptr[8 * (size_t)i + tt] + run[tt] + __popc(m & lt)] = make_uint2(j, neighbour_meta(a ^ b, a));
            run[tt] += __popc(m);
        }
    }
    if (!ptr) {
#pragma unroll
        for (int tt = 0; tt < 8; ++tt)
            if (lane == tt) cnt[8 * (size_t)i + tt] = run[tt];
    }
}

__global__ void k_set_u32(uint32_t *p, uint32_t v) { *p = v; }

constexpr uint32_t kMaxTypeNeighbours = 4096;

// Neighbour lists of one half list; false when they would exceed cap entries.
bool build_neighbours(qsd_ctx ctx, const uint64_t *L, int64_t n, int64_t cap, DevBuf &ptr, DevBuf &nbr,
                      int64_t &nnz) {
    cudaStream_t s = ctx->stream;
    const int64_t m = 8 * n;
    DevBuf cnt((size_t)m * 4);
    ptr.alloc((size_t)(m + 1) * 4);
    const unsigned blocks = (unsigned)blocks_for(n * 32, 256);
    k_neighbours<<<blocks, 256, 0, s>>>(L, (uint32_t)n, nullptr, cnt.as<uint32_t>(), nullptr);
    QSD_LAUNCH_CHECK();
    // at most kMaxTypeNeighbours per (string, type): a row's candidate count
    // (products of two lists, summed over at most 16 shapes) stays in 32 bits
    std::vector<uint32_t> h((size_t)m);
    QSD_CUDA(cudaMemcpyAsync(h.data(), cnt.p, (size_t)m * 4, cudaMemcpyDeviceToHost, s));
    QSD_CUDA(cudaStreamSynchronize(s));
    if (*std::max_element(h.begin(), h.end()) > kMaxTypeNeighbours) {
        ptr.release();
        return false;
    }
    const uint64_t total = exclusive_scan_u32(ctx, cnt.as<uint32_t>(), ptr.as<uint32_t>(), m, true);
    if (total > (uint64_t)cap) {
        ptr.release();
        return false;
    }
    k_set_u32<<<1, 1, 0, s>>>(ptr.as<uint32_t>() + m, (uint32_t)total);
    QSD_LAUNCH_CHECK();
    nbr.alloc((size_t)std::max<uint64_t>(total, 1) * 8);
    if (total > 0) {
        k_neighbours<<<blocks, 256, 0, s>>>(L, (uint32_t)n, ptr.as<uint32_t>(), nullptr, nbr.as<uint2>());
        QSD_LAUNCH_CHECK();
    }
    QSD_CUDA(cudaStreamSynchronize(s));  // cnt is freed on return
    nnz = (int64_t)total;
    return true;
}

// Half sums of the linear ranges (see qsd_internal.cuh): thread (i, l) adds
// the fixed-point coefficients d_l of the qubits set in string i (qubits
// offset + bit), plus K_l when kq is given.  Sums wrap modulo 2^64 like the
// product's own integer sums, so S_A + S_B is bitwise K + sum over the row.
__global__ void k_linear_halves(const uint64_t *__restrict__ strs, int64_t n, int offset,
                                const int64_t *__restrict__ dq, const int64_t *__restrict__ kq, int nq,
                                int64_t nlr, int64_t *out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * nlr) return;
    const int64_t i = idx / nlr, l = idx - i * nlr;
    uint64_t str = strs[i];
    uint64_t sum = kq ? (uint64_t)kq[l] : 0ull;
    const int64_t *__restrict__ d = dq + (size_t)l * nq + offset;
    while (str) {
        const int b = __ffsll((long long)str) - 1;
        str &= str - 1ull;
        sum += (uint64_t)d[b];
    }
    out[(size_t)i * nlr + l] = (int64_t)sum;
}

}  // namespace

void build_factored(qsd_ctx ctx, qsd_sub sub) {
    Factored &f = sub->fac;
    f = Factored{};
    const int n = sub->n_qubits;
    const int64_t D = sub->D;
    if (D <= 0 || n < 2 || n > 128) return;
    const int split = n / 2;
    cudaStream_t s = ctx->stream;
    DevBuf lo((size_t)D * 8), hi((size_t)D * 8);
    if (sub->W == 1)
        k_halves<1><<<blocks_for(D, 256), 256, 0, s>>>(sub->keys.as<uint64_t>(), D, split, lo.as<uint64_t>(),
                                                       hi.as<uint64_t>());
    else
        k_halves<2><<<blocks_for(D, 256), 256, 0, s>>>(sub->keys.as<uint64_t>(), D, split, lo.as<uint64_t>(),
                                                       hi.as<uint64_t>());
    QSD_LAUNCH_CHECK();
    // the keys are sorted by (high, low): the high halves already ascend
    const int64_t nB = unique_sorted(ctx, hi.as<uint64_t>(), 1, D, nullptr, 0);
    if (D % nB != 0) return;
    radix_sort(ctx, lo.as<uint64_t>(), 1, D, nullptr);
    const int64_t nA = unique_sorted(ctx, lo.as<uint64_t>(), 1, D, nullptr, 0);
    // at most 2^16 strings per half: the pair tests stay cheap and the
    // neighbour counts (at most n (n - 1)) within 32 bits
    if (nA * nB != D || nA > 65536 || nB > 65536) return;
    f.A.alloc((size_t)nA * 8);
    f.B.alloc((size_t)nB * 8);
    unique_sorted(ctx, lo.as<uint64_t>(), 1, D, f.A.as<uint64_t>(), nA);
    unique_sorted(ctx, hi.as<uint64_t>(), 1, D, f.B.as<uint64_t>(), nB);
    lo.release();
    hi.release();
    // neighbour entries are bounded so that the index stays a small part of
    // the subspace's memory (a full space of many qubits has dense lists)
    const int64_t cap = 64 * (nA + nB) + ((int64_t)1 << 20);
    if (!build_neighbours(ctx, f.A.as<uint64_t>(), nA, cap, f.ptrA, f.nbrA, f.nnzA) ||
        !build_neighbours(ctx, f.B.as<uint64_t>(), nB, cap - f.nnzA, f.ptrB, f.nbrB, f.nnzB)) {
        f = Factored{};
        return;
    }
    f.split = split;
    f.nA = nA;
    f.nB = nB;
    f.ok = true;
}

bool build_linear_halves(qsd_ctx ctx, qsd_op op, qsd_sub sub, cudaStream_t s, DevBuf &sa, DevBuf &sb) {
    const Factored &f = sub->fac;
    const int64_t nlr = op->n_lin_rows;
    if (!f.ok || nlr <= 0 || op->lin_dq.p == nullptr || op->exc_split != f.split) return false;
    // at most 1 GiB per pair (the 32-orbital workload: 3968 rows x 3000 strings x 8 B = 95 MB)
    if ((double)nlr * (double)(f.nA + f.nB) * 8.0 > (double)(1ull << 30)) return false;
    sa.alloc((size_t)(f.nA * nlr) * 8);
    sb.alloc((size_t)(f.nB * nlr) * 8);
    const int nq = op->n_qubits;
    k_linear_halves<<<blocks_for(f.nA * nlr, 256), 256, 0, s>>>(f.A.as<uint64_t>(), f.nA, 0, op->lin_dq.as<int64_t>(),
                                                                op->lin_kq.as<int64_t>(), nq, nlr, sa.as<int64_t>());
    k_linear_halves<<<blocks_for(f.nB * nlr, 256), 256, 0, s>>>(f.B.as<uint64_t>(), f.nB, f.split,
                                                                op->lin_dq.as<int64_t>(), nullptr, nq, nlr,
                                                                sb.as<int64_t>());
    QSD_LAUNCH_CHECK();
    QSD_CUDA(cudaStreamSynchronize(s));
    return true;
}

}  // namespace qsd
