// Subspace construction and lookup (Methods, "Subspace data structure").
//
// The paper keeps bit-sets in an insertion-ordered CPU hash map with an
// occupancy bit-set for fast rejection of empty buckets.  Here the strings are
// sorted by integer value on the device (index = rank, the order the MSOB
// triangle test needs) and stored as coalesced SoA words; a separate open
// addressing table of 8-slot buckets (8-bit tags, 32-bit row indices)
// serves lookups: one 8-byte load of eight one-byte tags rejects almost every
// absent key, as the occupancy bit-set did, and the load factor is kept
// <= 1/4 because D is known before the table is built.
#include <algorithm>

#include "qsd_internal.cuh"

namespace qsd {

namespace {

// Load factor <= 1/4 (measured on GB300: 1/8 gained 4 % on the 200-qubit
// Ising product and lost 11 % on the fermionic block product).
constexpr int64_t kLoadDiv = 4;

__global__ void k_aos_to_soa(const uint64_t *__restrict__ in, int W, int64_t n, uint64_t *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int w = 0; w < W; ++w) out[(size_t)w * n + i] = in[(size_t)i * W + w];
}

__global__ void k_soa_to_aos(const uint64_t *__restrict__ in, int W, int64_t n, uint64_t *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int w = 0; w < W; ++w) out[(size_t)i * W + w] = in[(size_t)w * n + i];
}

__global__ void k_mask_top(uint64_t *words, int W, int64_t n, uint64_t top_mask, uint32_t *err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (words[(size_t)i * W + W - 1] & ~top_mask) atomicOr(err, 2u);
}

// One thread per key.  The slots of a bucket are claimed in order, each by a
// compare-and-swap on the 32-bit word holding its tag byte; then the row
// index is stored.  So in the finished table every probe that would reach a
// later slot passes an occupied one.
__device__ __forceinline__ bool claim_slot(uint8_t *tags, uint32_t *sidx, uint64_t b, uint32_t tag, uint32_t i) {
    unsigned int *words = reinterpret_cast<unsigned int *>(tags + b * kBucketSlots);
    for (int s = 0; s < kBucketSlots; ++s) {
        unsigned int *w = words + (s >> 2);
        const int sh = 8 * (s & 3);
        unsigned int old = *reinterpret_cast<volatile unsigned int *>(w);
        while (((old >> sh) & 0xffu) == 0u) {
            const unsigned int prev = atomicCAS(w, old, old | (tag << sh));
            if (prev == old) {
                sidx[b * kBucketSlots + s] = i;
                return true;
            }
            old = prev;  // another byte of the word changed, or this slot was taken
        }
    }
    return false;
}

template <int W>
__global__ void k_hash_insert(const uint64_t *__restrict__ keys, int64_t D, const uint64_t *__restrict__ nib,
                              uint8_t *tags, uint32_t *sidx, uint64_t bucket_mask, int shift, uint64_t *hash_out,
                              uint32_t *occ, int occ_shift, uint32_t *err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= D) return;
    uint64_t x[W];
#pragma unroll
    for (int w = 0; w < W; ++w) x[w] = keys[(size_t)w * D + i];
    uint32_t tag;
    const uint64_t h = key_hash<W>(x, nib);
    if (hash_out) hash_out[i] = h;
    if (occ) {
        const uint32_t bi = (uint32_t)(h >> 32) >> occ_shift;
        atomicOr(occ + (bi >> 5), 1u << (bi & 31u));
    }
    uint64_t b = hash_bucket(h, shift, tag);
    for (uint64_t step = 0; step <= bucket_mask; ++step) {
        if (claim_slot(tags, sidx, b, tag, (uint32_t)i)) return;
        b = (b + 1) & bucket_mask;
    }
    atomicOr(err, 1u);
}

__global__ void k_hash_insert_dyn(const uint64_t *__restrict__ keys, int W, int64_t D,
                                  const uint64_t *__restrict__ nib, uint8_t *tags, uint32_t *sidx,
                                  uint64_t bucket_mask, int shift, uint32_t *err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= D) return;
    uint64_t x[kMaxWordsDyn];
    for (int w = 0; w < W; ++w) x[w] = keys[(size_t)w * D + i];
    uint32_t tag;
    uint64_t b = hash_bucket(key_hash_dyn(x, W, nib), shift, tag);
    for (uint64_t step = 0; step <= bucket_mask; ++step) {
        if (claim_slot(tags, sidx, b, tag, (uint32_t)i)) return;
        b = (b + 1) & bucket_mask;
    }
    atomicOr(err, 1u);
}

template <int W>
__global__ void k_index(const uint64_t *__restrict__ q, int64_t n, const HashView hv,
                        const uint64_t *__restrict__ nib, int64_t *out, uint32_t *err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t c[W];
#pragma unroll
    for (int w = 0; w < W; ++w) c[w] = q[(size_t)i * W + w];
    out[i] = hv.D > 0 ? probe<W>(c, key_hash<W>(c, nib), hv, err) : -1;
}

__global__ void k_index_dyn(const uint64_t *__restrict__ q, int W, int64_t n, const HashView hv,
                            const uint64_t *__restrict__ nib, int64_t *out, uint32_t *err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t c[kMaxWordsDyn];
    for (int w = 0; w < W; ++w) c[w] = q[(size_t)i * W + w];
    out[i] = hv.D > 0 ? probe_dyn(c, W, key_hash_dyn(c, W, nib), hv, err) : -1;
}

// Occupied slots per bucket (slots fill in order: the count is the index of
// the first empty slot).
__global__ void k_bucket_counts(const uint8_t *__restrict__ tags, int64_t nb, uint32_t *cnt) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const uint2 t = reinterpret_cast<const uint2 *>(tags)[b];
    cnt[b] = (uint32_t)((__popc(__vcmpne4(t.x, 0u)) + __popc(__vcmpne4(t.y, 0u))) >> 3);
}

// Rows in slot order (bucket order) and their keys at those positions.
template <int W>
__global__ void k_hash_order(const uint32_t *__restrict__ sidx, const uint32_t *__restrict__ start, int64_t nb,
                             const uint8_t *__restrict__ tags, const uint64_t *__restrict__ keys,
                             const uint64_t *__restrict__ rhash, int64_t D, uint32_t *perm, uint64_t *hkeys,
                             uint64_t *hhash) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const uint2 t = reinterpret_cast<const uint2 *>(tags)[b];
    const int n = (__popc(__vcmpne4(t.x, 0u)) + __popc(__vcmpne4(t.y, 0u))) >> 3;
    uint32_t pos = start[b];
    for (int i = 0; i < n; ++i, ++pos) {
        const uint32_t row = sidx[b * kBucketSlots + i];
        perm[pos] = row;
        hhash[pos] = rhash[row];
#pragma unroll
        for (int w = 0; w < W; ++w) hkeys[(size_t)w * D + pos] = keys[(size_t)w * D + row];
    }
}

uint64_t next_pow2(uint64_t v) {
    uint64_t p = 1;
    while (p < v) p <<= 1;
    return p;
}

}  // namespace

void build_subspace(qsd_ctx ctx, qsd_sub sub, const uint64_t *words, int64_t n_in, bool on_device) {
    cudaStream_t s = ctx->stream;
    const int W = sub->W;
    ensure_nibble_tables(ctx, W);
    const uint64_t top_bits = (uint64_t)(sub->n_qubits - 64 * (W - 1));
    const uint64_t top_mask = top_bits >= 64 ? ~0ull : ((1ull << top_bits) - 1);
    DevBuf soa;
    int64_t D = 0;
    if (n_in > 0) {
        DevBuf staged;
        const uint64_t *aos = words;
        if (!on_device) {
            staged.alloc((size_t)n_in * W * 8);
            QSD_CUDA(cudaMemcpyAsync(staged.p, words, (size_t)n_in * W * 8, cudaMemcpyHostToDevice, s));
            aos = staged.as<uint64_t>();
        }
        QSD_CUDA(cudaMemsetAsync(ctx->d_err, 0, 4, s));
        k_mask_top<<<blocks_for(n_in, 256), 256, 0, s>>>(const_cast<uint64_t *>(aos), W, n_in, top_mask, ctx->d_err);
        QSD_LAUNCH_CHECK();
        if (take_device_error(ctx) & 2u)
            fail(QSD_ERR_QUBIT_RANGE, "build_subspace: a bit-string has bits set at or above n_qubits");
        soa.alloc((size_t)n_in * W * 8);
        k_aos_to_soa<<<blocks_for(n_in, 256), 256, 0, s>>>(aos, W, n_in, soa.as<uint64_t>());
        QSD_LAUNCH_CHECK();
        radix_sort(ctx, soa.as<uint64_t>(), W, n_in, nullptr);
        D = unique_sorted(ctx, soa.as<uint64_t>(), W, n_in, nullptr, 0);
        if (D > (int64_t)0xfffffffeLL) fail(QSD_ERR_CAPACITY, "build_subspace: more than 2^32-2 distinct strings");
    }
    sub->D = D;
    sub->keys.alloc((size_t)std::max<int64_t>(D, 1) * W * 8);
    if (D > 0) unique_sorted(ctx, soa.as<uint64_t>(), W, n_in, sub->keys.as<uint64_t>(), D);
    soa.release();
    if (W <= kMaxWordsStatic) sub->rhash.alloc((size_t)std::max<int64_t>(D, 1) * 8);
    HashTable t = build_hash(ctx, sub->keys.as<uint64_t>(), W, D, sub->rhash.as<uint64_t>(), true);
    sub->n_buckets = t.n_buckets;
    sub->bucket_shift = t.shift;
    sub->tags = std::move(t.tags);
    sub->sidx = std::move(t.sidx);
    sub->occ = std::move(t.occ);
    sub->occ_shift = t.occ_shift;
    if (D > 0 && W <= kMaxWordsStatic) build_hash_order(ctx, sub);
    build_factored(ctx, sub);
    sub->key0.assign(W, 0);
    if (D > 0)
        for (int w = 0; w < W; ++w)
            QSD_CUDA(cudaMemcpyAsync(&sub->key0[w], sub->keys.as<uint64_t>() + (size_t)w * D, 8,
                                     cudaMemcpyDeviceToHost, s));
    QSD_CUDA(cudaStreamSynchronize(s));
}

// Positions of the rows in bucket order: a scan of the per-bucket counts,
// then each bucket writes its rows (and their keys) at its offset.
void build_hash_order(qsd_ctx ctx, qsd_sub sub) {
    cudaStream_t s = ctx->stream;
    const int64_t nb = sub->n_buckets, D = sub->D;
    const int W = sub->W;
    DevBuf start((size_t)nb * 4);
    k_bucket_counts<<<blocks_for(nb, 256), 256, 0, s>>>(sub->tags.as<uint8_t>(), nb, start.as<uint32_t>());
    QSD_LAUNCH_CHECK();
    exclusive_scan_u32(ctx, start.as<uint32_t>(), start.as<uint32_t>(), nb, false);
    sub->hperm.alloc((size_t)D * 4);
    sub->hkeys.alloc((size_t)D * W * 8);
    sub->hhash.alloc((size_t)D * 8);
    const uint64_t *rh = sub->rhash.as<uint64_t>();
    uint64_t *hh = sub->hhash.as<uint64_t>();
    const uint32_t *si = sub->sidx.as<uint32_t>();
    const uint8_t *tg = sub->tags.as<uint8_t>();
    const uint64_t *keys = sub->keys.as<uint64_t>();
    uint32_t *perm = sub->hperm.as<uint32_t>();
    uint64_t *hk = sub->hkeys.as<uint64_t>();
    const int g = blocks_for(nb, 256);
    switch (W) {
    case 1: k_hash_order<1><<<g, 256, 0, s>>>(si, start.as<uint32_t>(), nb, tg, keys, rh, D, perm, hk, hh); break;
    case 2: k_hash_order<2><<<g, 256, 0, s>>>(si, start.as<uint32_t>(), nb, tg, keys, rh, D, perm, hk, hh); break;
    case 3: k_hash_order<3><<<g, 256, 0, s>>>(si, start.as<uint32_t>(), nb, tg, keys, rh, D, perm, hk, hh); break;
    default: k_hash_order<4><<<g, 256, 0, s>>>(si, start.as<uint32_t>(), nb, tg, keys, rh, D, perm, hk, hh); break;
    }
    QSD_LAUNCH_CHECK();
    QSD_CUDA(cudaStreamSynchronize(s));  // start is freed on return
}

HashTable build_hash(qsd_ctx ctx, const uint64_t *keys, int W, int64_t D, uint64_t *hash_out, bool with_filter) {
    cudaStream_t s = ctx->stream;
    HashTable t;
    // load factor <= 1/4 over buckets of 8 slots: a bucket overflows into the
    // next one with probability ~1e-3, so probes almost never diverge
    t.n_buckets = (int64_t)next_pow2((uint64_t)std::max<int64_t>(2, (kLoadDiv * D + kBucketSlots - 1) / kBucketSlots));
    int lg = 0;
    while ((1ll << lg) < t.n_buckets) ++lg;
    if (lg > 32) fail(QSD_ERR_CAPACITY, "hash table larger than 2^32 buckets");
    t.shift = 64 - lg;
    const size_t cap = (size_t)t.n_buckets * kBucketSlots;
    t.tags.alloc(cap);
    t.sidx.alloc(cap * 4);
    QSD_CUDA(cudaMemsetAsync(t.tags.p, 0, cap, s));
    uint32_t *occ = nullptr;
    if (with_filter && W <= kMaxWordsStatic && lg <= kOccMaxBucketsLog2) {
        const size_t words = std::max<size_t>(1, ((size_t)t.n_buckets << kOccBitsPerBucketLog2) / 32);
        t.occ.alloc(words * 4);
        QSD_CUDA(cudaMemsetAsync(t.occ.p, 0, words * 4, s));
        t.occ_shift = 32 - (lg + kOccBitsPerBucketLog2);
        occ = t.occ.as<uint32_t>();
    }
    if (D > 0) {
        QSD_CUDA(cudaMemsetAsync(ctx->d_err, 0, 4, s));
        const uint64_t mask = (uint64_t)t.n_buckets - 1;
        auto *tg = t.tags.as<uint8_t>();
        auto *si = t.sidx.as<uint32_t>();
        const uint64_t *nib = ctx->nib.as<uint64_t>();
        const int nb = blocks_for(D, 256);
        const int shift = t.shift;
        switch (W) {
        case 1:
            k_hash_insert<1><<<nb, 256, 0, s>>>(keys, D, nib, tg, si, mask, shift, hash_out, occ, t.occ_shift, ctx->d_err);
            break;
        case 2:
            k_hash_insert<2><<<nb, 256, 0, s>>>(keys, D, nib, tg, si, mask, shift, hash_out, occ, t.occ_shift, ctx->d_err);
            break;
        case 3:
            k_hash_insert<3><<<nb, 256, 0, s>>>(keys, D, nib, tg, si, mask, shift, hash_out, occ, t.occ_shift, ctx->d_err);
            break;
        case 4:
            k_hash_insert<4><<<nb, 256, 0, s>>>(keys, D, nib, tg, si, mask, shift, hash_out, occ, t.occ_shift, ctx->d_err);
            break;
        default: k_hash_insert_dyn<<<nb, 256, 0, s>>>(keys, W, D, nib, tg, si, mask, shift, ctx->d_err);
        }
        QSD_LAUNCH_CHECK();
        if (take_device_error(ctx)) fail(QSD_ERR_INTERNAL, "hash table overflow");
    }
    return t;
}

void subspace_index(qsd_ctx ctx, qsd_sub sub, int64_t n, const uint64_t *q, int64_t *out) {
    if (n <= 0) return;
    cudaStream_t s = ctx->stream;
    const HashView hv = hash_view(sub);
    const uint64_t *nib = ctx->nib.as<uint64_t>();
    const int nb = blocks_for(n, 256);
    switch (sub->W) {
    case 1: k_index<1><<<nb, 256, 0, s>>>(q, n, hv, nib, out, ctx->d_err); break;
    case 2: k_index<2><<<nb, 256, 0, s>>>(q, n, hv, nib, out, ctx->d_err); break;
    case 3: k_index<3><<<nb, 256, 0, s>>>(q, n, hv, nib, out, ctx->d_err); break;
    case 4: k_index<4><<<nb, 256, 0, s>>>(q, n, hv, nib, out, ctx->d_err); break;
    default: k_index_dyn<<<nb, 256, 0, s>>>(q, sub->W, n, hv, nib, out, ctx->d_err);
    }
    QSD_LAUNCH_CHECK();
}

void subspace_keys_aos(qsd_ctx ctx, qsd_sub sub, uint64_t *out_dev) {
    if (sub->D <= 0) return;
    k_soa_to_aos<<<blocks_for(sub->D, 256), 256, 0, ctx->stream>>>(sub->keys.as<uint64_t>(), sub->W, sub->D, out_dev);
    QSD_LAUNCH_CHECK();
}

}  // namespace qsd
