// Internal declarations of the GB300 subspace Hamiltonian library.
//
// Layout in device memory (all arrays are plain cudaMalloc allocations owned
// by the handles):
//   subspace  keys   uint64 [W][D]   SoA, sorted ascending (word W-1 most
//                                    significant); row index = rank
//             tags   uint16 [cap]    8-slot buckets (16 bytes), 0 = empty
//             sidx   uint32 [cap]    row index per slot; load factor <= 1/4
//   operator  off-diagonal terms grouped by flip mask F (Methods, properties
//             1-3): per group F[W][G], hash of F, term range, ladder table;
//             per term P/V/Z masks [W][T] and the real phase phi[T]
//             diagonal terms separately (the cached diagonal, Methods
//             "Matrix evaluation")
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <tuple>
#include <stdexcept>
#include <string>
#include <utility>
#include <vector>

#include "../../include/qsd.h"

namespace qsd {

// ------------------------------------------------------------------ errors
struct Error : std::runtime_error {
    int code;
    Error(int c, const std::string &m) : std::runtime_error(m), code(c) {}
};

[[noreturn]] void fail(int code, const std::string &msg);
void cuda_check(cudaError_t e, const char *what, const char *file, int line);
#define QSD_CUDA(call) ::qsd::cuda_check((call), #call, __FILE__, __LINE__)
#define QSD_LAUNCH_CHECK() ::qsd::cuda_check(cudaGetLastError(), "kernel launch", __FILE__, __LINE__)

// ------------------------------------------------------------------ memory
// Owning device allocation.  Allocation failure throws QSD_ERR_OOM.  With a
// stream the memory is stream-ordered (cudaMallocAsync / cudaFreeAsync on
// that stream), so allocating or freeing never synchronises the device.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaStream_t stream = nullptr;
    bool async = false;
    DevBuf() = default;
    explicit DevBuf(size_t n) { alloc(n); }
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept : p(o.p), bytes(o.bytes), stream(o.stream), async(o.async) {
        o.p = nullptr;
        o.bytes = 0;
    }
    DevBuf &operator=(DevBuf &&o) noexcept {
        if (this != &o) {
            release();
            p = o.p; bytes = o.bytes; stream = o.stream; async = o.async;
            o.p = nullptr; o.bytes = 0;
        }
        return *this;
    }
    ~DevBuf() { release(); }
    void alloc(size_t n);
    // stream-ordered from `pool` (nullptr: the device's default pool)
    void alloc_pool(size_t n, cudaMemPool_t pool, cudaStream_t s);
    void alloc_async(size_t n, cudaStream_t s);
    void release();
    template <typename T> T *as() const { return static_cast<T *>(p); }
};

// Grow-only scratch buffer (reused between calls on one context).
struct Scratch {
    DevBuf buf;
    void *get(size_t bytes) {
        if (buf.bytes < bytes) { buf.release(); buf.alloc(bytes + bytes / 4); }
        return buf.p;
    }
};

// ------------------------------------------------------------------ handles
struct Binding;

}  // namespace qsd

namespace qsd {
// Pass-1 result of the CSR build, kept between the sizing and the filling call.
struct CsrState {
    const void *op = nullptr, *sub = nullptr;
    bool lower = false;
    int64_t nnz = -1;
    DevBuf cnt, cnt_up, len, off;  // uint32 [D]: evaluated, mirrored, segment length and start
    void clear() {
        op = sub = nullptr;
        nnz = -1;
        cnt.release();
        cnt_up.release();
        len.release();
        off.release();
    }
};
}  // namespace qsd

struct qsd_ctx_s {
    int device = 0;
    int tune_mode = 0;    // product path: 0 auto, 1 group scan, 2 excitation index, 3 half evaluation,
                          // 4 sector-factored where it applies (else auto), 5 filter/verify scan
                          // where it applies (else auto)
    int tune_lanes = 0;   // lanes per row of the group scan: 0 auto, 1 or 8
    int allow_sym = 0;    // the autotuner may pick the half-evaluation product
    int row_order = 0;    // lane-per-row scans: 0 auto, 1 index order, 2 hash order
    int autotune = 1;     // measure the product paths on first use and cache the fastest
    int linear_halves = 1;  // factored product: half sums of the linear ranges per pair
    std::mutex tune_mu;
    std::map<std::tuple<const void *, const void *, int, int>, int> tune_cache;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 0;
    std::string last_error;
    std::mutex mu;
    qsd::Scratch scratch[5];  // 0, 1: host-buffer products; 2, 3: residuals; 4: widened x
    // (operator, subspace) -> cached diagonal; dropped when either is freed
    std::map<std::pair<const void *, const void *>, qsd::Binding *> bindings;
    // device copy of the nibble tables of the linear key hash
    qsd::DevBuf nib;
    int nib_words = 0;
    qsd::CsrState csr;
    uint32_t *d_err = nullptr;   // device error word of the last kernels
    uint32_t *h_err = nullptr;   // pinned mirror
    // stream-ordered pool of the eigensolver's workspace: freed blocks up to
    // its release threshold stay mapped for the next solve on the context
    cudaMemPool_t pool = nullptr;
};

namespace qsd {
// Sector-factored index of a subspace S whose strings split at qubit `split`
// into a low half a (qubits [0, split)) and a high half b (qubits
// [split, n)).  Built when S is exactly the product A x B of its distinct
// halves (|S| = |A| |B|); S is then sorted by (b, a) and row = ib * |A| + ia
// for a = A[ia], b = B[ib].  Per half list, each string's neighbours in the
// same list by excitation type: the other strings reached by turning dOcc of
// its set bits off and dEmp of its clear bits on (0 <= dOcc, dEmp <= 2, not
// both 0), type t = 3 dOcc + dEmp - 1, ascending by index.  An entry is
// (index j, meta) with meta = rank of the flipped positions F = L[i] ^ L[j]
// in the combinatorial number system (bits 0-19), L[i]'s bits on them in
// ascending order (bits 20-23) and popc(F) (bits 24-26).
struct Factored {
    bool ok = false;
    int split = 0;
    int64_t nA = 0, nB = 0;
    DevBuf A, B;        // uint64 [nA], [nB]: distinct halves, ascending
    DevBuf ptrA, ptrB;  // uint32 [8 n + 1]: start of (string i, type t) at 8 i + t
    DevBuf nbrA, nbrB;  // uint2: (neighbour index, meta)
    int64_t nnzA = 0, nnzB = 0;
};
}  // namespace qsd

struct qsd_sub_s {
    qsd_ctx ctx = nullptr;
    int32_t n_qubits = 0;
    int W = 1;
    int64_t D = 0;
    int64_t n_buckets = 0;  // power of two >= 2; capacity = 8 * n_buckets slots
    int bucket_shift = 63;  // 64 - log2(n_buckets)
    qsd::DevBuf keys;   // uint64 [W][D]
    qsd::DevBuf tags;   // uint8 [8 * n_buckets], 0 = empty
    qsd::DevBuf sidx;   // uint32 [8 * n_buckets]
    qsd::DevBuf occ;    // uint32 occupancy filter (HashView::occ), W <= 4 and n_buckets <= 2^25
    int occ_shift = 0;
    // hash order (W <= 4): the rows in bucket order and their keys
    qsd::DevBuf rhash;  // uint64 [D] hash h of each row (W <= 4)
    qsd::DevBuf hperm;  // uint32 [D] row at each position
    qsd::DevBuf hkeys;  // uint64 [W][D] keys[w][hperm[i]] at i
    qsd::DevBuf hhash;  // uint64 [D] rhash[hperm[i]] at i
    std::vector<uint64_t> key0;  // host copy of the first (smallest) string
    qsd::Factored fac;           // product subspaces (n <= 128), split n / 2
};

struct qsd_op_s {
    qsd_ctx ctx = nullptr;
    int32_t n_qubits = 0;
    int W = 1;
    qsd_op_info info{};
    double identity = 0.0;
    double identity_im = 0.0;
    // off-diagonal groups (G) and terms (T), group order
    int64_t G = 0, T = 0;
    qsd::DevBuf gF;      // uint64 [W][G]
    qsd::DevBuf ghash;   // uint64 [G]  hash h of F
    qsd::DevBuf grange;  // int32  [G+1] term offsets
    qsd::DevBuf gL;      // uint8  [G]  ladder bits with a table (0: scan the group)
    qsd::DevBuf gpos;    // uint64 [G]  4 x 16-bit flipped-qubit positions, ascending
    qsd::DevBuf gptr;    // int32  [G][17] ladder-integer term offsets (absolute)
    qsd::DevBuf grec;    // GroupRec [G] (32 bytes): what the product reads per group
    qsd::DevBuf amp;     // double [n_amp] matrix element per support pattern (table groups)
    qsd::DevBuf ampf;    // float2 [n_amp] the same split into FP32 (hi, lo)
    int64_t n_amp = 0, n_table_groups = 0;
    int64_t max_table_size = 0;  // largest amplitude table (2^support size) of a group (0: scan group)
    int64_t min_table_size = 0;  // smallest
    // excitation index of the ladder groups (fermionic operators)
    bool exc_ok = false;
    int exc_split = 0, n_shapes = 0;
    uint32_t shapes[16] = {0};
    int64_t G_exc = 0, G_rest = 0;
    qsd::DevBuf excF;      // uint64 [W][G_exc] flip masks of the indexed groups
    qsd::DevBuf exc_gid;   // int32 [G_exc]
    qsd::DevBuf rest_gid;  // int32 [G_rest]
    qsd::DevBuf gtags, gsidx;
    // dense rank index of the excitation groups (when it fits): per sector
    // bit-count signature (b0, b1), entry base + rank0 * C(n1, b1) + rank1
    // holds the group of that flip mask or -1 (ranks in the combinatorial
    // number system of the bits' positions within their sector)
    bool dense_ok = false;
    qsd::DevBuf dense;     // int32 [dense entries]
    uint32_t dbase[16] = {0}, dstride[16] = {0};  // per shape
    int64_t g_nbuckets = 0;
    int g_shift = 63;
    qsd::DevBuf tP, tV, tZ;  // uint64 [W][T]
    qsd::DevBuf tphi;    // double [T] real phase * coefficient
    qsd::DevBuf tphi_im; // double [T]
    qsd::DevBuf tflag;   // uint8  [T] bit0: P != 0, bit1: Z != 0
    qsd::DevBuf trec;    // TermRec<W> [T]: P, V, Z, fixed-point phase (W <= 2, excitation index built)
    // linear ranges (W <= 2): lin_base[g] = first table row of group g (-1:
    // none), row = lin_base[g] + ladder integer; per row Zref [W], K and d [n]
    // per qubit in the fixed point of trec
    int64_t n_lin_rows = 0;
    qsd::DevBuf lin_base, lin_z, lin_kq, lin_dq;
    // range index: uint32 [dense entries][16], the rank index resolved by
    // ladder integer (linear-table row, or first term and length)
    bool range_ok = false;
    qsd::DevBuf rix;
    double qscale = 1.0; // value of one fixed-point unit of trec, 2^-qexp
    int qexp = 0;
    qsd::DevBuf gmsob;   // uint16 [G] most significant flipped qubit (built by the first CSR call)
    // diagonal terms (Td)
    int64_t Td = 0;
    qsd::DevBuf dP, dV, dZ;  // uint64 [W][Td]
    qsd::DevBuf dphi;        // double [Td]
    qsd::DevBuf dphi_im;     // double [Td] imaginary parts (complex operators)
    // input terms as masks, for the term table
    int64_t T_in = 0;
    qsd::DevBuf iF, iP, iV, iZ;  // uint64 [W][T_in]
    qsd::DevBuf iY;              // uint8 [T_in] number of Y letters mod 4
    std::vector<uint64_t> host_groups;  // [G][W]
    // the input words as given (host), for operators derived from this one
    std::vector<int64_t> in_term_ptr;
    std::vector<int32_t> in_qubit;
    std::vector<uint8_t> in_code;
    std::vector<double> in_re, in_im;
};

namespace qsd {

struct Binding {
    DevBuf diag;  // double [D]
};

// ------------------------------------------------------------ device hash
// Keys are hashed by one random GF(2)-linear map h: every word w of a key is
// split into 16 nibbles and each nibble indexes a table of 16 random 64-bit
// values (one 128-byte line), h(x) = xor of the W * 16 entries.  A random
// linear map is a universal hash family (pairwise collision probability
// 2^-m on m output bits; Carter and Wegman 1979), and its linearity gives
// h(r xor F) = h(r) xor h(F): a row's hash is computed once and each group
// costs one xor.  The bucket is the top log2(n_buckets) bits of h and the
// tag its low 8 bits (0 mapped to 1).
//
// Because the bucket is itself linear, bucket(r xor F) = bucket(r) xor
// bucket(F): rows taken in bucket order (the table's own slot order) send
// the lookups of one group to buckets that stay together -- xor with a
// constant maps an aligned run of buckets onto another aligned run -- so a
// warp of consecutive rows probes a few cache lines instead of 32
// (the hash-order traversal of the product).
//
// Table layout: buckets of 8 slots.  tags: uint8 [8 * n_buckets], 0 = empty,
// one 8-byte load per bucket; sidx: uint32 [8 * n_buckets], the row index of
// each occupied slot, read only when its tag matches.  Slots of a bucket fill
// in order, so a bucket whose last slot is empty ends the probe.  Tag
// collisions only cost a key comparison: every hit is verified against the
// full key.
constexpr int kBucketSlots = 8;

__host__ __device__ __forceinline__ uint64_t fmix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// bucket = top (64 - shift) bits of h, in [0, 2^(64 - shift)), with
// 32 <= shift <= 63 (at most 2^32 buckets): a 32-bit shift of h's high word;
// tag in [1, 255].
__host__ __device__ __forceinline__ uint32_t hash_bucket(uint64_t h, int shift, uint32_t &tag) {
    const uint32_t t = (uint32_t)h & 0xffu;
    tag = t ? t : 1u;
    return (uint32_t)(h >> 32) >> (shift - 32);
}

// nib: [w][16 nibble positions][16 values] for words 0..W-1
template <int W>
__device__ __forceinline__ uint64_t key_hash(const uint64_t (&x)[W], const uint64_t *__restrict__ nib) {
    uint64_t h = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const uint64_t *t = nib + (size_t)w * 256;
#pragma unroll
        for (int j = 0; j < 16; ++j) h ^= __ldg(t + j * 16 + ((x[w] >> (4 * j)) & 15));
    }
    return h;
}

__device__ __forceinline__ uint64_t key_hash_dyn(const uint64_t *x, int W, const uint64_t *__restrict__ nib) {
    uint64_t h = 0;
    for (int w = 0; w < W; ++w) {
        const uint64_t *t = nib + (size_t)w * 256;
#pragma unroll
        for (int j = 0; j < 16; ++j) h ^= __ldg(t + j * 16 + ((x[w] >> (4 * j)) & 15));
    }
    return h;
}

// h of the single bit q (the nibble entry with only that bit set).
__device__ __forceinline__ uint64_t bit_hash(int q, const uint64_t *__restrict__ nib) {
    return __ldg(nib + (size_t)(q >> 6) * 256 + ((q >> 2) & 15) * 16 + (1 << (q & 3)));
}

// Nibble tables for words 0..W-1 (host copy), [W*256].
std::vector<uint64_t> host_nibble_tables(int W);
void ensure_nibble_tables(qsd_ctx ctx, int W);

// The 8 one-byte tags of bucket b (slot i in byte i of the 8-byte word).
__device__ __forceinline__ uint2 load_tags(const uint8_t *__restrict__ tags, uint64_t b) {
    return __ldg(reinterpret_cast<const uint2 *>(tags) + b);
}

// Nonzero iff some byte of v is zero (the "has a zero byte" test of Hacker's
// Delight, section 6-1; exact as an existence test).
__device__ __forceinline__ uint32_t zero_byte(uint32_t v) { return (v - 0x01010101u) & ~v & 0x80808080u; }

// Bit 7 of each byte of v, packed into bits 0..3: with x = v >> 7 (bits at
// 0, 8, 16, 24), x * 0x01020408 moves bit 8i to 24 + i and every cross term
// to a distinct position below 24 (3, 10, 11, 17, 18, 19), so no carry
// reaches bits 24..27.
__device__ __forceinline__ uint32_t pack_byte_msbs(uint32_t v) { return (((v >> 7) * 0x01020408u) >> 24) & 0xfu; }

// Bit i set when tag i of the bucket equals `tag` (exact per slot: a byte-wise
// compare, then one bit per byte).
__device__ __forceinline__ uint32_t tag_match(const uint2 t, uint32_t tag) {
    const uint32_t tt = tag * 0x01010101u;
    return pack_byte_msbs(__vcmpeq4(t.x, tt) & 0x80808080u) | (pack_byte_msbs(__vcmpeq4(t.y, tt) & 0x80808080u) << 4);
}

// Some tag of the bucket equals `tag`.
__device__ __forceinline__ bool tag_any(const uint2 t, uint32_t tag) {
    const uint32_t tt = tag * 0x01010101u;
    return (zero_byte(t.x ^ tt) | zero_byte(t.y ^ tt)) != 0u;
}

// The bucket's last slot is occupied: the probe continues in the next bucket.
__device__ __forceinline__ bool bucket_full(const uint2 t) { return (t.y >> 24) != 0u; }

struct HashView {
    const uint8_t *tags;
    const uint32_t *sidx;
    const uint64_t *keys;  // [W][D]
    int64_t D;
    uint64_t bmask;
    int shift;
    // occupancy filter (nullptr: none): bit (hi32(h) >> occ_shift) is set for
    // the hash h of every key -- the top log2(n_buckets) + 7 bits of h, 128
    // bits per bucket, so at load <= 1/4 at most 1/64 of the bits are set;
    // a clear bit proves the key absent
    const uint32_t *occ;
    int occ_shift;
};

// Occupancy filter bits per bucket (log2) and the largest bucket count it covers.
constexpr int kOccBitsPerBucketLog2 = 7;
constexpr int kOccMaxBucketsLog2 = 32 - kOccBitsPerBucketLog2;

// Index of the verified key among the matching slots of bucket b, or -1.
template <int W>
__device__ __forceinline__ int64_t verify_matches(const HashView &hv, uint64_t b, uint32_t match,
                                                  const uint64_t (&c)[W]) {
    while (match) {
        const int i = __ffs(match) - 1;
        match &= match - 1;
        const uint64_t cand = __ldg(hv.sidx + b * kBucketSlots + i);
        bool eq = true;
#pragma unroll
        for (int w = 0; w < W; ++w) eq &= (__ldg(hv.keys + (size_t)w * hv.D + cand) == c[w]);
        if (eq) return (int64_t)cand;
    }
    return -1;
}

// verify_matches for a one-column product: x[cand] is loaded beside the
// candidate's key words (both depend only on the candidate row), so a hit
// costs one dependent load after the slot's row index instead of two; xv
// receives x of the verified row.
template <int W, typename TX>
__device__ __forceinline__ int64_t verify_matches_x(const HashView &hv, uint64_t b, uint32_t match,
                                                    const uint64_t (&c)[W], const TX *__restrict__ x0, int64_t ld,
                                                    TX &xv) {
    while (match) {
        const int i = __ffs(match) - 1;
        match &= match - 1;
        const uint64_t cand = __ldg(hv.sidx + b * kBucketSlots + i);
        const TX xs = __ldg(x0 + cand * ld);
        bool eq = true;
#pragma unroll
        for (int w = 0; w < W; ++w) eq &= (__ldg(hv.keys + (size_t)w * hv.D + cand) == c[w]);
        if (eq) {
            xv = xs;
            return (int64_t)cand;
        }
    }
    return -1;
}

// Continue a probe after bucket b (whose tags were already inspected).
template <int W>
__device__ int64_t probe_from(const HashView &hv, uint64_t b, uint32_t tag, const uint64_t (&c)[W], uint32_t *err) {
    for (uint64_t step = 1; step <= hv.bmask; ++step) {
        b = (b + 1) & hv.bmask;
        const uint2 t = load_tags(hv.tags, b);
        const int64_t idx = verify_matches<W>(hv, b, tag_match(t, tag), c);
        if (idx >= 0) return idx;
        if (!bucket_full(t)) return -1;
    }
    if (err) atomicOr(err, 1u);
    return -1;
}

// Lookup of column key c (W words, key_hash hc); returns the row index or -1.
// At most n_buckets buckets are visited (a full table yields -1, sets *err).
template <int W>
__device__ __forceinline__ int64_t probe(const uint64_t (&c)[W], uint64_t hc, const HashView &hv, uint32_t *err) {
    uint32_t tag;
    const uint64_t b = hash_bucket(hc, hv.shift, tag);
    const uint2 t = load_tags(hv.tags, b);
    const int64_t idx = verify_matches<W>(hv, b, tag_match(t, tag), c);
    if (idx >= 0 || !bucket_full(t)) return idx;
    return probe_from<W>(hv, b, tag, c, err);
}

__device__ __forceinline__ int64_t probe_dyn(const uint64_t *c, int W, uint64_t hc, const HashView &hv,
                                             uint32_t *err) {
    uint32_t tag;
    uint64_t b = hash_bucket(hc, hv.shift, tag);
    for (uint64_t step = 0; step <= hv.bmask; ++step) {
        const uint2 t = load_tags(hv.tags, b);
        uint32_t match = tag_match(t, tag);
        while (match) {
            const int i = __ffs(match) - 1;
            match &= match - 1;
            const uint64_t cand = __ldg(hv.sidx + b * kBucketSlots + i);
            bool eq = true;
            for (int w = 0; w < W; ++w) eq &= (__ldg(hv.keys + (size_t)w * hv.D + cand) == c[w]);
            if (eq) return (int64_t)cand;
        }
        if (!bucket_full(t)) return -1;
        b = (b + 1) & hv.bmask;
    }
    if (err) atomicOr(err, 1u);
    return -1;
}

// Largest W handled by the unrolled (template) kernels; larger W use the
// run-time-W kernels with keys in local memory up to kMaxWordsDyn.
constexpr int kMaxWordsStatic = 4;
constexpr int kMaxWordsDyn = 64;  // 4096 qubits

// ----------------------------------------------------------- primitives
// Exclusive prefix sum of n uint32 (in place allowed); returns the total.
uint64_t exclusive_scan_u32(qsd_ctx ctx, const uint32_t *in, uint32_t *out, int64_t n, bool want_total);
// Stable LSD radix sort of n items by K-word keys (SoA, keys[w*n+i], word
// K-1 most significant) with an optional uint32 payload, 8-bit digits;
// digits that are equal for every item are skipped.
void radix_sort(qsd_ctx ctx, uint64_t *keys, int K, int64_t n, uint32_t *payload);
// flags[i] = 1 when item i of the sorted SoA keys starts a run of equal keys.
void diff_flags(qsd_ctx ctx, const uint64_t *keys, int K, int64_t n, uint32_t *flags);
// Keep the first of each run of equal K-word keys in the sorted SoA array;
// writes the unique keys (SoA with stride n_out) to out and returns n_out.
int64_t unique_sorted(qsd_ctx ctx, const uint64_t *keys, int K, int64_t n, uint64_t *out, int64_t out_cap);

// ----------------------------------------------------------- operations
void build_subspace(qsd_ctx ctx, qsd_sub sub, const uint64_t *words, int64_t n_in, bool on_device);
void subspace_index(qsd_ctx ctx, qsd_sub sub, int64_t n, const uint64_t *q, int64_t *out);
void subspace_keys_aos(qsd_ctx ctx, qsd_sub sub, uint64_t *out_dev);
struct HashTable {
    DevBuf tags, sidx;
    DevBuf occ;  // uint32 occupancy filter words (with_filter), else empty
    int64_t n_buckets = 0;
    int shift = 63;
    int occ_shift = 0;
};
// Hash table over n keys given as SoA words keys[w*n + i] (table layout of
// the subspace index); hash_out (optional, [n], W <= 4): each key's hash h.
HashTable build_hash(qsd_ctx ctx, const uint64_t *keys, int W, int64_t n, uint64_t *hash_out = nullptr,
                     bool with_filter = false);
// The subspace's rows in bucket order (hperm, hkeys; W <= 4).
void build_hash_order(qsd_ctx ctx, qsd_sub sub);
void build_excitation_index(qsd_ctx ctx, qsd_op op);
// Sector-factored index of the subspace at split n / 2 (n <= 128), kept only
// when the subspace is the product of its distinct halves.
void build_factored(qsd_ctx ctx, qsd_sub sub);
// Half sums of the operator's linear ranges over the subspace's two half
// lists: sa [nA][n_lin_rows] = K + sum of d over the qubits set in A[i],
// sb [nB][n_lin_rows] = sum of d over the qubits set in B[i] (shifted by the
// split), int64 fixed point.  A linear candidate of row (ia, ib) then sums
// two entries instead of one per occupied qubit.  False (nothing allocated)
// when the pair has no linear ranges or the tables would exceed 1 GiB;
// synchronises s.
bool build_linear_halves(qsd_ctx ctx, qsd_op op, qsd_sub sub, cudaStream_t s, DevBuf &sa, DevBuf &sb);
// The pair's half-sum tables, built on first use on stream s outside a stream
// capture (nullptr pointers: not built, or disabled); cached per (operator,
// subspace) until either is freed.
struct LinearHalves {
    const int64_t *sa = nullptr, *sb = nullptr;
};
LinearHalves linear_halves(qsd_ctx ctx, qsd_op op, qsd_sub sub, cudaStream_t s, bool may_build = true);
// Everything a product of (op, sub) builds on first use, done now (outside any
// capture): call before capturing products into a graph.
void prepare_product(qsd_ctx ctx, qsd_op op, qsd_sub sub, cudaStream_t s);
void drop_linear_halves(const void *handle);
// Candidate flip masks per row of the excitation path for the subspace's
// first string, or -1 when the operator has no excitation index.
double excitation_candidates(qsd_op op, qsd_sub sub);
inline HashView hash_view(qsd_sub sub) {
    return HashView{sub->tags.as<uint8_t>(), sub->sidx.as<uint32_t>(), sub->keys.as<uint64_t>(), sub->D,
                    (uint64_t)sub->n_buckets - 1, sub->bucket_shift, sub->occ.as<uint32_t>(), sub->occ_shift};
}
void load_operator(qsd_ctx ctx, qsd_op op, int64_t n_terms, const int64_t *term_ptr,
                   const int32_t *op_qubit, const uint8_t *op_code, const double *coef_re,
                   const double *coef_im);
Binding *get_binding(qsd_ctx ctx, qsd_op op, qsd_sub sub);
void drop_bindings(qsd_ctx ctx, const void *handle);
void compute_diagonal(qsd_ctx ctx, qsd_op op, qsd_sub sub, double *d);
void compute_diagonal_on(qsd_ctx ctx, qsd_op op, qsd_sub sub, double *d, cudaStream_t s);
// y = H_S x on `stream`.  may_tune: a product shape seen for the first time
// may be timed on the stream to pick the fastest path (never while the
// stream is being captured).  may_allocate = false: the product allocates
// nothing (per-pair tables not yet built are not built; the product is the
// same, bitwise).
void apply_H(qsd_ctx ctx, qsd_op op, qsd_sub sub, const double *diag, int precision, int k,
             const void *x, void *y, cudaStream_t stream, bool may_tune = false, bool may_allocate = true);
// Path of a product shape (see apply_H); measures it once when allowed.
// CSR form of H_S (csr.cu).  Sizing call (indptr, indices, data_re NULL):
// returns nnz and keeps the pass-1 counts; filling call: writes the arrays.
int64_t to_csr(qsd_ctx ctx, qsd_op op, qsd_sub sub, bool lower, int64_t *indptr, void *indices, int index_bits,
               double *data_re, double *data_im, const double *diag);

// Block eigensolver (lobpcg.cu); returns the status it also stores in info.
int lobpcg(qsd_ctx ctx, qsd_op op, qsd_sub sub, const double *diag, const qsd_lobpcg_params &p, double *evals,
           double *evecs, qsd_lobpcg_info *info);

// Group trimming (trim.cu): `out` is a fresh operator handle (ctx, n_qubits,
// W set) loaded from the kept input words of `op`.
void trim_operator(qsd_ctx ctx, qsd_op op, qsd_sub sub, const double *diag, double tol, qsd_op out,
                   qsd_trim_info *info);

// Complex product (apply_complex.cu): x, y complex128 [D][k] interleaved.
void apply_H_complex(qsd_ctx ctx, qsd_op op, qsd_sub sub, int k, const void *x, void *y);

// RAMPS refinement from the rows of `start` (ramps.cu); `out` is a fresh
// subspace handle (ctx, n_qubits, W set) that receives the output rows.
void ramps(qsd_ctx ctx, qsd_op op, qsd_sub start, double E, double tau, int max_levels, qsd_sub allowed,
           int64_t max_rows, qsd_sub out, qsd_ramps_info *info);

int product_path(qsd_ctx ctx, qsd_op op, qsd_sub sub, const double *diag, int precision, int KB, const void *x,
                 void *y, int64_t ld, int64_t col0, cudaStream_t stream, bool may_tune);
void target_table(qsd_ctx ctx, qsd_op op, qsd_sub sub, int64_t row0, int64_t nrows, int64_t *out);
void term_table(qsd_ctx ctx, qsd_op op, qsd_sub sub, int64_t row0, int64_t nrows, int8_t *out);
void rayleigh_quotient(qsd_ctx ctx, qsd_op op, qsd_sub sub, const double *diag, const double *u, double *out);
int lanczos_ground_state(qsd_ctx ctx, qsd_op op, qsd_sub sub, const qsd_lanczos_params &p,
                         double *energy, double *vec_out, qsd_lanczos_info *info);

// Read and clear the device error word (synchronises the stream).
uint32_t take_device_error(qsd_ctx ctx);

inline int blocks_for(int64_t n, int threads) { return (int)((n + threads - 1) / threads); }
inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace qsd
