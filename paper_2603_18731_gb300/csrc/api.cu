// C ABI entry points (include/qsd.h): argument checks, handle management,
// error translation, and the host side of the product dispatch.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>

#include "apply_fv.cuh"
#include "factor_kernel.cuh"
#include "qsd_internal.cuh"

namespace qsd {

thread_local std::string g_thread_error;

void fail(int code, const std::string &msg) { throw Error(code, msg); }

void cuda_check(cudaError_t e, const char *what, const char *file, int line) {
    if (e == cudaSuccess) return;
    const int code = (e == cudaErrorMemoryAllocation) ? QSD_ERR_OOM : QSD_ERR_CUDA;
    const char *f = std::strrchr(file, '/');
    throw Error(code, std::string(what) + ": " + cudaGetErrorString(e) + " (" + (f ? f + 1 : file) + ":" +
                          std::to_string(line) + ")");
}

// Test hook: the next g_fail_allocs device allocations fail as if the
// device were out of memory (no CUDA call is made for them).
static std::atomic<int64_t> g_fail_allocs{0};

static bool injected_failure() {
    int64_t n = g_fail_allocs.load();
    while (n > 0)
        if (g_fail_allocs.compare_exchange_weak(n, n - 1)) return true;
    return false;
}

void DevBuf::alloc(size_t n) {
    release();
    if (n == 0) return;
    if (injected_failure())
        throw Error(QSD_ERR_OOM, "device allocation of " + std::to_string(n) + " bytes failed: injected failure");
    const cudaError_t e = cudaMalloc(&p, n);
    if (e != cudaSuccess) {
        p = nullptr;
        (void)cudaGetLastError();
        throw Error(QSD_ERR_OOM, "device allocation of " + std::to_string(n) + " bytes failed: " + cudaGetErrorString(e));
    }
    bytes = n;
}

void DevBuf::alloc_async(size_t n, cudaStream_t s) { alloc_pool(n, nullptr, s); }

void DevBuf::alloc_pool(size_t n, cudaMemPool_t pool, cudaStream_t s) {
    release();
    if (n == 0) return;
    if (injected_failure())
        throw Error(QSD_ERR_OOM, "device allocation of " + std::to_string(n) + " bytes failed: injected failure");
    const cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, n, pool, s) : cudaMallocAsync(&p, n, s);
    if (e != cudaSuccess) {
        p = nullptr;
        (void)cudaGetLastError();
        throw Error(QSD_ERR_OOM, "device allocation of " + std::to_string(n) + " bytes failed: " + cudaGetErrorString(e));
    }
    bytes = n;
    stream = s;
    async = true;
}

void DevBuf::release() {
    if (p) {
        if (async) cudaFreeAsync(p, stream);
        else cudaFree(p);
    }
    p = nullptr;
    bytes = 0;
    async = false;
    stream = nullptr;
}

// ------------------------------------------------------------ hash tables
namespace {
uint64_t splitmix_next(uint64_t &state) {
    state += 0x9E3779B97F4A7C15ull;
    return fmix64(state);
}
std::mutex g_nib_mu;
std::vector<uint64_t> g_nib;  // [W*256]
int g_nib_words = 0;
}  // namespace

std::vector<uint64_t> host_nibble_tables(int W) {
    std::lock_guard<std::mutex> lk(g_nib_mu);
    if (W > g_nib_words) {
        // random GF(2) columns Q[q] for qubits 0..64W-1, fixed seed (the
        // columns of a smaller W are a prefix: tables only ever grow)
        uint64_t st = 0x5153445F48415348ull;  // "QSD_HASH"
        std::vector<uint64_t> Q((size_t)64 * W);
        for (auto &v : Q) v = splitmix_next(st);
        g_nib.assign((size_t)W * 256, 0);
        for (int w = 0; w < W; ++w)
            for (int j = 0; j < 16; ++j)
                for (int v = 0; v < 16; ++v) {
                    uint64_t h = 0;
                    for (int b = 0; b < 4; ++b)
                        if ((v >> b) & 1) h ^= Q[(size_t)64 * w + 4 * j + b];
                    g_nib[(size_t)w * 256 + j * 16 + v] = h;
                }
        g_nib_words = W;
    }
    // a copy taken under the lock: another thread may grow the tables
    return std::vector<uint64_t>(g_nib.begin(), g_nib.begin() + (size_t)W * 256);
}

void ensure_nibble_tables(qsd_ctx ctx, int W) {
    const int want = std::max(W, 8);
    if (ctx->nib_words >= want) return;
    const std::vector<uint64_t> t = host_nibble_tables(want);
    QSD_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->nib.alloc(t.size() * 8);
    QSD_CUDA(cudaMemcpy(ctx->nib.p, t.data(), t.size() * 8, cudaMemcpyHostToDevice));
    ctx->nib_words = want;
}

uint32_t take_device_error(qsd_ctx ctx) {
    QSD_CUDA(cudaMemcpyAsync(ctx->h_err, ctx->d_err, 4, cudaMemcpyDeviceToHost, ctx->stream));
    QSD_CUDA(cudaStreamSynchronize(ctx->stream));
    const uint32_t e = *ctx->h_err;
    if (e) QSD_CUDA(cudaMemsetAsync(ctx->d_err, 0, 4, ctx->stream));
    return e;
}

// ------------------------------------------------------------ bindings
Binding *get_binding(qsd_ctx ctx, qsd_op op, qsd_sub sub) {
    auto key = std::make_pair((const void *)op, (const void *)sub);
    auto it = ctx->bindings.find(key);
    if (it != ctx->bindings.end()) return it->second;
    auto *b = new Binding();
    try {
        b->diag.alloc((size_t)std::max<int64_t>(sub->D, 1) * 8);
        compute_diagonal(ctx, op, sub, b->diag.as<double>());
        QSD_CUDA(cudaStreamSynchronize(ctx->stream));
    } catch (...) {
        delete b;
        throw;
    }
    ctx->bindings[key] = b;
    return b;
}

// ------------------------------------------------ linear half-sum tables
// Per (operator, subspace) pair, shared by every context that runs the pair's
// factored product; dropped when either handle is freed.
namespace {
struct HalvesEntry {
    DevBuf sa, sb;
    bool built = false;
};
bool capturing(cudaStream_t s);  // below
std::mutex g_halves_mu;
std::map<std::pair<const void *, const void *>, std::unique_ptr<HalvesEntry>> g_halves;
}  // namespace

LinearHalves linear_halves(qsd_ctx ctx, qsd_op op, qsd_sub sub, cudaStream_t s, bool may_build) {
    LinearHalves out;
    if (!ctx->linear_halves || op->n_lin_rows <= 0 || !sub->fac.ok) return out;
    std::lock_guard<std::mutex> lk(g_halves_mu);
    const auto key = std::make_pair((const void *)op, (const void *)sub);
    auto it = g_halves.find(key);
    if (it == g_halves.end()) {
        if (!may_build || capturing(s)) return out;  // never allocate or build inside a capture
        auto e = std::make_unique<HalvesEntry>();
        e->built = build_linear_halves(ctx, op, sub, s, e->sa, e->sb);
        it = g_halves.emplace(key, std::move(e)).first;
    }
    if (it->second->built) {
        out.sa = it->second->sa.as<int64_t>();
        out.sb = it->second->sb.as<int64_t>();
    }
    return out;
}

void drop_linear_halves(const void *handle) {
    std::lock_guard<std::mutex> lk(g_halves_mu);
    for (auto it = g_halves.begin(); it != g_halves.end();) {
        if (it->first.first == handle || it->first.second == handle) it = g_halves.erase(it);
        else ++it;
    }
}

void prepare_product(qsd_ctx ctx, qsd_op op, qsd_sub sub, cudaStream_t s) {
    if (sub->fac.ok && op->n_lin_rows > 0) (void)linear_halves(ctx, op, sub, s);
}

void drop_bindings(qsd_ctx ctx, const void *handle) {
    if (ctx->csr.op == handle || ctx->csr.sub == handle) ctx->csr.clear();
    {
        std::lock_guard<std::mutex> lk(ctx->tune_mu);
        for (auto it = ctx->tune_cache.begin(); it != ctx->tune_cache.end();) {
            if (std::get<0>(it->first) == handle || std::get<1>(it->first) == handle) it = ctx->tune_cache.erase(it);
            else ++it;
        }
    }
    for (auto it = ctx->bindings.begin(); it != ctx->bindings.end();) {
        if (it->first.first == handle || it->first.second == handle) {
            delete it->second;
            it = ctx->bindings.erase(it);
        } else {
            ++it;
        }
    }
}

// ------------------------------------------------------------ product
// Lanes per row: a lane per row once the rows fill the GPU; 8 lanes per row
// for small subspaces with enough groups to share.
static int choose_lanes(qsd_ctx ctx, int64_t D, int64_t G) {
    if (ctx->tune_lanes == 1 || ctx->tune_lanes == 8) return ctx->tune_lanes;
    const int64_t slots = (int64_t)ctx->num_sms * 2048;
    return (D < slots / 2 && G >= 16) ? 8 : 1;
}

// Excitation path when a row reaches far fewer candidate flip masks than the
// operator has groups (the per-row scan visits every group).
static bool use_excitation(qsd_ctx ctx, qsd_op op, qsd_sub sub) {
    if (!op->exc_ok || ctx->tune_mode == 1) return false;
    if (ctx->tune_mode == 2) return true;
    const double cand = excitation_candidates(op, sub);
    return cand >= 0.0 && 4.0 * cand < (double)op->G;
}

// The sector-factored path applies when the subspace is the product of its
// halves at the operator's sector split and the operator's ladder groups have
// a dense rank index (W <= 2).
static bool use_factored(qsd_ctx ctx, qsd_op op, qsd_sub sub) {
    if (ctx->tune_mode == 1 || ctx->tune_mode == 2 || ctx->tune_mode == 3) return false;
    return sub->fac.ok && op->exc_ok && op->dense_ok && op->W <= 2 && op->exc_split == sub->fac.split &&
           op->trec.p != nullptr && op->lin_base.p != nullptr;
}

// The filter/verify scan applies to single-column and 16-column products of
// operators whose groups are all table groups, over subspaces with a hash
// order and an occupancy filter (W <= 4), within its shared-memory staging
// limits.
static bool fv_ok(qsd_ctx ctx, qsd_op op, qsd_sub sub, int KB) {
    return (KB == 1 || KB == 16) && op->W <= kMaxWordsStatic && sub->hperm.p != nullptr && sub->occ.p != nullptr &&
           op->G >= 1 &&
           op->n_table_groups == op->G && op->G <= kFvMaxGroups && op->n_amp <= kFvMaxAmps &&
           fv_smem_bytes(op->G, op->n_amp) <= 48 * 1024 && ctx->row_order != 1;
}

namespace {

ApplyParams make_params(qsd_ctx ctx, qsd_op op, qsd_sub sub, const double *diag, int k, const void *x, void *y) {
    ApplyParams p{};
    p.keys = sub->keys.as<uint64_t>();
    p.D = sub->D;
    p.hv = hash_view(sub);
    p.nib = ctx->nib.as<uint64_t>();
    p.G = op->G;
    p.grec = op->grec.as<GroupRec>();
    p.amp = op->amp.as<double>();
    p.ampf = op->ampf.as<float2>();
    p.n_amp = op->n_amp;
    p.table_nb = -1;
    if (op->min_table_size == op->max_table_size && op->max_table_size == 1) p.table_nb = 0;
    if (op->min_table_size == op->max_table_size && op->max_table_size == 4 && op->n_qubits <= 256) p.table_nb = 2;
    p.gF = op->gF.as<uint64_t>();
    p.grange = op->grange.as<int32_t>();
    p.gL = op->gL.as<uint8_t>();
    p.gpos = op->gpos.as<uint64_t>();
    p.gptr = op->gptr.as<int32_t>();
    p.T = op->T;
    p.tP = op->tP.as<uint64_t>();
    p.tV = op->tV.as<uint64_t>();
    p.tZ = op->tZ.as<uint64_t>();
    p.tphi = op->tphi.as<double>();
    p.tflag = op->tflag.as<uint8_t>();
    p.diag = diag;
    p.rhash = sub->rhash.as<uint64_t>();
    p.hperm = sub->hperm.as<uint32_t>();
    p.hkeys = sub->hkeys.as<uint64_t>();
    p.hhash = sub->hhash.as<uint64_t>();
    p.x = x;
    p.y = y;
    p.ld = k;
    p.err = ctx->d_err;
    p.num_sms = ctx->num_sms;
    return p;
}

ExcParams make_exc(qsd_op op) {
    ExcParams e{};
    e.ght = HashView{op->gtags.as<uint8_t>(), op->gsidx.as<uint32_t>(), op->excF.as<uint64_t>(), op->G_exc,
                     (uint64_t)op->g_nbuckets - 1, op->g_shift};
    e.exc_gid = op->exc_gid.as<int32_t>();
    e.dense = op->dense_ok ? op->dense.as<int32_t>() : nullptr;
    for (int i = 0; i < op->n_shapes; ++i) {
        e.dbase[i] = op->dbase[i];
        e.dstride[i] = op->dstride[i];
    }
    e.rest_gid = op->rest_gid.as<int32_t>();
    e.n_rest = op->G_rest;
    e.split = op->exc_split;
    e.n_qubits = op->n_qubits;
    e.n_shapes = op->n_shapes;
    for (int i = 0; i < op->n_shapes; ++i) e.shapes[i] = op->shapes[i];
    return e;
}

FacParams make_fac(qsd_ctx ctx, qsd_op op, qsd_sub sub, cudaStream_t stream, bool may_build = true) {
    const Factored &f = sub->fac;
    FacParams r{};
    const LinearHalves lh = linear_halves(ctx, op, sub, stream, may_build);
    r.lsA = lh.sa;
    r.lsB = lh.sb;
    r.nlr = op->n_lin_rows;
    r.trec = op->trec.p;
    r.qscale = op->qscale;
    r.qexp = op->qexp;
    r.lin_base = op->lin_base.as<int32_t>();
    r.lin_z = op->lin_z.as<uint64_t>();
    r.lin_kq = op->lin_kq.as<int64_t>();
    r.lin_dq = op->lin_dq.as<int64_t>();
    r.nq = op->n_qubits;
    r.rix = op->range_ok ? op->rix.as<uint32_t>() : nullptr;
    r.A = f.A.as<uint64_t>();
    r.B = f.B.as<uint64_t>();
    r.ptrA = f.ptrA.as<uint32_t>();
    r.ptrB = f.ptrB.as<uint32_t>();
    r.nbrA = f.nbrA.as<uint2>();
    r.nbrB = f.nbrB.as<uint2>();
    r.nA = (uint32_t)f.nA;
    r.nB = (uint32_t)f.nB;
    r.split = f.split;
    return r;
}

// Product paths: 0 = per-row group scan with one lane per row, 1 = the same
// with 8 lanes per row, 2 = excitation index (warp per row), 3 and 4 = the
// half-evaluation scan (lower-triangle groups, mirrored by atomic adds) with
// 1 or 8 lanes per row, 5 and 6 = paths 0 and 3 with the rows in hash order,
// 7 = sector-factored enumeration (warp per row, product subspaces),
// 8 = filter/verify scan (lane per row, hash order, table groups, k = 1).
void launch_path(int path, const ApplyParams &p, const ExcParams &e, const FacParams &f, int W, int precision,
                 int KB, cudaStream_t stream) {
    if (path == 8) {
        const int na = (int)p.n_amp;
        const int nb = p.table_nb;
        if (precision == QSD_FP64) launch_apply_fv<QSD_FP64>(p, na, W, nb, KB, p.num_sms, stream);
        else if (precision == QSD_FP32_MIXED) launch_apply_fv<QSD_FP32_MIXED>(p, na, W, nb, KB, p.num_sms, stream);
        else launch_apply_fv<QSD_FP32_DOT2>(p, na, W, nb, KB, p.num_sms, stream);
        return;
    }
    if (path == 7) {
        if (precision == QSD_FP64) launch_apply_fac<QSD_FP64>(p, e, f, W, KB, stream);
        else if (precision == QSD_FP32_MIXED) launch_apply_fac<QSD_FP32_MIXED>(p, e, f, W, KB, stream);
        else launch_apply_fac<QSD_FP32_DOT2>(p, e, f, W, KB, stream);
        return;
    }
    if (path == 3 || path == 4 || path == 6) {
        launch_apply_sym(p, W, path == 4 ? 8 : 1, KB, stream, path == 6);
        return;
    }
    if (path == 2) {
        if (precision == QSD_FP64) launch_apply_exc<QSD_FP64>(p, e, W, KB, stream);
        else if (precision == QSD_FP32_MIXED) launch_apply_exc<QSD_FP32_MIXED>(p, e, W, KB, stream);
        else launch_apply_exc<QSD_FP32_DOT2>(p, e, W, KB, stream);
        return;
    }
    const int R = path == 1 ? 8 : 1;
    const bool ho = path == 5;
    if (precision == QSD_FP64) launch_apply<QSD_FP64>(p, W, R, KB, stream, ho);
    else if (precision == QSD_FP32_MIXED) launch_apply<QSD_FP32_MIXED>(p, W, R, KB, stream, ho);
    else launch_apply<QSD_FP32_DOT2>(p, W, R, KB, stream, ho);
}

// The half-evaluation counterpart of a scan path.
int half_of(int path) { return path == 5 ? 6 : path + 3; }

int heuristic_path(qsd_ctx ctx, qsd_op op, qsd_sub sub) {
    if (use_factored(ctx, op, sub)) return 7;
    if (use_excitation(ctx, op, sub)) return 2;
    return choose_lanes(ctx, sub->D, op->G) == 8 ? 1 : 0;
}

bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(s, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone;
}

}  // namespace

ApplyParams product_params(qsd_ctx ctx, qsd_op op, qsd_sub sub, const double *diag, int k, const void *x, void *y) {
    return make_params(ctx, op, sub, diag, k, x, y);
}

FacPair factored_params(qsd_ctx ctx, qsd_op op, qsd_sub sub, const double *diag, int k, const void *x, void *y) {
    return FacPair{make_params(ctx, op, sub, diag, k, x, y), make_exc(op), make_fac(ctx, op, sub, ctx->stream)};
}

int pack_class(qsd_ctx ctx, qsd_op op, qsd_sub sub, bool lanes8) {
    if (use_factored(ctx, op, sub)) return kPackFacClass + op->W - 1;
    if (op->W > kMaxWordsStatic) return -1;
    if (lanes8 && choose_lanes(ctx, sub->D, op->G) == 8) return kPackScan8Class + op->W - 1;
    return op->W - 1;
}

// Path for (op, sub, precision, KB): a forced choice, the tuned choice in
// the context's cache, a fresh measurement (when allowed), or the heuristic.
int product_path(qsd_ctx ctx, qsd_op op, qsd_sub sub, const double *diag, int precision, int KB, const void *x,
                 void *y, int64_t ld, int64_t col0, cudaStream_t stream, bool may_tune) {
    // the half evaluation needs H = H^T (real Hermitian), FP64 storage and W <= 4
    const bool sym_ok = op->info.is_hermitian && op->info.is_real && precision == QSD_FP64 &&
                        op->W <= kMaxWordsStatic;
    // hash order: lane-per-row scans of subspaces that have one (W <= 4)
    const bool ho_ok = op->W <= kMaxWordsStatic && sub->hperm.p != nullptr;
    int lanes_path = (ctx->tune_lanes ? ctx->tune_lanes : choose_lanes(ctx, sub->D, op->G)) == 8 ? 1 : 0;
    if (lanes_path == 0 && ho_ok && ctx->row_order == 2) lanes_path = 5;
    if (ctx->tune_mode == 1 || (ctx->tune_mode == 3 && !sym_ok)) return lanes_path;
    if (ctx->tune_mode == 3) return half_of(lanes_path);
    if (ctx->tune_mode == 2 && op->exc_ok) return 2;
    if (ctx->tune_mode == 5 && fv_ok(ctx, op, sub, KB)) return 8;
    // a product subspace with an indexed operator: the factored enumeration
    // reaches only columns in S, so no other path is timed against it
    if (use_factored(ctx, op, sub)) return 7;
    const bool ho_open = ho_ok && ctx->row_order == 0 && lanes_path == 0;
    if (ctx->tune_lanes != 0 && !op->exc_ok && !(sym_ok && ctx->allow_sym) && !ho_open && !fv_ok(ctx, op, sub, KB))
        return lanes_path;
    const auto key = std::make_tuple((const void *)op, (const void *)sub, precision, KB);
    {
        std::lock_guard<std::mutex> lk(ctx->tune_mu);
        auto it = ctx->tune_cache.find(key);
        if (it != ctx->tune_cache.end()) return it->second;
    }
    const int guess = [&] {
        const int g = heuristic_path(ctx, op, sub);
        return (g == 0 && ho_ok && ctx->row_order == 2) ? 5 : g;
    }();
    if (!may_tune || !ctx->autotune || capturing(stream) || sub->D < 2048) return guess;
    // Candidates: the excitation index only where a row reaches fewer flip
    // masks than there are groups, the group scans only where the index does
    // not reach 16x fewer.  The heuristic's guess runs first; each candidate
    // runs once untimed (its first launch in a process loads its module, and
    // that would count against it) and then up to three times, stopping once
    // it is 4x slower than the best.
    const double cand = excitation_candidates(op, sub);
    std::vector<int> cands;
    if (guess == 2) cands.push_back(2);
    if (!(cand >= 0.0 && 16.0 * cand < (double)op->G)) {
        if (ctx->tune_lanes) {
            cands.push_back(lanes_path);
        } else {
            cands.push_back(guess == 1 ? 1 : 0);
            cands.push_back(guess == 1 ? 0 : 1);
        }
        if (ho_ok && ctx->row_order != 1) {
            // the lane-per-row scan in hash order: beside index order (auto)
            // or in its place (forced)
            bool had0 = false;
            for (int &c : cands)
                if (c == 0 && ctx->row_order == 2) c = 5;
                else if (c == 0) had0 = true;
            if (had0) cands.push_back(5);
        }
        if (sym_ok && ctx->allow_sym) {
            const size_t m = cands.size();
            for (size_t i = 0; i < m; ++i)
                if (cands[i] < 2 || cands[i] == 5) cands.push_back(half_of(cands[i]));
        }
    }
    if (guess != 2 && cand >= 0.0 && cand < (double)op->G) cands.push_back(2);
    if (fv_ok(ctx, op, sub, KB)) cands.push_back(8);
    if (cands.size() < 2) {
        std::lock_guard<std::mutex> lk(ctx->tune_mu);
        ctx->tune_cache[key] = guess;
        return guess;
    }
    ApplyParams p = make_params(ctx, op, sub, diag, (int)ld, x, y);
    p.col0 = col0;
    const ExcParams e = op->exc_ok ? make_exc(op) : ExcParams{};
    const FacParams f{};
    cudaEvent_t a, b;
    QSD_CUDA(cudaEventCreate(&a));
    QSD_CUDA(cudaEventCreate(&b));
    int best = guess;
    float best_ms = 1e30f;
    for (int c : cands) {
        float ms = 1e30f;
        launch_path(c, p, e, f, op->W, precision, KB, stream);
        for (int rep = 0; rep < 3; ++rep) {
            QSD_CUDA(cudaEventRecord(a, stream));
            launch_path(c, p, e, f, op->W, precision, KB, stream);
            QSD_CUDA(cudaEventRecord(b, stream));
            QSD_CUDA(cudaEventSynchronize(b));
            float t = 0.f;
            QSD_CUDA(cudaEventElapsedTime(&t, a, b));
            ms = std::min(ms, t);
            if (ms > 4.f * best_ms) break;
        }
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    std::lock_guard<std::mutex> lk(ctx->tune_mu);
    ctx->tune_cache[key] = best;
    return best;
}

namespace {
__global__ void k_widen(const float *__restrict__ x, int64_t n, double *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (double)x[i];
}
}  // namespace

void apply_H(qsd_ctx ctx, qsd_op op, qsd_sub sub, const double *diag, int precision, int k, const void *x, void *y,
             cudaStream_t stream, bool may_tune, bool may_allocate) {
    ApplyParams p = make_params(ctx, op, sub, diag, k, x, y);
    ExcParams e{};
    FacParams f{};
    bool have_e = false;
    // FP32-mixed block products on the factored and filter/verify paths: x
    // widened exactly to FP64 once (context scratch), then the FP64 block
    // kernel with FP32 y -- bitwise the same product, without a conversion
    // per gathered value (which cost the factored gather loop 15 % more
    // instructions and a block of residency per SM)
    const double *xw = nullptr;
    const bool may_widen = precision == QSD_FP32_MIXED && k >= 4 && may_allocate && stream == ctx->stream &&
                           sub->D > 0 && !capturing(stream);
    int64_t c = 0;
    while (c < k) {
        const int KB = (k - c >= 16) ? 16 : (k - c >= 4 ? 4 : 1);
        p.col0 = c;
        const int path = product_path(ctx, op, sub, diag, precision, KB, x, y, k, c, stream, may_tune);
        if ((path == 2 || path == 7) && !have_e) {
            e = make_exc(op);
            f = make_fac(ctx, op, sub, stream, may_allocate);
            have_e = true;
        }
        const bool wide = may_widen && ((path == 7 && KB > 1) || (path == 8 && KB == 16));
        if (wide && !xw) {
            const int64_t n = sub->D * (int64_t)k;
            double *buf = static_cast<double *>(ctx->scratch[4].get((size_t)n * 8));
            k_widen<<<(unsigned)std::min<int64_t>(blocks_for(n, 256), 8 * (int64_t)ctx->num_sms), 256, 0, stream>>>(
                static_cast<const float *>(x), n, buf);
            QSD_LAUNCH_CHECK();
            xw = buf;
        }
        if (wide) {
            ApplyParams pw = p;
            pw.x = xw;
            if (path == 7) launch_apply_fac<kPrecWideX>(pw, e, f, op->W, KB, stream);
            else launch_apply_fv<kFvWideX>(pw, (int)pw.n_amp, op->W, pw.table_nb, KB, pw.num_sms, stream);
        } else {
            launch_path(path, p, e, f, op->W, precision, KB, stream);
        }
        c += KB;
    }
}

}  // namespace qsd

using namespace qsd;

// ------------------------------------------------------------ ABI helpers
#define QSD_GUARD(ctxp, ...)                                           \
    do {                                                               \
        try {                                                          \
            __VA_ARGS__;                                               \
            return QSD_OK;                                             \
        } catch (const qsd::Error &e) {                                \
            if (ctxp) (ctxp)->last_error = e.what();                   \
            else qsd::g_thread_error = e.what();                       \
            return e.code;                                             \
        } catch (const std::bad_alloc &) {                             \
            if (ctxp) (ctxp)->last_error = "host allocation failed";   \
            return QSD_ERR_OOM;                                        \
        } catch (const std::exception &e) {                            \
            if (ctxp) (ctxp)->last_error = e.what();                   \
            return QSD_ERR_INTERNAL;                                   \
        }                                                              \
    } while (0)

static void set_device(qsd_ctx ctx) { QSD_CUDA(cudaSetDevice(ctx->device)); }

static int W_of(int32_t n) { return n <= 64 ? 1 : (n + 63) / 64; }

extern "C" {

int qsd_create(int device, void *cuda_stream, qsd_ctx *out) {
    qsd_ctx ctx = nullptr;
    try {
        if (!out) fail(QSD_ERR_INVALID_ARG, "qsd_create: out is NULL");
        int n = 0;
        QSD_CUDA(cudaGetDeviceCount(&n));
        if (device < 0 || device >= n) fail(QSD_ERR_INVALID_ARG, "qsd_create: no such device");
        ctx = new qsd_ctx_s();
        ctx->device = device;
        QSD_CUDA(cudaSetDevice(device));
        QSD_CUDA(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device));
        if (cuda_stream) {
            ctx->stream = (cudaStream_t)cuda_stream;
        } else {
            QSD_CUDA(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
            ctx->own_stream = true;
        }
        QSD_CUDA(cudaMalloc(&ctx->d_err, 4));
        QSD_CUDA(cudaMemset(ctx->d_err, 0, 4));
        QSD_CUDA(cudaMallocHost(&ctx->h_err, 4));
        {
            // the eigensolver's workspace pool keeps up to 1/16 of the
            // device's memory mapped between solves (a solve's basis is
            // (steps + 1) D values: mapping it anew cost a warm 300,000-row
            // solve about 0.4 ms of its 7.5)
            cudaMemPoolProps props{};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = device;
            QSD_CUDA(cudaMemPoolCreate(&ctx->pool, &props));
            size_t free_b = 0, total_b = 0;
            QSD_CUDA(cudaMemGetInfo(&free_b, &total_b));
            uint64_t keep = total_b / 16;
            QSD_CUDA(cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep));
        }
        ensure_nibble_tables(ctx, 8);
        *out = ctx;
        return QSD_OK;
    } catch (const qsd::Error &e) {
        g_thread_error = e.what();
        if (ctx) qsd_destroy(ctx);
        return e.code;
    } catch (const std::exception &e) {
        g_thread_error = e.what();
        if (ctx) qsd_destroy(ctx);
        return QSD_ERR_INTERNAL;
    }
}

int qsd_destroy(qsd_ctx ctx) {
    if (!ctx) return QSD_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    for (auto &kv : ctx->bindings) delete kv.second;
    ctx->bindings.clear();
    ctx->nib.release();
    for (auto &s : ctx->scratch) s.buf.release();
    if (ctx->d_err) cudaFree(ctx->d_err);
    if (ctx->h_err) cudaFreeHost(ctx->h_err);
    if (ctx->pool) {
        if (ctx->stream) cudaStreamSynchronize(ctx->stream);
        cudaMemPoolDestroy(ctx->pool);
    }
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return QSD_OK;
}

const char *qsd_last_error(qsd_ctx ctx) { return ctx ? ctx->last_error.c_str() : g_thread_error.c_str(); }

int qsd_inject_alloc_failures(int64_t n) {
    if (n < 0) return QSD_ERR_INVALID_ARG;
    g_fail_allocs.store(n);
    return QSD_OK;
}

int qsd_load_operator(qsd_ctx ctx, int32_t n_qubits, int64_t n_terms, const int64_t *term_ptr,
                      const int32_t *op_qubit, const uint8_t *op_code, const double *coef_re,
                      const double *coef_im, qsd_op *out) {
    if (!ctx) return QSD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    QSD_GUARD(ctx, {
        if (!out || n_qubits < 1) fail(QSD_ERR_INVALID_ARG, "qsd_load_operator: bad arguments");
        set_device(ctx);
        auto *op = new qsd_op_s();
        op->ctx = ctx;
        op->n_qubits = n_qubits;
        op->W = W_of(n_qubits);
        if (op->W > kMaxWordsDyn) {
            delete op;
            fail(QSD_ERR_INVALID_ARG, "qsd_load_operator: more than 4096 qubits");
        }
        try {
            load_operator(ctx, op, n_terms, term_ptr, op_qubit, op_code, coef_re, coef_im);
        } catch (...) {
            delete op;
            throw;
        }
        *out = op;
    });
}

int qsd_op_get_info(qsd_op op, qsd_op_info *info) {
    if (!op || !info) return QSD_ERR_INVALID_ARG;
    *info = op->info;
    return QSD_OK;
}

int qsd_op_groups(qsd_op op, uint64_t *groups_out) {
    if (!op || (!groups_out && op->G > 0)) return QSD_ERR_INVALID_ARG;
    if (op->G > 0) std::memcpy(groups_out, op->host_groups.data(), op->host_groups.size() * 8);
    return QSD_OK;
}

int qsd_free_op(qsd_op op) {
    if (!op) return QSD_ERR_INVALID_ARG;
    qsd_ctx ctx = op->ctx;
    std::lock_guard<std::mutex> lk(ctx->mu);
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    drop_bindings(ctx, op);
    drop_linear_halves(op);
    delete op;
    return QSD_OK;
}

int qsd_build_subspace(qsd_ctx ctx, int32_t n_qubits, int64_t n_in, const uint64_t *words, int words_on_device,
                       qsd_sub *out, int64_t *dim_out) {
    if (!ctx) return QSD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    QSD_GUARD(ctx, {
        if (!out || n_qubits < 1 || n_in < 0 || (n_in > 0 && !words))
            fail(QSD_ERR_INVALID_ARG, "qsd_build_subspace: bad arguments");
        set_device(ctx);
        auto *sub = new qsd_sub_s();
        sub->ctx = ctx;
        sub->n_qubits = n_qubits;
        sub->W = W_of(n_qubits);
        if (sub->W > kMaxWordsDyn) {
            delete sub;
            fail(QSD_ERR_INVALID_ARG, "qsd_build_subspace: more than 4096 qubits");
        }
        try {
            build_subspace(ctx, sub, words, n_in, words_on_device != 0);
        } catch (...) {
            delete sub;
            throw;
        }
        *out = sub;
        if (dim_out) *dim_out = sub->D;
    });
}

int qsd_subspace_info(qsd_sub sub, int64_t *dim, int32_t *n_qubits, int64_t *capacity) {
    if (!sub) return QSD_ERR_INVALID_ARG;
    if (dim) *dim = sub->D;
    if (n_qubits) *n_qubits = sub->n_qubits;
    if (capacity) *capacity = sub->n_buckets * kBucketSlots;
    return QSD_OK;
}

int qsd_subspace_factored(qsd_sub sub, int32_t *is_product, int32_t *split, int64_t *n_a, int64_t *n_b,
                          int64_t *neighbours) {
    if (!sub) return QSD_ERR_INVALID_ARG;
    const Factored &f = sub->fac;
    if (is_product) *is_product = f.ok ? 1 : 0;
    if (split) *split = f.ok ? f.split : 0;
    if (n_a) *n_a = f.nA;
    if (n_b) *n_b = f.nB;
    if (neighbours) *neighbours = f.nnzA + f.nnzB;
    return QSD_OK;
}

int qsd_subspace_keys(qsd_ctx ctx, qsd_sub sub, uint64_t *out, int out_on_device) {
    if (!ctx || !sub) return QSD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    QSD_GUARD(ctx, {
        if (sub->D > 0 && !out) fail(QSD_ERR_INVALID_ARG, "qsd_subspace_keys: out is NULL");
        set_device(ctx);
        if (sub->D == 0) return QSD_OK;
        if (out_on_device) {
            subspace_keys_aos(ctx, sub, out);
        } else {
            DevBuf tmp((size_t)sub->D * sub->W * 8);
            subspace_keys_aos(ctx, sub, tmp.as<uint64_t>());
            QSD_CUDA(cudaMemcpyAsync(out, tmp.p, tmp.bytes, cudaMemcpyDeviceToHost, ctx->stream));
            QSD_CUDA(cudaStreamSynchronize(ctx->stream));
        }
    });
}

int qsd_subspace_index(qsd_ctx ctx, qsd_sub sub, int64_t n, const uint64_t *keys, int64_t *idx_out) {
    if (!ctx || !sub) return QSD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    QSD_GUARD(ctx, {
        if (n < 0 || (n > 0 && (!keys || !idx_out))) fail(QSD_ERR_INVALID_ARG, "qsd_subspace_index: bad arguments");
        set_device(ctx);
        subspace_index(ctx, sub, n, keys, idx_out);
    });
}

int qsd_free_sub(qsd_sub sub) {
    if (!sub) return QSD_ERR_INVALID_ARG;
    qsd_ctx ctx = sub->ctx;
    std::lock_guard<std::mutex> lk(ctx->mu);
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    drop_bindings(ctx, sub);
    drop_linear_halves(sub);
    delete sub;
    return QSD_OK;
}

static void check_pair(qsd_ctx ctx, qsd_op op, qsd_sub sub) {
    if (!op || !sub) fail(QSD_ERR_INVALID_ARG, "NULL operator or subspace");
    if (op->ctx != ctx || sub->ctx != ctx) fail(QSD_ERR_INVALID_ARG, "handles belong to another context");
    if (op->n_qubits != sub->n_qubits)
        fail(QSD_ERR_INVALID_ARG, "operator has " + std::to_string(op->n_qubits) + " qubits, subspace " +
                                      std::to_string(sub->n_qubits));
}

int qsd_apply_H(qsd_ctx ctx, qsd_op op, qsd_sub sub, int precision, int32_t k, const void *x, void *y) {
    if (!ctx) return QSD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    QSD_GUARD(ctx, {
        check_pair(ctx, op, sub);
        if (k < 1 || precision < QSD_FP64 || precision > QSD_FP32_DOT2)
            fail(QSD_ERR_INVALID_ARG, "qsd_apply_H: bad k or precision");
        if (!op->info.is_real) fail(QSD_ERR_COMPLEX_UNSUPPORTED, "qsd_apply_H: operator has complex matrix elements");
        if (sub->D == 0) return QSD_OK;
        if (!x || !y) fail(QSD_ERR_INVALID_ARG, "qsd_apply_H: NULL vector");
        set_device(ctx);
        Binding *b = get_binding(ctx, op, sub);
        apply_H(ctx, op, sub, b->diag.as<double>(), precision, k, x, y, ctx->stream, true);
    });
}

int qsd_apply_H_complex(qsd_ctx ctx, qsd_op op, qsd_sub sub, int32_t k, const void *x, void *y) {
    if (!ctx) return QSD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    QSD_GUARD(ctx, {
        check_pair(ctx, op, sub);
        if (k < 1) fail(QSD_ERR_INVALID_ARG, "qsd_apply_H_complex: k < 1");
        if (op->W > kMaxWordsStatic) fail(QSD_ERR_INVALID_ARG, "qsd_apply_H_complex: more than 256 qubits");
        if (sub->D == 0) return QSD_OK;
        if (!x || !y) fail(QSD_ERR_INVALID_ARG, "qsd_apply_H_complex: NULL vector");
        set_device(ctx);
        apply_H_complex(ctx, op, sub, k, x, y);
    });
}

int qsd_apply_H_batch(qsd_ctx ctx, int32_t n, const qsd_op *ops, const qsd_sub *subs, int precision, int32_t k,
                      const void *const *xs, void *const *ys) {
    if (!ctx) return QSD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    QSD_GUARD(ctx, {
        if (n < 0 || (n > 0 && (!ops || !subs || !xs || !ys)) || k < 1 || precision < QSD_FP64 ||
            precision > QSD_FP32_DOT2)
            fail(QSD_ERR_INVALID_ARG, "qsd_apply_H_batch: bad n, arrays, k or precision");
        set_device(ctx);
        // pairs by packed class (key width; factored or scan); empty
        // subspaces need no work
        std::map<int, std::vector<int>> by_class;
        std::vector<const double *> diag(n);
        for (int i = 0; i < n; ++i) {
            check_pair(ctx, ops[i], subs[i]);
            if (!ops[i]->info.is_real) fail(QSD_ERR_COMPLEX_UNSUPPORTED, "qsd_apply_H_batch: complex operator");
            if (ops[i]->W > kMaxWordsStatic) fail(QSD_ERR_INVALID_ARG, "qsd_apply_H_batch: more than 256 qubits");
            if (subs[i]->D == 0) continue;
            if (!xs[i] || !ys[i]) fail(QSD_ERR_INVALID_ARG, "qsd_apply_H_batch: NULL vector");
            diag[i] = get_binding(ctx, ops[i], subs[i])->diag.as<double>();
            by_class[pack_class(ctx, ops[i], subs[i], false)].push_back(i);
        }
        cudaStream_t s = ctx->stream;
        for (auto &[cls, idx] : by_class) {
            const bool fac = cls >= kPackFacClass;
            const int W = pack_class_width(cls);
            const int rows = pack_class_rows(cls);
            const size_t rec = fac ? sizeof(FacPair) : sizeof(ApplyParams);
            const int m = (int)idx.size();
            // device block: queue, tile starts, parameter records
            const size_t o_t = align_up(sizeof(TileQueue), 256), o_p = align_up(o_t + (size_t)m * 8, 256);
            std::vector<unsigned char> h(o_p + (size_t)m * rec);
            TileQueue *hq = reinterpret_cast<TileQueue *>(h.data());
            int64_t *t0 = reinterpret_cast<int64_t *>(h.data() + o_t);
            int64_t tiles = 0;
            for (int j = 0; j < m; ++j) {
                t0[j] = tiles;
                tiles += (subs[idx[j]]->D + rows - 1) / rows;
            }
            if (tiles >= (int64_t)0x7fffffff) fail(QSD_ERR_CAPACITY, "qsd_apply_H_batch: too many rows");
            hq->n = m;
            hq->tiles = tiles;  // claim counters zero
            DevBuf d;
            d.alloc_async(h.size(), s);
            unsigned char *dd = static_cast<unsigned char *>(d.p);
            for (int64_t c = 0; c < k;) {
                const int KB = (k - c >= 16) ? 16 : (k - c >= 4 ? 4 : 1);
                for (int j = 0; j < m; ++j) {
                    const int i = idx[j];
                    ApplyParams ap = make_params(ctx, ops[i], subs[i], diag[i], k, xs[i], ys[i]);
                    ap.col0 = c;
                    if (fac) {
                        FacPair fp{ap, make_exc(ops[i]), make_fac(ctx, ops[i], subs[i], s)};
                        std::memcpy(h.data() + o_p + (size_t)j * rec, &fp, rec);
                    } else {
                        std::memcpy(h.data() + o_p + (size_t)j * rec, &ap, rec);
                    }
                }
                // pageable source: the copy is staged before the call returns;
                // the queue's counters are back at zero after each launch
                QSD_CUDA(cudaMemcpyAsync(dd, h.data(), h.size(), cudaMemcpyHostToDevice, s));
                TileQueue *dq = reinterpret_cast<TileQueue *>(dd);
                const int64_t *dt = reinterpret_cast<const int64_t *>(dd + o_t);
                if (fac) {
                    const FacPair *dp = reinterpret_cast<const FacPair *>(dd + o_p);
                    if (precision == QSD_FP64)
                        launch_apply_fac_queue<QSD_FP64>(dp, dt, dq, tiles, W, KB, ctx->num_sms, s);
                    else if (precision == QSD_FP32_MIXED)
                        launch_apply_fac_queue<QSD_FP32_MIXED>(dp, dt, dq, tiles, W, KB, ctx->num_sms, s);
                    else
                        launch_apply_fac_queue<QSD_FP32_DOT2>(dp, dt, dq, tiles, W, KB, ctx->num_sms, s);
                } else {
                    launch_apply_queue(reinterpret_cast<const ApplyParams *>(dd + o_p), dt, dq, tiles, W, 1, KB,
                                       precision, ctx->num_sms, s);
                }
                c += KB;
            }
        }
    });
}

int qsd_apply_H_host(qsd_ctx ctx, qsd_op op, qsd_sub sub, int precision, int32_t k, const void *x_host,
                     void *y_host) {
    if (!ctx) return QSD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    QSD_GUARD(ctx, {
        check_pair(ctx, op, sub);
        if (k < 1 || precision < QSD_FP64 || precision > QSD_FP32_DOT2)
            fail(QSD_ERR_INVALID_ARG, "qsd_apply_H_host: bad k or precision");
        if (!op->info.is_real) fail(QSD_ERR_COMPLEX_UNSUPPORTED, "qsd_apply_H_host: complex operator");
        if (sub->D == 0) return QSD_OK;
        if (!x_host || !y_host) fail(QSD_ERR_INVALID_ARG, "qsd_apply_H_host: NULL vector");
        set_device(ctx);
        Binding *b = get_binding(ctx, op, sub);
        const size_t bytes = (size_t)sub->D * k * (precision == QSD_FP64 ? 8 : 4);
        Scratch &sx = ctx->scratch[0], &sy = ctx->scratch[1];
        void *dx = sx.get(bytes), *dy = sy.get(bytes);
        QSD_CUDA(cudaMemcpyAsync(dx, x_host, bytes, cudaMemcpyHostToDevice, ctx->stream));
        apply_H(ctx, op, sub, b->diag.as<double>(), precision, k, dx, dy, ctx->stream, true);
        QSD_CUDA(cudaMemcpyAsync(y_host, dy, bytes, cudaMemcpyDeviceToHost, ctx->stream));
        QSD_CUDA(cudaStreamSynchronize(ctx->stream));
    });
}

int qsd_diagonal(qsd_ctx ctx, qsd_op op, qsd_sub sub, double *d_out) {
    if (!ctx) return QSD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    QSD_GUARD(ctx, {
        check_pair(ctx, op, sub);
        if (sub->D == 0) return QSD_OK;
        if (!d_out) fail(QSD_ERR_INVALID_ARG, "qsd_diagonal: NULL output");
        set_device(ctx);
        Binding *b = get_binding(ctx, op, sub);
        QSD_CUDA(cudaMemcpyAsync(d_out, b->diag.p, (size_t)sub->D * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    });
}

int qsd_target_table(qsd_ctx ctx, qsd_op op, qsd_sub sub, int64_t row0, int64_t nrows, int64_t *out) {
    if (!ctx) return QSD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    QSD_GUARD(ctx, {
        check_pair(ctx, op, sub);
        if (row0 < 0 || nrows < 0 || row0 + nrows > sub->D) fail(QSD_ERR_INVALID_ARG, "qsd_target_table: bad row range");
        if (nrows > 0 && op->G > 0 && !out) fail(QSD_ERR_INVALID_ARG, "qsd_target_table: NULL output");
        set_device(ctx);
        target_table(ctx, op, sub, row0, nrows, out);
    });
}

int qsd_term_table(qsd_ctx ctx, qsd_op op, qsd_sub sub, int64_t row0, int64_t nrows, int8_t *out) {
    if (!ctx) return QSD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    QSD_GUARD(ctx, {
        check_pair(ctx, op, sub);
        if (row0 < 0 || nrows < 0 || row0 + nrows > sub->D) fail(QSD_ERR_INVALID_ARG, "qsd_term_table: bad row range");
        if (nrows > 0 && op->T_in > 0 && !out) fail(QSD_ERR_INVALID_ARG, "qsd_term_table: NULL output");
        set_device(ctx);
        term_table(ctx, op, sub, row0, nrows, out);
    });
}

int qsd_rayleigh_quotient(qsd_ctx ctx, qsd_op op, qsd_sub sub, const double *u, double *out) {
    if (!ctx) return QSD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    QSD_GUARD(ctx, {
        check_pair(ctx, op, sub);
        if (!u || !out || sub->D == 0) fail(QSD_ERR_INVALID_ARG, "qsd_rayleigh_quotient: bad arguments");
        if (!op->info.is_real) fail(QSD_ERR_COMPLEX_UNSUPPORTED, "qsd_rayleigh_quotient: complex operator");
        set_device(ctx);
        Binding *b = get_binding(ctx, op, sub);
        rayleigh_quotient(ctx, op, sub, b->diag.as<double>(), u, out);
    });
}

int qsd_set_tuning(qsd_ctx ctx, int32_t knob, int64_t value) {
    if (!ctx) return QSD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    switch (knob) {
    case QSD_TUNE_APPLY_PATH:
        if (value < 0 || value > 5) return QSD_ERR_INVALID_ARG;
        ctx->tune_mode = (int)value;
        return QSD_OK;
    case QSD_TUNE_LANES_PER_ROW:
        if (value != 0 && value != 1 && value != 8) return QSD_ERR_INVALID_ARG;
        ctx->tune_lanes = (int)value;
        return QSD_OK;
    case QSD_TUNE_HALF_EVALUATION:
        if (value != 0 && value != 1) return QSD_ERR_INVALID_ARG;
        ctx->allow_sym = (int)value;
        {
            std::lock_guard<std::mutex> lk2(ctx->tune_mu);
            ctx->tune_cache.clear();
        }
        return QSD_OK;
    case QSD_TUNE_LINEAR_HALVES:
        if (value != 0 && value != 1) return QSD_ERR_INVALID_ARG;
        ctx->linear_halves = (int)value;
        return QSD_OK;
    case QSD_TUNE_ROW_ORDER:
        if (value < 0 || value > 2) return QSD_ERR_INVALID_ARG;
        ctx->row_order = (int)value;
        {
            std::lock_guard<std::mutex> lk2(ctx->tune_mu);
            ctx->tune_cache.clear();
        }
        return QSD_OK;
    case QSD_TUNE_AUTOTUNE:
        if (value != 0 && value != 1) return QSD_ERR_INVALID_ARG;
        ctx->autotune = (int)value;
        if (!value) {
            std::lock_guard<std::mutex> lk2(ctx->tune_mu);
            ctx->tune_cache.clear();
        }
        return QSD_OK;
    default:
        return QSD_ERR_INVALID_ARG;
    }
}

int qsd_to_csr(qsd_ctx ctx, qsd_op op, qsd_sub sub, int32_t flags, int64_t *nnz_out, int64_t *indptr,
               void *indices, int32_t index_bits, double *data_re, double *data_im) {
    if (!ctx) return QSD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    QSD_GUARD(ctx, {
        check_pair(ctx, op, sub);
        if (!nnz_out) fail(QSD_ERR_INVALID_ARG, "qsd_to_csr: NULL nnz_out");
        if (flags & ~QSD_CSR_FULL) fail(QSD_ERR_INVALID_ARG, "qsd_to_csr: unknown flag bits");
        if (index_bits != 32 && index_bits != 64) fail(QSD_ERR_INVALID_ARG, "qsd_to_csr: index_bits must be 32 or 64");
        if (index_bits == 32 && sub->D > 0x7fffffffLL)
            fail(QSD_ERR_INVALID_ARG, "qsd_to_csr: dimension needs 64-bit indices");
        const bool sizing = !indptr && !indices && !data_re;
        if (!sizing && (!indptr || !indices || !data_re))
            fail(QSD_ERR_INVALID_ARG, "qsd_to_csr: indptr, indices and data_re must all be given (or all NULL)");
        const bool lower = !(flags & QSD_CSR_FULL);
        if (!op->info.is_hermitian && (lower || !op->info.is_real))
            fail(QSD_ERR_NOT_HERMITIAN, "qsd_to_csr: the triangle evaluation (and complex data) needs a Hermitian operator");
        if (!op->info.is_real && !sizing && !data_im)
            fail(QSD_ERR_COMPLEX_UNSUPPORTED, "qsd_to_csr: complex operator needs data_im");
        Binding *b = get_binding(ctx, op, sub);
        *nnz_out = to_csr(ctx, op, sub, lower, indptr, indices, index_bits, data_re, data_im, b->diag.as<double>());
    });
}

int qsd_trim_operator(qsd_ctx ctx, qsd_op op, qsd_sub sub, double tol, qsd_op *out, qsd_trim_info *info) {
    if (!ctx) return QSD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    QSD_GUARD(ctx, {
        check_pair(ctx, op, sub);
        if (!out || !(tol >= 0.0)) fail(QSD_ERR_INVALID_ARG, "qsd_trim_operator: NULL out or tol < 0");
        set_device(ctx);
        Binding *b = get_binding(ctx, op, sub);
        auto *o = new qsd_op_s();
        o->ctx = ctx;
        o->n_qubits = op->n_qubits;
        o->W = op->W;
        qsd_trim_info local{};
        try {
            trim_operator(ctx, op, sub, b->diag.as<double>(), tol, o, info ? info : &local);
        } catch (...) {
            delete o;
            throw;
        }
        *out = o;
    });
}

void qsd_lobpcg_default_params(qsd_lobpcg_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->k = 1;
    p->max_iters = 500;
    p->tol = 1e-9;
    p->precondition = 1;
}

int qsd_lobpcg(qsd_ctx ctx, qsd_op op, qsd_sub sub, const qsd_lobpcg_params *p, double *evals, double *evecs,
               qsd_lobpcg_info *info) {
    if (!ctx) return QSD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    int status = QSD_OK;
    const int rc = [&]() -> int {
        QSD_GUARD(ctx, {
            check_pair(ctx, op, sub);
            if (!p || !evals || !info) fail(QSD_ERR_INVALID_ARG, "qsd_lobpcg: NULL params, evals or info");
            if (p->k < 1 || p->k > 16 || sub->D < 3 * (int64_t)p->k)
                fail(QSD_ERR_INVALID_ARG, "qsd_lobpcg: need 1 <= k <= 16 and dim >= 3k");
            if (p->start != 0 && p->start != 1) fail(QSD_ERR_INVALID_ARG, "qsd_lobpcg: start must be 0 or 1");
            if (!op->info.is_real) fail(QSD_ERR_COMPLEX_UNSUPPORTED, "qsd_lobpcg: complex operator");
            if (!op->info.is_hermitian) fail(QSD_ERR_NOT_HERMITIAN, "qsd_lobpcg: operator is not Hermitian");
            set_device(ctx);
            Binding *b = get_binding(ctx, op, sub);
            status = lobpcg(ctx, op, sub, b->diag.as<double>(), *p, evals, evecs, info);
        });
    }();
    if (rc != QSD_OK) return rc;
    if (status != QSD_OK) ctx->last_error = "qsd_lobpcg: not converged";
    return status;
}

int qsd_ramps(qsd_ctx ctx, qsd_op op, qsd_sub start, double E, double tau, int32_t max_levels,
              qsd_sub restrict_to, int64_t max_rows, qsd_sub *out, qsd_ramps_info *info) {
    if (!ctx) return QSD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    QSD_GUARD(ctx, {
        check_pair(ctx, op, start);
        if (restrict_to) check_pair(ctx, op, restrict_to);
        if (!out || !info) fail(QSD_ERR_INVALID_ARG, "qsd_ramps: NULL out or info");
        if (!(E != 0.0 && std::isfinite(E)) || !(tau >= 0.0) || max_levels < 0)
            fail(QSD_ERR_INVALID_ARG, "qsd_ramps: E must be finite and nonzero, tau >= 0, max_levels >= 0");
        if (op->W > kMaxWordsStatic) fail(QSD_ERR_INVALID_ARG, "qsd_ramps: more than 256 qubits");
        set_device(ctx);
        auto *sub = new qsd_sub_s();
        sub->ctx = ctx;
        sub->n_qubits = op->n_qubits;
        sub->W = op->W;
        try {
            ramps(ctx, op, start, E, tau, max_levels, restrict_to, max_rows, sub, info);
        } catch (...) {
            delete sub;
            throw;
        }
        *out = sub;
    });
}

int qsd_product_path(qsd_ctx ctx, qsd_op op, qsd_sub sub, int32_t precision, int64_t k, int32_t *path_out) {
    if (!ctx) return QSD_ERR_INVALID_ARG;
    QSD_GUARD(ctx, {
        check_pair(ctx, op, sub);
        if (!path_out || k < 1) fail(QSD_ERR_INVALID_ARG, "NULL path_out or k < 1");
        if (precision < QSD_FP64 || precision > QSD_FP32_DOT2) fail(QSD_ERR_INVALID_ARG, "unknown precision");
        std::lock_guard<std::mutex> lk(ctx->mu);
        const int KB = k >= 16 ? 16 : (k >= 4 ? 4 : 1);
        *path_out = product_path(ctx, op, sub, nullptr, precision, KB, nullptr, nullptr, k, 0, ctx->stream, false);
    });
}

void qsd_lanczos_default_params(qsd_lanczos_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->precision = QSD_FP64;
    p->max_steps = 300;
    p->tol = 1e-9;
    p->refine_tol = 1e-10;
    p->check_every = 10;
    p->refine_steps = 30;
    p->max_refine = 5;
    p->use_graphs = 1;
    p->seed = 1;
    p->v0 = nullptr;
    p->time_limit_s = 0.0;
}

int qsd_lanczos_ground_state(qsd_ctx ctx, qsd_op op, qsd_sub sub, const qsd_lanczos_params *p, double *energy,
                             double *vec_out, qsd_lanczos_info *info) {
    if (!ctx) return QSD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    int rc = QSD_OK;
    try {
        check_pair(ctx, op, sub);
        if (!p || !energy || p->max_steps < 1 || p->check_every < 1 || p->precision < QSD_FP64 ||
            p->precision > QSD_FP32_DOT2)
            fail(QSD_ERR_INVALID_ARG, "qsd_lanczos_ground_state: bad arguments");
        if (!op->info.is_real) fail(QSD_ERR_COMPLEX_UNSUPPORTED, "qsd_lanczos_ground_state: complex operator");
        if (!op->info.is_hermitian) fail(QSD_ERR_NOT_HERMITIAN, "qsd_lanczos_ground_state: operator is not Hermitian");
        if (sub->D == 0) fail(QSD_ERR_INVALID_ARG, "qsd_lanczos_ground_state: empty subspace");
        set_device(ctx);
        rc = lanczos_ground_state(ctx, op, sub, *p, energy, vec_out, info);
        if (rc != QSD_OK && rc != QSD_ERR_NOT_CONVERGED) ctx->last_error = "lanczos: status " + std::to_string(rc);
        if (rc == QSD_ERR_NOT_CONVERGED) ctx->last_error = "lanczos: max_steps reached before tol";
    } catch (const qsd::Error &e) {
        ctx->last_error = e.what();
        rc = e.code;
    } catch (const std::exception &e) {
        ctx->last_error = e.what();
        rc = QSD_ERR_INTERNAL;
    }
    if (info) info->status = rc;
    return rc;
}

}  // extern "C"
