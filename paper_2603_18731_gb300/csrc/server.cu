// Continuous-batching ground-state server.
//
// Requests (operator, subspace, Lanczos parameters) are queued by any thread
// and admitted by one scheduler thread when a slot is free and their device
// footprint fits the byte budget (largest-first blocking is avoided: the
// queue is FIFO, but a request that does not fit while others run waits only
// until memory frees up; a request larger than the whole budget is admitted
// alone).  Each admitted request owns a CUDA stream and advances through a
// small state machine, one asynchronous piece at a time:
//   MAIN   graph-captured chunks of Lanczos steps (FP64 or FP32 basis)
//   RESID  Ritz vector, FP64 Rayleigh quotient and residual
//   REFINE FP64 Lanczos restarts from the Ritz vector (mixed precision only)
// The scheduler enqueues the next piece of a request as soon as its previous
// piece has passed (cudaEventQuery), so the work of all admitted requests
// overlaps on the device and a request arriving while others run starts as
// soon as a slot and memory free up.
//
// Small requests (at most `pack_rows` rows, with a packable product: the
// factored product or a group scan of few groups) are packed: whenever a
// pack's previous chunk has passed, one chunk of Lanczos steps is enqueued
// for all its members that wait for one -- a CUDA-graph replay whose
// launches serve every member (the products from device tile queues, each
// Lanczos kernel once for all), on the pack's stream -- so many small solves
// cost the launches of one.  Requests join and leave a pack at chunk
// boundaries; their other pieces (start, Ritz vector, residual) run on their
// own streams between chunks, ordered by the host.  All device memory of a request is
// stream-ordered (cudaMallocAsync / cudaFreeAsync), so admitting and retiring
// requests never synchronises the device.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <thread>

#include "lanczos.cuh"

namespace qsd {

namespace {

using Clock = std::chrono::steady_clock;

enum class RState { Queued, Main, ResidMain, Refine, ResidRefine, Done };

struct Request {
    uint64_t ticket = 0;
    qsd_op op = nullptr;
    qsd_sub sub = nullptr;
    qsd_lanczos_params p{};
    RState state = RState::Queued;
    int status = QSD_PENDING;
    double energy = 0.0;
    qsd_lanczos_info info{};
    size_t footprint = 0;
    int slot = -1;
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    bool inflight = false;
    bool cancel = false;
    bool admitted = false;
    bool packed = false;             // small request: chunks run in packed launches
    LanczosJob *want = nullptr;      // packed: job waiting for the pack's next chunk
    int in_pack = -1;                // packed: the pack whose chunk in flight holds the job
    std::unique_ptr<LanczosJob> J, K;
    std::unique_ptr<ResidJob> R;
    DevBuf diag, u, start;
    double prev = 0.0;
    int restarts = 0;
    Clock::time_point t_submit, t_admit, t_done;
};

size_t request_footprint(int64_t D, const qsd_lanczos_params &p, int num_sms) {
    const bool mixed = p.precision != QSD_FP64;
    size_t f = LanczosJob::footprint(D, p.max_steps, mixed, num_sms);
    f += (size_t)D * 8 * 5;  // diag, u, start, residual hu and r
    if (mixed) f += LanczosJob::footprint(D, std::max(p.refine_steps, 2), false, num_sms);
    return f;
}

}  // namespace

}  // namespace qsd

struct qsd_server_s {
    qsd_ctx ctx = nullptr;
    size_t budget = 0;
    int max_active = 1;
    std::vector<cudaStream_t> streams;
    std::vector<int> free_slots;
    std::mutex mu;
    std::condition_variable cv_done, cv_work;
    std::deque<qsd::Request *> queue;
    std::vector<qsd::Request *> active;
    std::map<uint64_t, qsd::Request *> all;
    size_t used = 0, peak = 0;
    uint64_t next_ticket = 1;
    int64_t completed = 0, failed = 0, admitted = 0;
    bool stop = false;
    std::thread th;
    qsd::Clock::time_point t0;
    std::string last_error;
    double *pinned = nullptr;  // 16 doubles of pinned host memory per slot
    // packs of small requests, one per product precision
    int64_t pack_rows = 0;  // packing off unless asked for (qsd_server_set_pack_rows)
    cudaStream_t pack_stream = nullptr;
    qsd::Pack pack[3];
    std::vector<qsd::Request *> pack_members[3];  // of each pack's chunk in flight
    cudaEvent_t pack_ev[3] = {nullptr, nullptr, nullptr};
    bool pack_inflight[3] = {false, false, false};
    int64_t packed_requests = 0, packed_chunks = 0;
};

namespace qsd {

namespace {

double secs(Clock::time_point a, Clock::time_point b) { return std::chrono::duration<double>(b - a).count(); }

// Called with S->mu held.  The counters move here, not at retirement, so
// that a waiter that sees the result also sees it counted.
void finish(qsd_server_s *S, Request *r, int status) {
    if (status == QSD_OK) ++S->completed;
    else ++S->failed;
    r->status = status;
    r->state = RState::Done;
    r->t_done = Clock::now();
    r->info.status = status;
}

// Enqueue the next asynchronous piece of an admitted request.
void advance(qsd_server_s *S, Request *r) {
    const qsd_lanczos_params &p = r->p;
    const bool mixed = p.precision != QSD_FP64;
    const double tol = p.tol > 0 ? p.tol : 1e-9;
    const bool graphs = p.use_graphs != 0;
    const bool late = p.time_limit_s > 0 && secs(r->t_admit, Clock::now()) > p.time_limit_s;
    if (r->cancel) { finish(S, r, QSD_ERR_CANCELLED); return; }
    switch (r->state) {
    case RState::Main: {
        const double phase_tol = mixed ? std::max(tol, 1e-5) : tol;
        if (r->J->chunks > 0 && (r->J->converged(phase_tol) || r->J->steps_done >= r->J->m || late)) {
            double theta, est, hb;
            int n;
            r->J->read(theta, est, hb, n);
            r->info.energy_unrefined = theta;
            r->info.steps += r->J->steps_done;
            r->info.applies += r->J->steps_done + 1;
            r->J->enqueue_ritz(r->u.as<double>());
            r->R->enqueue(r->op, r->sub, r->diag.as<double>(), r->u.as<double>());
            r->state = RState::ResidMain;
        } else if (r->packed) {
            r->want = r->J.get();
            return;  // the pack's next chunk records the event
        } else {
            r->J->enqueue_chunk(graphs);
        }
        break;
    }
    case RState::ResidMain:
    case RState::ResidRefine: {
        double rq, resid;
        r->R->read(rq, resid);
        r->info.residual = resid;
        bool converged;
        if (r->state == RState::ResidMain) {
            r->energy = mixed ? rq : r->info.energy_unrefined;
            converged = resid <= tol || (!mixed && r->J->converged(tol));
            r->prev = rq;
        } else {
            r->energy = rq;
            ++r->restarts;
            const double change = std::fabs(rq - r->prev) / std::max(std::fabs(rq), 1e-300);
            r->prev = rq;
            converged = resid <= tol || change <= (p.refine_tol > 0 ? p.refine_tol : 1e-10);
        }
        r->info.refine_restarts = r->restarts;
        if (late) { finish(S, r, QSD_ERR_TIMEOUT); return; }
        if (converged || !mixed || r->restarts >= std::max(p.max_refine, 0)) {
            finish(S, r, converged ? QSD_OK : QSD_ERR_NOT_CONVERGED);
            return;
        }
        if (!r->K) {
            r->K.reset(new LanczosJob());
            r->K->hpin = S->pinned + (size_t)r->slot * 16 + 4;
            r->K->own_pin = false;
            r->K->init(S->ctx, r->op, r->sub, r->diag.as<double>(), QSD_FP64, std::max(p.refine_steps, 2),
                       p.check_every, r->s, true);
        }
        QSD_CUDA(cudaMemcpyAsync(r->start.p, r->u.p, (size_t)r->sub->D * 8, cudaMemcpyDeviceToDevice, r->s));
        r->K->enqueue_start(r->start.as<double>(), p.seed);
        r->state = RState::Refine;
        if (!r->packed) r->K->enqueue_chunk(graphs);
        break;  // packed: the first chunk follows once the start has passed
    }
    case RState::Refine: {
        if (r->K->chunks > 0 && (r->K->converged(tol) || r->K->steps_done >= r->K->m)) {
            r->info.steps += r->K->steps_done;
            r->info.applies += r->K->steps_done + 1;
            r->K->enqueue_ritz(r->u.as<double>());
            r->R->enqueue(r->op, r->sub, r->diag.as<double>(), r->u.as<double>());
            r->state = RState::ResidRefine;
        } else if (r->packed) {
            r->want = r->K.get();
            return;
        } else {
            r->K->enqueue_chunk(graphs);
        }
        break;
    }
    default:
        return;
    }
    QSD_CUDA(cudaEventRecord(r->ev, r->s));
    r->inflight = true;
}

// Device set-up of an admitted request (on its own stream) and its first piece.
void start_request(qsd_server_s *S, Request *r) {
    const int64_t D = r->sub->D;
    if (!r->ev) QSD_CUDA(cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming));
    r->diag.alloc_async((size_t)D * 8, r->s);
    r->u.alloc_async((size_t)D * 8, r->s);
    r->start.alloc_async((size_t)D * 8, r->s);
    compute_diagonal_on(S->ctx, r->op, r->sub, r->diag.as<double>(), r->s);
    double *pin = S->pinned + (size_t)r->slot * 16;
    r->J.reset(new LanczosJob());
    r->J->hpin = pin;
    r->J->own_pin = false;
    r->J->init(S->ctx, r->op, r->sub, r->diag.as<double>(), r->p.precision, r->p.max_steps, r->p.check_every, r->s,
               true);
    r->R.reset(new ResidJob());
    r->R->hpin = pin + 8;
    r->R->own_pin = false;
    r->R->init(S->ctx, D, r->s, true);
    r->J->enqueue_start(r->p.v0, r->p.seed);
    r->state = RState::Main;
    if (r->packed) {
        // the chunks run on the pack stream: join one once the start has passed
        QSD_CUDA(cudaEventRecord(r->ev, r->s));
        r->inflight = true;
        return;
    }
    advance(S, r);
}

void release_request(qsd_server_s *S, Request *r) {
    // stream-ordered frees: the memory returns to the pool once the stream
    // has passed the request's last piece
    r->J.reset();
    r->K.reset();
    r->R.reset();
    r->diag.release();
    r->u.release();
    r->start.release();
}

void scheduler(qsd_server_s *S) {
    cudaSetDevice(S->ctx->device);
    std::vector<Request *> admit;
    while (true) {
        admit.clear();
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->stop && S->active.empty()) break;
            while (!S->stop && !S->queue.empty() && !S->free_slots.empty()) {
                Request *r = S->queue.front();
                if (r->cancel) {
                    S->queue.pop_front();
                    finish(S, r, QSD_ERR_CANCELLED);
                    S->cv_done.notify_all();
                    continue;
                }
                if (S->used + r->footprint > S->budget && !S->active.empty()) break;
                S->queue.pop_front();
                r->slot = S->free_slots.back();
                S->free_slots.pop_back();
                r->packed = r->sub->D <= S->pack_rows && packable(S->ctx, r->op, r->sub);
                r->s = S->streams[r->slot];
                if (r->packed) ++S->packed_requests;
                S->used += r->footprint;
                S->peak = std::max(S->peak, S->used);
                r->t_admit = Clock::now();
                r->admitted = true;
                ++S->admitted;
                S->active.push_back(r);
                admit.push_back(r);
            }
            if (S->active.empty()) {
                S->cv_work.wait_for(lk, std::chrono::milliseconds(5));
                continue;
            }
        }
        for (Request *r : admit) {
            try {
                start_request(S, r);
            } catch (const Error &e) {
                std::lock_guard<std::mutex> lk(S->mu);
                S->last_error = e.what();
                finish(S, r, e.code);
            }
        }
        bool progressed = !admit.empty();
        std::vector<Request *> done;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            for (Request *r : S->active) {
                if (r->state == RState::Done) {
                    if (!r->inflight || cudaEventQuery(r->ev) != cudaErrorNotReady) done.push_back(r);
                    continue;
                }
                if (r->in_pack >= 0 || !r->inflight) continue;  // packed: advanced with its chunk
                const cudaError_t q = cudaEventQuery(r->ev);
                if (q == cudaErrorNotReady) continue;
                r->inflight = false;
                progressed = true;
                if (q != cudaSuccess) {
                    S->last_error = cudaGetErrorString(q);
                    finish(S, r, QSD_ERR_CUDA);
                    continue;
                }
                try {
                    advance(S, r);
                } catch (const Error &e) {
                    S->last_error = e.what();
                    finish(S, r, e.code);
                }
            }
        }
        // packed chunks: once a pack's chunk has passed, its members' results
        // move to their pinned words and each member advances (its next
        // piece on its own stream, or a wish for the next chunk); then every
        // pack takes all its members that wait for a chunk.  A member's own
        // stream is idle while it waits, and its next piece follows only once
        // the chunk has passed, so the host orders the two streams.  Only
        // this thread touches the members.
        for (int k = 0; k < 3; ++k) {
            if (S->pack_inflight[k]) {
                const cudaError_t q = cudaEventQuery(S->pack_ev[k]);
                if (q == cudaErrorNotReady) continue;
                if (q == cudaSuccess) S->pack[k].finish_chunk();
                std::lock_guard<std::mutex> lk(S->mu);
                for (Request *r : S->pack_members[k]) {
                    r->in_pack = -1;
                    r->inflight = false;
                    if (q != cudaSuccess) {
                        S->last_error = cudaGetErrorString(q);
                        finish(S, r, QSD_ERR_CUDA);
                        continue;
                    }
                    try {
                        advance(S, r);
                    } catch (const Error &e) {
                        S->last_error = e.what();
                        finish(S, r, e.code);
                    }
                }
                S->pack_members[k].clear();
                S->pack_inflight[k] = false;
                progressed = true;
            }
            std::vector<Request *> members;
            std::vector<LanczosJob *> jobs;
            {
                std::lock_guard<std::mutex> lk(S->mu);
                for (Request *r : S->active)
                    if (r->want && r->state != RState::Done && r->want->prec == k) {
                        members.push_back(r);
                        jobs.push_back(r->want);
                    }
            }
            if (jobs.empty()) continue;
            std::string err;
            int code = QSD_OK;
            try {
                if (!S->pack[k].host) S->pack[k].init(S->ctx, S->max_active, S->pack_stream);
                S->pack[k].enqueue_chunk(jobs);
                QSD_CUDA(cudaEventRecord(S->pack_ev[k], S->pack_stream));
            } catch (const Error &e) {
                err = e.what();
                code = e.code;
            }
            std::lock_guard<std::mutex> lk(S->mu);
            if (code == QSD_OK) {
                S->pack_inflight[k] = true;
                S->pack_members[k] = members;
                ++S->packed_chunks;
                for (Request *r : members) {
                    r->want = nullptr;
                    r->in_pack = k;
                }
            } else {
                S->last_error = err;
                for (Request *r : members) {
                    r->want = nullptr;
                    finish(S, r, code);
                }
            }
            progressed = true;
        }
        for (Request *r : done) {
            release_request(S, r);
            std::lock_guard<std::mutex> lk(S->mu);
            S->active.erase(std::find(S->active.begin(), S->active.end(), r));
            S->free_slots.push_back(r->slot);
            S->used -= r->footprint;
            S->cv_done.notify_all();
            progressed = true;
        }
        if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

}  // namespace

}  // namespace qsd

using namespace qsd;

extern "C" {

int qsd_server_create(qsd_ctx ctx, size_t budget_bytes, int32_t max_active, qsd_server *out) {
    if (!ctx || !out || max_active < 1 || max_active > 256) return QSD_ERR_INVALID_ARG;
    auto *S = new qsd_server_s();
    try {
        S->ctx = ctx;
        S->budget = budget_bytes;
        S->max_active = max_active;
        S->t0 = Clock::now();
        QSD_CUDA(cudaSetDevice(ctx->device));
        // requests may come from other contexts with any key width: the hash
        // tables of every width, allocated once before any request runs
        ensure_nibble_tables(ctx, kMaxWordsDyn);
        QSD_CUDA(cudaMallocHost(&S->pinned, (size_t)max_active * 16 * sizeof(double)));
        // keep memory freed by retired requests in the stream-ordered pool
        cudaMemPool_t pool;
        QSD_CUDA(cudaDeviceGetDefaultMemPool(&pool, ctx->device));
        uint64_t keep = std::max<uint64_t>(budget_bytes, 1ull << 30);
        QSD_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
        for (int i = 0; i < max_active; ++i) {
            cudaStream_t s;
            QSD_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
            S->streams.push_back(s);
            S->free_slots.push_back(max_active - 1 - i);
        }
        QSD_CUDA(cudaStreamCreateWithFlags(&S->pack_stream, cudaStreamNonBlocking));
        for (auto &e : S->pack_ev) QSD_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        S->th = std::thread(scheduler, S);
    } catch (const Error &e) {
        ctx->last_error = e.what();
        for (auto s : S->streams) cudaStreamDestroy(s);
        if (S->pack_stream) cudaStreamDestroy(S->pack_stream);
        for (auto e2 : S->pack_ev)
            if (e2) cudaEventDestroy(e2);
        if (S->pinned) cudaFreeHost(S->pinned);
        delete S;
        return e.code;
    }
    *out = S;
    return QSD_OK;
}

int qsd_server_submit(qsd_server S, qsd_op op, qsd_sub sub, const qsd_lanczos_params *p, uint64_t *ticket) {
    if (!S || !op || !sub || !p || !ticket) return QSD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    if (op->n_qubits != sub->n_qubits || sub->D == 0 || p->max_steps < 1 || p->check_every < 1 ||
        p->precision < QSD_FP64 || p->precision > QSD_FP32_DOT2) {
        S->last_error = "qsd_server_submit: bad request";
        return QSD_ERR_INVALID_ARG;
    }
    if (!op->info.is_real) { S->last_error = "qsd_server_submit: complex operator"; return QSD_ERR_COMPLEX_UNSUPPORTED; }
    if (!op->info.is_hermitian) { S->last_error = "qsd_server_submit: operator is not Hermitian"; return QSD_ERR_NOT_HERMITIAN; }
    if (S->stop) return QSD_ERR_CANCELLED;
    auto *r = new Request();
    r->ticket = S->next_ticket++;
    r->op = op;
    r->sub = sub;
    r->p = *p;
    r->footprint = request_footprint(sub->D, *p, S->ctx->num_sms);
    r->t_submit = Clock::now();
    S->all[r->ticket] = r;
    S->queue.push_back(r);
    *ticket = r->ticket;
    S->cv_work.notify_one();
    return QSD_OK;
}

static int fill_result(qsd_server S, Request *r, double *energy, qsd_lanczos_info *info, double *times) {
    if (energy) *energy = r->energy;
    if (info) *info = r->info;
    if (times) {
        times[0] = secs(S->t0, r->t_submit);
        times[1] = r->admitted ? secs(S->t0, r->t_admit) : -1.0;
        times[2] = secs(S->t0, r->t_done);
    }
    return r->status;
}

int qsd_server_poll(qsd_server S, uint64_t ticket, double *energy, qsd_lanczos_info *info, double *times) {
    if (!S) return QSD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return QSD_ERR_INVALID_ARG;
    Request *r = it->second;
    if (r->state != RState::Done) return QSD_PENDING;
    // done, but the slot may still be draining: results are final once Done
    return fill_result(S, r, energy, info, times);
}

int qsd_server_wait(qsd_server S, uint64_t ticket, double timeout_s, double *energy, qsd_lanczos_info *info,
                    double *times) {
    if (!S) return QSD_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return QSD_ERR_INVALID_ARG;
    Request *r = it->second;
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                             std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 1e9));
    while (r->state != RState::Done) {
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && r->state != RState::Done)
            return QSD_ERR_TIMEOUT;
    }
    return fill_result(S, r, energy, info, times);
}

int qsd_server_cancel(qsd_server S, uint64_t ticket) {
    if (!S) return QSD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return QSD_ERR_INVALID_ARG;
    it->second->cancel = true;
    S->cv_work.notify_one();
    return QSD_OK;
}

int qsd_server_release(qsd_server S, uint64_t ticket) {
    if (!S) return QSD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return QSD_ERR_INVALID_ARG;
    Request *r = it->second;
    if (r->state != RState::Done || std::find(S->active.begin(), S->active.end(), r) != S->active.end())
        return QSD_PENDING;
    S->all.erase(it);
    if (r->ev) cudaEventDestroy(r->ev);
    delete r;
    return QSD_OK;
}

int qsd_server_get_stats(qsd_server S, qsd_server_stats *st) {
    if (!S || !st) return QSD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    st->queued = (int64_t)S->queue.size();
    st->active = (int64_t)S->active.size();
    st->completed = S->completed;
    st->failed = S->failed;
    st->admitted = S->admitted;
    st->bytes_in_use = S->used;
    st->peak_bytes = S->peak;
    st->budget_bytes = S->budget;
    st->packed_requests = S->packed_requests;
    st->packed_chunks = S->packed_chunks;
    return QSD_OK;
}

int qsd_server_set_pack_rows(qsd_server S, int64_t rows) {
    if (!S || rows < 0) return QSD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    S->pack_rows = rows;
    return QSD_OK;
}

const char *qsd_server_last_error(qsd_server S) { return S ? S->last_error.c_str() : ""; }

int qsd_server_destroy(qsd_server S) {
    if (!S) return QSD_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        for (auto *r : S->queue) {
            finish(S, r, QSD_ERR_CANCELLED);
        }
        S->queue.clear();
        for (auto *r : S->active) r->cancel = true;
        S->cv_work.notify_all();
    }
    if (S->th.joinable()) S->th.join();
    for (auto &kv : S->all) {
        if (kv.second->ev) cudaEventDestroy(kv.second->ev);
        delete kv.second;
    }
    for (auto s : S->streams) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
    if (S->pack_stream) {
        // the packs' device blocks are stream-ordered on the pack stream:
        // free them while it exists
        for (auto &pk : S->pack) pk.release();
        cudaStreamSynchronize(S->pack_stream);
        cudaStreamDestroy(S->pack_stream);
    }
    for (auto e : S->pack_ev)
        if (e) cudaEventDestroy(e);
    if (S->pinned) cudaFreeHost(S->pinned);
    delete S;
    return QSD_OK;
}

}  // extern "C"
