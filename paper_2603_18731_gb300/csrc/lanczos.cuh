// Lanczos state shared by the synchronous solver and the request server.
#pragma once

#include <map>
#include <vector>

#include "apply_kernel.cuh"

namespace qsd {

constexpr int kLanczosThreads = 256;
constexpr int kLanczosMaxSteps = 700;  // the tridiagonal CTA keeps 8 m doubles in shared memory

// Row blocks of the dot passes for D rows.
int dot_blocks(int64_t D, int num_sms);

// One Lanczos run on one stream: Krylov basis, tridiagonal coefficients and a
// device step counter.  enqueue_* only enqueue work; results of a chunk are in
// pinned host memory once the stream has passed it.
struct LanczosJob {
    qsd_ctx ctx = nullptr;
    qsd_op op = nullptr;
    qsd_sub sub = nullptr;
    const double *diag = nullptr;
    int prec = QSD_FP64;  // product precision
    bool fp32 = false;    // Krylov basis storage
    int64_t D = 0;
    int m = 0, B = 1, nbD = 1, check_every = 10;
    int steps_done = 0, chunks = 0;
    cudaStream_t s = nullptr;
    DevBuf V, vcur, hv, w, h, part, alpha, beta, tri, jdev;
    double *hpin = nullptr;  // [theta, estimate, beta_m, m]
    bool own_pin = true;     // false: hpin lent by the caller (set before init)
    cudaMemPool_t pool = nullptr;  // set before init: the buffers come from it (stream-ordered)
    cudaGraphExec_t graph = nullptr;

    LanczosJob() = default;
    LanczosJob(const LanczosJob &) = delete;
    LanczosJob &operator=(const LanczosJob &) = delete;
    ~LanczosJob();
    void init(qsd_ctx c, qsd_op o, qsd_sub su, const double *d, int product_precision, int steps, int check,
              cudaStream_t st, bool stream_ordered);
    static size_t footprint(int64_t D, int steps, bool fp32, int num_sms);
    void enqueue_start(const double *start, uint64_t seed);
    void enqueue_chunk(bool use_graph);
    void enqueue_ritz(double *u);
    void read(double &theta, double &est, double &beta_last, int &nvec) const;
    bool converged(double tol) const;
};

// A pack: Lanczos jobs of one product precision advanced together, one
// chunk of steps at a time, by CUDA-graph replays whose launches serve every
// member (lanczos.cu).  The device block and its pinned staging have fixed
// offsets for `cap` members, so a graph captured for one chunk shape (the
// product classes present and the number of steps) replays for any
// membership: a chunk costs the copy of the changed descriptors and one graph
// launch.  Members' results (theta, estimate, beta_m, m) reach their hpin in
// finish_chunk, once the stream has passed the chunk.
struct Pack {
    qsd_ctx ctx = nullptr;
    int cap = 0;
    cudaStream_t s = nullptr;
    DevBuf dev;
    unsigned char *host = nullptr;  // pinned staging (same layout)
    size_t bytes = 0;
    std::map<uint32_t, cudaGraphExec_t> graphs;  // by (classes present, steps)
    std::vector<LanczosJob *> members;           // of the chunk in flight
    int64_t chunks = 0, graph_builds = 0;

    Pack() = default;
    Pack(const Pack &) = delete;
    Pack &operator=(const Pack &) = delete;
    ~Pack();
    void init(qsd_ctx c, int capacity, cudaStream_t st);
    void release();  // before `s` is destroyed; waits for s
    // One chunk for jobs (at most cap; shared basis type and product
    // precision; each packable): min(check_every, m - steps_done) steps each.
    void enqueue_chunk(const std::vector<LanczosJob *> &jobs);
    // After the stream has passed the chunk: the members' results to their hpin.
    void finish_chunk();
};

// Whether the product of (op, sub) can run in a pack: the factored product
// (W <= 2) or a group scan of at most kPackMaxScanGroups groups (W <= 4; one
// or eight lanes per row, as the single product would choose).
constexpr int64_t kPackMaxScanGroups = 4096;
bool packable(qsd_ctx ctx, qsd_op op, qsd_sub sub);

// FP64 Rayleigh quotient and residual of a vector, enqueued on a stream.
struct ResidJob {
    qsd_ctx ctx = nullptr;
    int64_t D = 0;
    int B = 1;
    cudaStream_t s = nullptr;
    DevBuf hu, r, part;
    double *hpin = nullptr;  // [u^T H u, u^T u, |H u - theta u|]
    bool own_pin = true;     // false: hpin lent by the caller (set before init)
    cudaMemPool_t pool = nullptr;  // set before init: the buffers come from it (stream-ordered)

    ResidJob() = default;
    ResidJob(const ResidJob &) = delete;
    ResidJob &operator=(const ResidJob &) = delete;
    ~ResidJob();
    void init(qsd_ctx c, int64_t Dn, cudaStream_t st, bool stream_ordered);
    void enqueue(qsd_op op, qsd_sub sub, const double *diag, const double *u);
    void read(double &theta, double &resid_rel) const;
};

}  // namespace qsd
