// Lanczos state shared by the synchronous solver and the request server.
#pragma once

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

// Device block and pinned staging of a pack's descriptors (grown on demand;
// reused once the stream has passed the previous chunk that used them).
struct PackBuffers {
    DevBuf dev;
    unsigned char *host = nullptr;
    size_t cap = 0;
    PackBuffers() = default;
    PackBuffers(const PackBuffers &) = delete;
    PackBuffers &operator=(const PackBuffers &) = delete;
    ~PackBuffers();
    void reserve(size_t bytes, cudaStream_t s);
    void release();  // before the stream of `dev` is destroyed
};

// One chunk of steps for every job of a pack with packed launches on stream
// s: the product of all jobs (group scan, one launch per key width) and each
// Lanczos kernel once for all jobs.  Jobs share the basis type and product
// precision and have W <= 4; each advances min(check_every, m - steps_done)
// steps and its tridiagonal results reach its hpin as after enqueue_chunk.
void enqueue_packed_chunk(qsd_ctx ctx, const std::vector<LanczosJob *> &jobs, cudaStream_t s, PackBuffers &pb);

// FP64 Rayleigh quotient and residual of a vector, enqueued on a stream.
struct ResidJob {
    qsd_ctx ctx = nullptr;
    int64_t D = 0;
    int B = 1;
    cudaStream_t s = nullptr;
    DevBuf hu, r, part;
    double *hpin = nullptr;  // [u^T H u, u^T u, |H u - theta u|]
    bool own_pin = true;     // false: hpin lent by the caller (set before init)

    ResidJob() = default;
    ResidJob(const ResidJob &) = delete;
    ResidJob &operator=(const ResidJob &) = delete;
    ~ResidJob();
    void init(qsd_ctx c, int64_t Dn, cudaStream_t st, bool stream_ordered);
    void enqueue(qsd_op op, qsd_sub sub, const double *diag, const double *u);
    void read(double &theta, double &resid_rel) const;
};

}  // namespace qsd
