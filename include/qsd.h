/*
 * qsd.h -- C ABI of the GB300 subspace Hamiltonian library.
 *
 * The library evaluates the matrix-free product y = H_S x of a Hamiltonian
 * written in the extended alphabet [Z, 0, 1, X, Y, -, +] over a subspace S
 * of sampled bit-strings, and finds the ground state of H_S with a Lanczos
 * solver on the device (arXiv 2603.18731, "A generalized framework for
 * quantum subspace diagonalization": Methods "Qubit Hamiltonians",
 * "Subspace data structure" and "Matrix evaluation").
 *
 * Conventions that hold for every call:
 *  - Bit-strings over n qubits are W = ceil(n/64) little-endian uint64 words;
 *    qubit q is bit q%64 of word q/64.  Arrays of bit-strings are row-major
 *    [count][W].  There is no upper limit on n other than memory.
 *  - Letters are coded [Z, 0, 1, X, Y, -, +] -> 0..6 as in the paper
 *    (Methods, "Qubit Hamiltonians"): 0 = |0><0|, 1 = |1><1|,
 *    + = |1><0| (raising), - = |0><1| (lowering).
 *  - Subspace index of a bit-string = its rank in ascending integer order
 *    (word W-1 most significant) after duplicates are dropped (Methods,
 *    "Lower / upper triangle evaluation" sorts the subspace by integer value).
 *  - Every call returns a status code (QSD_OK = 0).  On error the context's
 *    message is set (qsd_last_error) and no output is written unless stated.
 *  - Input arrays are read during the call and stay owned by the caller.
 *    Handles are owned by the library until freed.
 *  - Device pointers must be device memory of the context's device.  Device
 *    work is enqueued on the context's stream; calls that return a host
 *    value (dimensions, energies) synchronise that stream.
 *  - A handle must not be used from two threads at once; distinct contexts
 *    may be used concurrently.
 */
#ifndef QSD_H
#define QSD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------- status codes */
#define QSD_OK                      0
#define QSD_ERR_INVALID_ARG         1  /* bad pointer, size, enum or handle */
#define QSD_ERR_QUBIT_RANGE         2  /* qubit index < 0 or >= n, or letter code > 6 */
#define QSD_ERR_REPEATED_INDEX      3  /* a qubit appears twice in one word */
#define QSD_ERR_NOT_HERMITIAN       4  /* operator is not Hermitian (eigensolvers only) */
#define QSD_ERR_COMPLEX_UNSUPPORTED 5  /* operator has complex matrix elements */
#define QSD_ERR_OOM                 6  /* device or host allocation failed */
#define QSD_ERR_NOT_CONVERGED       7  /* eigensolver hit max_steps; best estimate returned */
#define QSD_ERR_TIMEOUT             8  /* a bounded device or host wait ran out */
#define QSD_ERR_CUDA                9  /* a CUDA runtime call failed */
#define QSD_ERR_CAPACITY           10  /* subspace larger than 2^32 - 2 rows */
#define QSD_ERR_CANCELLED          11  /* request cancelled before completion */
#define QSD_PENDING                12  /* server request still running */
#define QSD_ERR_INTERNAL           13  /* a device-side consistency check failed */

/* ------------------------------------------------------------- precision */
#define QSD_FP64        0  /* x, y stored as double; FP64 accumulation */
#define QSD_FP32_MIXED  1  /* x, y stored as float; each row accumulated in FP64 */
#define QSD_FP32_DOT2   2  /* x, y stored as float; each row accumulated in FP32 with
                              error-free transformations (TwoProduct, TwoSum: the
                              "Dot2" scheme of Ogita, Rump and Oishi, 2005), as
                              accurate as accumulating in twice the FP32 precision,
                              with no FP64 arithmetic (GB300 issues FP64 at 1/64 of
                              the FP32 rate) */

typedef struct qsd_ctx_s *qsd_ctx;
typedef struct qsd_op_s *qsd_op;
typedef struct qsd_sub_s *qsd_sub;

/* ------------------------------------------------------------- contexts */
/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * to enqueue on (e.g. a PyTorch stream), or NULL for a stream owned by the
 * context.  *out receives the handle.  The context owns a stream-ordered
 * memory pool for the eigensolver's workspace: blocks freed at the end of a
 * solve stay mapped, up to 1/16 of the device's memory, so that the next
 * solve on the context allocates without mapping memory again. */
int qsd_create(int device, void *cuda_stream, qsd_ctx *out);

/* Destroy a context (and its pool).  Operators and subspaces made on it must
 * be freed first. */
int qsd_destroy(qsd_ctx ctx);

/* Message of the last failed call on `ctx` (or of the calling thread's last
 * failed qsd_create when ctx is NULL).  Valid until the next call. */
const char *qsd_last_error(qsd_ctx ctx);

/* --------------------------------------------------------------- operators */
typedef struct {
    int32_t n_qubits;
    int32_t n_words;          /* W */
    int64_t n_terms_in;       /* terms passed to qsd_load_operator */
    int64_t n_terms;          /* off-diagonal terms after combining equal words */
    int64_t n_diag_terms;     /* diagonal terms (no flipped qubit) after combining */
    int64_t n_groups;         /* off-diagonal groups (distinct flip sets) */
    int64_t n_ladder_groups;  /* groups that use the ladder-integer table */
    int64_t n_excitation_groups; /* ladder groups in the excitation index (0: none) */
    int32_t n_excitation_shapes; /* distinct occupied/empty shapes of their terms */
    int32_t excitation_rank_index; /* 1: the index finds a flip mask's group by its
                                      rank (one load); 0: through a hash table */
    int64_t max_group_terms;
    int32_t is_real;          /* every matrix element is real */
    int32_t is_hermitian;     /* term set closed under adjoint (rel. 1e-14) */
    double identity_coef;     /* real part of the constant (empty-word) term */
    int64_t n_linear_ranges;  /* ladder ranges tabulated as a constant plus one
                                 coefficient per occupied qubit (single
                                 excitations of a two-body fermionic operator;
                                 used by the factored product) */
} qsd_op_info;

/* Load H = sum_t c_t W_t (Methods, "Qubit Hamiltonians": a term is a
 * coefficient, the sorted qubit indices of its non-identity factors and
 * their letters).  Term t owns factors term_ptr[t] .. term_ptr[t+1]-1 of
 * op_qubit (int32) and op_code (uint8, 0..6).  coef_im may be NULL (real
 * coefficients).  An empty word is the identity and adds its coefficient to
 * the diagonal.  Terms with a zero coefficient are dropped.  All arrays are
 * host memory.
 *
 * The call converts every word to masks over the row bits (flip F, test P
 * and V, sign Z), combines equal words, and groups the off-diagonal terms on
 * the device by their off-diagonal structure F ordered by (popcount F, F)
 * (Methods, "Qubit Hamiltonians", properties 1-3 and Fig. 3a); inside a group
 * terms are ordered by their ladder integer, and groups whose flipped qubits
 * all carry ladder letters get the int_ptrs table of the ladder integer
 * (Methods, "Fermionic Hamiltonians", Fig. 3b).
 * Errors: QSD_ERR_QUBIT_RANGE, QSD_ERR_REPEATED_INDEX, QSD_ERR_INVALID_ARG. */
int qsd_load_operator(qsd_ctx ctx, int32_t n_qubits, int64_t n_terms,
                      const int64_t *term_ptr, const int32_t *op_qubit,
                      const uint8_t *op_code, const double *coef_re,
                      const double *coef_im, qsd_op *out);

int qsd_op_get_info(qsd_op op, qsd_op_info *info);

/* Group flip sets in the library's group order, row-major [n_groups][W]
 * (host output). */
int qsd_op_groups(qsd_op op, uint64_t *groups_out);

int qsd_free_op(qsd_op op);

/* --------------------------------------------------------------- subspaces */
/* Build the subspace from n_in bit-strings (row-major [n_in][W], host memory
 * when words_on_device == 0, else device memory), any order, duplicates
 * allowed (Methods, "Subspace data structure").  The strings are sorted by
 * integer value on the device, duplicates dropped, and an open-addressing
 * hash table (load factor <= 1/4, buckets of eight 8-bit tags with a 32-bit
 * row index per slot, bucket and tag taken from one GF(2)-linear hash of the
 * string) is built for lookups; for n <= 256 the rows are also listed in
 * bucket order (4 + 8 W bytes per row) for the hash-order product, and an
 * occupancy filter over the hash (128 bits per bucket, 16 bytes per bucket)
 * lets the filter/verify product reject absent columns with one 4-byte load
 * (the paper's occupancy bit-set).  *dim_out receives D.  Synchronises.
 * Errors: QSD_ERR_CAPACITY when D would exceed 2^32 - 2. */
int qsd_build_subspace(qsd_ctx ctx, int32_t n_qubits, int64_t n_in,
                       const uint64_t *words, int words_on_device,
                       qsd_sub *out, int64_t *dim_out);

/* Dimension, qubit count and hash capacity (slots) of a subspace. */
int qsd_subspace_info(qsd_sub sub, int64_t *dim, int32_t *n_qubits, int64_t *capacity);

/* Sector-factored index of a subspace (Results: chemistry subspaces are the
 * products of alpha and beta strings).  The build splits every string at
 * qubit split = n / 2 (n <= 128) into a low half a and a high half b; when
 * S is exactly A x B for its distinct halves A and B (D = |A| |B|), it keeps
 * A and B sorted and, per string of each, its neighbours in the same list by
 * excitation type (up to two set bits cleared and two clear bits set), so
 * that row = ib |A| + ia and the factored product needs no lookup.  Outputs
 * (any may be NULL): *is_product 1 or 0, *split, *n_a = |A|, *n_b = |B|,
 * *neighbours = entries of both neighbour lists (0 when not a product).
 * A product subspace is not indexed when a string has more than 4096
 * neighbours of one type or the lists exceed 64 (|A| + |B|) + 2^20 entries. */
int qsd_subspace_factored(qsd_sub sub, int32_t *is_product, int32_t *split, int64_t *n_a, int64_t *n_b,
                          int64_t *neighbours);

/* Copy the sorted bit-strings, row-major [D][W], to `out` (device memory when
 * out_on_device != 0, else host memory; host copies synchronise). */
int qsd_subspace_keys(qsd_ctx ctx, qsd_sub sub, uint64_t *out, int out_on_device);

/* Index of each of n query strings (device, row-major [n][W]) in the
 * subspace, or -1 when absent; idx_out is device int64 [n]. */
int qsd_subspace_index(qsd_ctx ctx, qsd_sub sub, int64_t n,
                       const uint64_t *keys, int64_t *idx_out);

int qsd_free_sub(qsd_sub sub);

/* ------------------------------------------------------------------ CSR */
/* Explicit CSR form of H_S by the two-pass build (Methods, "Matrix
 * evaluation"): pass 1 counts each row's entries, pass 2 evaluates them again
 * and writes them.  By default a row evaluates only its lower-triangle groups,
 * those whose most significant flipped qubit is set in the row (Supplementary,
 * "Lower / upper triangle evaluation" and "Most-significant off-diagonal
 * bit"), and each lower entry h at (r, c) also fills (c, r) with conj(h); this
 * needs a Hermitian operator.  QSD_CSR_FULL evaluates every group of every row
 * instead (any real operator).
 *
 * Structure: row r holds its diagonal (always, even when zero) and every
 * column c != r of S such that at least one term maps column c to row r with
 * its projector tests passed; values are stored even when terms cancel.
 * Columns ascend within a row.  Integer-exact; values are FP64 sums.
 *
 * Call once with indptr = indices = data_re = data_im = NULL: *nnz_out gets
 * the number of entries and the pass-1 counts are kept in the context.  Then
 * call with device arrays indptr int64 [D+1], indices int32 or int64
 * (index_bits 32 | 64) [nnz], data_re double [nnz] and data_im double [nnz]
 * (may be NULL for a real operator; required for a complex one, whose
 * operator must be Hermitian).  The arrays are caller-owned device memory; the
 * call is synchronous on the context's stream.  Errors: QSD_ERR_NOT_HERMITIAN
 * (triangle evaluation of a non-Hermitian operator), QSD_ERR_CAPACITY (nnz
 * >= 2^32 - 1), QSD_ERR_OOM (device temporaries: about 20 bytes per entry). */
#define QSD_CSR_FULL 1
int qsd_to_csr(qsd_ctx ctx, qsd_op op, qsd_sub sub, int32_t flags, int64_t *nnz_out,
               int64_t *indptr, void *indices, int32_t index_bits,
               double *data_re, double *data_im);

/* ---------------------------------------------------------------- LOBPCG */
/* The k lowest eigenpairs of the real symmetric H_S by LOBPCG with a shifted
 * Jacobi (diagonal) preconditioner -- the eigensolver the paper uses for its
 * chemistry results (Results: PRIMME's LOBPCG from a vector spiked at the
 * lowest diagonal, diagonal preconditioner shifted by the current eigenvalue
 * estimate).  Directions W = R / max(|d - theta|, 1e-8 max|d|) column by
 * column; the basis [X, W, P] is kept orthonormal; FP64 block products (one
 * lookup per group serves the k columns); Rayleigh-Ritz with the small
 * eigenproblem solved on the host; reproducible (fixed reduction orders).
 * Requires a real Hermitian operator, 1 <= k <= 16 and dim >= 3k.  evals:
 * host double [k] ascending; evecs: device double [dim][k] (row-major,
 * orthonormal columns) or NULL.  Returns QSD_OK when every pair meets tol,
 * else QSD_ERR_NOT_CONVERGED with the last estimates. */
typedef struct {
    int32_t k;             /* eigenpairs wanted (block width), 1..16 */
    int32_t max_iters;     /* iteration limit */
    double tol;            /* max over pairs of |H x - theta x| / |theta|, unit x */
    uint64_t seed;         /* random entries U(-1,1) from SplitMix64(seed xor index) */
    const double *x0;      /* optional device [dim][k] start block (NULL: see start) */
    int32_t precondition;  /* 1: shifted Jacobi; 0: none */
    int32_t start;         /* 0: unit spikes at the k lowest diagonal entries plus
                              1e-3 random entries (the paper's start); 1: random */
} qsd_lobpcg_params;
typedef struct {
    int32_t iters, converged;
    double max_residual;
    int32_t status, reserved;
} qsd_lobpcg_info;
/* k 1, 500 iterations, tol 1e-9, seed 0, precondition 1, start 0 */
void qsd_lobpcg_default_params(qsd_lobpcg_params *p);
int qsd_lobpcg(qsd_ctx ctx, qsd_op op, qsd_sub sub, const qsd_lobpcg_params *p, double *evals,
               double *evecs, qsd_lobpcg_info *info);

/* -------------------------------------------------------------- trimming */
/* Operator group trimming (Results, chemistry: groups whose matrix elements
 * are small against the smallest diagonal energy splitting of the subspace
 * are removed before matrix evaluation).  A group's elements are bounded by
 * m_g = sum of |phi_t| over its terms (equal words combined); the splitting is
 * Delta = min over rows of sub with d_r > d_min of (d_r - d_min).  Groups with
 * m_g / Delta < tol are removed; diagonal words and the identity are kept
 * (everything is kept when all diagonal entries of sub are equal).  *out gets
 * a new operator loaded from the kept input words (caller frees it); info
 * (may be NULL) reports the counts, d_min and Delta. */
typedef struct {
    int64_t groups_in, groups_kept;
    int64_t terms_in, terms_kept;  /* input words */
    double d_min, splitting;
} qsd_trim_info;
int qsd_trim_operator(qsd_ctx ctx, qsd_op op, qsd_sub sub, double tol, qsd_op *out, qsd_trim_info *info);

/* ------------------------------------------------------------------ RAMPS */
/* Subspace refinement RAMPS (Supplementary, "Recursive algorithm for a
 * minimal perturbative subspace", Algorithm S1; expansion Eq. S2), run level
 * by level on the device with every (row, group) pair of a level in parallel
 * (the paper's implementation is serial).  From the rows of `start` with
 * prefactor 1/E, each level adds every column b_k reached from a level row
 * b_j through an off-diagonal group with |amp| > tau, amp = pre_j
 * |H_jk|^2 / (E - H_kk), H_kk the diagonal of b_k; the added rows carry
 * prefactor amp / (E - H_kk) into the next level.  Rows already in the
 * output are not revisited; a column reached from several rows of a level
 * keeps its largest |amp|; a column with H_kk = E is added and not expanded.
 * restrict_to (may be NULL): only its rows may be added (the restricted
 * variant, Supplementary).  max_levels ends the recursion (the paper's
 * maximum number of recursions); max_rows > 0 stops after the level that
 * reaches that many output rows.  *out receives a new subspace handle with
 * the start rows and every added row (caller frees it).  Elements may be
 * complex (|H_jk|^2 uses the modulus).  Errors: QSD_ERR_INVALID_ARG (E == 0
 * or not finite, tau < 0, n > 256 qubits), QSD_ERR_CAPACITY (2^32 candidate
 * columns in one level). */
typedef struct {
    int32_t levels;            /* levels run */
    int32_t stopped_by_limit;  /* 1: max_levels ended a recursion that had rows left */
    int32_t truncated;         /* 1: max_rows was reached */
    int32_t reserved;
    int64_t rows_out;          /* rows of *out */
    int64_t candidates;        /* columns above tau over all levels, before merging */
    int64_t level_rows[64];    /* rows added by each of the first 64 levels */
} qsd_ramps_info;
int qsd_ramps(qsd_ctx ctx, qsd_op op, qsd_sub start, double E, double tau, int32_t max_levels,
              qsd_sub restrict_to, int64_t max_rows, qsd_sub *out, qsd_ramps_info *info);

/* ------------------------------------------------------------------ tuning */
#define QSD_TUNE_APPLY_PATH     1  /* 0 auto; 1 per-row scan of all groups; 2 excitation
                                      index (ladder groups enumerated from each row's
                                      occupation; ignored when the operator has none);
                                      3 half evaluation (below; a plain scan where it
                                      does not apply); 4 sector-factored enumeration
                                      where it applies (QSD_PATH_FACTORED), else as 0;
                                      5 filter/verify scan where it applies
                                      (QSD_PATH_FILTER_VERIFY), else as 0.
                                      Auto takes the factored path whenever it applies. */
#define QSD_TUNE_LANES_PER_ROW  2  /* per-row scan: 0 auto, 1 or 8 lanes per row */
#define QSD_TUNE_AUTOTUNE       3  /* 1 (default): the first product of each (operator,
                                      subspace, precision, block width) on a context times
                                      the candidate paths on the stream and caches the
                                      fastest; 0: heuristic choice */
#define QSD_TUNE_HALF_EVALUATION 4 /* 1: the autotuner may also pick the half evaluation;
                                      0 (default): it does not.  Half evaluation (real
                                      Hermitian operator, QSD_FP64, n <= 256): a row
                                      evaluates only its lower-triangle groups, those whose
                                      most significant flipped qubit is set in the row
                                      (Supplementary, "Lower / upper triangle evaluation"),
                                      and each element h at (r, c) adds h x[c] to y[r] and
                                      h x[r] to y[c] by FP64 atomic adds: half the element
                                      evaluations and lookups, but a summation order (so
                                      the last bits of y) that varies from run to run. */
#define QSD_TUNE_ROW_ORDER      5  /* lane-per-row scans (n <= 256): 0 auto (the autotuner
                                      also times hash order), 1 index order, 2 hash order.
                                      Hash order takes the rows in the order of the
                                      subspace's hash buckets instead of by index: the key
                                      hash is GF(2)-linear, so the column r xor F of every
                                      row of a warp falls in a few neighbouring buckets and
                                      each group's 32 lookups share cache lines.  Per row
                                      the result is bitwise that of index order (same
                                      groups, same order).  No counterpart in the paper. */
#define QSD_TUNE_LINEAR_HALVES  6  /* sector-factored product: 1 (default) per (operator,
                                      subspace) pair, tables of the linear ranges' sums
                                      over each half string (built on the first product
                                      outside a stream capture, freed with either handle);
                                      a single-excitation element then costs two loads
                                      instead of one per occupied qubit.  Bitwise the
                                      same products either way.  0: no tables. */

/* Set a product-path choice on a context (later products of this context
 * use it).  Results are identical up to summation order for every choice; a
 * given choice other than the half evaluation is bitwise reproducible. */
int qsd_set_tuning(qsd_ctx ctx, int32_t knob, int64_t value);

/* The product path that the next qsd_apply_H of (op, sub, precision) with k
 * columns takes for its first column block (16, 4 or 1 columns wide), without
 * timing anything: QSD_PATH_SCAN_1 (per-row group scan, one lane per row),
 * QSD_PATH_SCAN_8 (eight lanes per row), QSD_PATH_EXCITATION, or the half
 * evaluation with one or eight lanes per row (QSD_PATH_HALF_1, _8), or a
 * one-lane path in hash order (QSD_PATH_SCAN_HASH, _HALF_HASH).  After a
 * tuned product it is the cached measurement, else the forced choice or the
 * heuristic.  No counterpart in the paper (its kernel has one launch shape). */
#define QSD_PATH_SCAN_1     0
#define QSD_PATH_SCAN_8     1
#define QSD_PATH_EXCITATION 2
#define QSD_PATH_HALF_1     3
#define QSD_PATH_HALF_8     4
#define QSD_PATH_SCAN_HASH  5  /* QSD_PATH_SCAN_1 with the rows in hash order */
#define QSD_PATH_HALF_HASH  6  /* QSD_PATH_HALF_1 with the rows in hash order */
#define QSD_PATH_FACTORED   7  /* product subspace S = A x B of its halves at qubit n/2
                                  (see qsd_subspace_factored) and an operator whose
                                  ladder groups have a rank index (qsd_op_info
                                  excitation_rank_index, n <= 128): each row enumerates
                                  only the columns in S -- products of its halves'
                                  neighbours in A and B by excitation type -- and
                                  computes their index as ib' |A| + ia' (no lookup);
                                  bulk group rejection, named as future work in the
                                  paper's Discussion */
#define QSD_PATH_FILTER_VERIFY 8  /* single-column products of operators whose groups all
                                  test and sign at most 5 qubits (spin models; at most
                                  1024 groups and 2048 tabulated elements), rows in
                                  hash order (n <= 256): a filter pass over the
                                  groups, with group records and elements staged in
                                  shared memory, loads each row's bucket and queues
                                  only tag matches and overflowing buckets; a verify
                                  pass resolves 32 queued lookups at a time, one per
                                  lane, and returns the found elements to their rows
                                  in group order: bitwise QSD_PATH_SCAN_HASH */
int qsd_product_path(qsd_ctx ctx, qsd_op op, qsd_sub sub, int32_t precision,
                     int64_t k, int32_t *path_out);

/* --------------------------------------------------------------- products */
/* y = H_S x for k right-hand sides (Methods, "Matrix evaluation": the
 * matrix-free product recomputes each element per call, in parallel over
 * row bit-strings; each row gathers from the columns its groups reach).
 * x and y are device arrays [D][k] row-major, of double (QSD_FP64) or float
 * (QSD_FP32_MIXED: each row accumulated in FP64 and rounded once;
 * QSD_FP32_DOT2: each row accumulated by the Dot2 scheme and rounded once).
 * x and y must not overlap.  Per row the diagonal is applied first, then the
 * groups in group order, and the terms of a group in term order, so results
 * are deterministic.  Asynchronous on the context stream.  The first product
 * of an (operator, subspace) pair computes and caches the diagonal of H_S
 * (Methods, "Matrix evaluation": the diagonal is computed once and cached).
 * Errors: QSD_ERR_COMPLEX_UNSUPPORTED when the operator has complex matrix
 * elements; QSD_ERR_INVALID_ARG on qubit-count mismatch or k < 1. */
int qsd_apply_H(qsd_ctx ctx, qsd_op op, qsd_sub sub, int precision, int32_t k,
                const void *x, void *y);

/* Complex product y = H_S x for any operator, including complex matrix
 * elements and non-Hermitian operators (Methods, "Qubit Hamiltonians":
 * complex coefficients c_i), FP64.  x, y: device complex128 [dim][k], each
 * entry (re, im) interleaved (the layout of C99 double complex and of
 * torch.complex128).  Every group is evaluated term by term; one lookup per
 * group with a passing term; deterministic.  n <= 256 qubits.  Asynchronous
 * on the context's stream. */
int qsd_apply_H_complex(qsd_ctx ctx, qsd_op op, qsd_sub sub, int32_t k,
                        const void *x, void *y);

/* Packed products: y_i = H_S(ops[i], subs[i]) x_i for i < n, for many small
 * subspaces whose single products would each fill only a few blocks.  Pairs
 * are grouped by class -- the sector-factored product (QSD_PATH_FACTORED)
 * where it applies to the pair, else the one-lane group scan
 * (QSD_PATH_SCAN_1), by key width -- and each class runs as one persistent
 * launch over a device tile queue (8-row tiles of factored pairs, 256-row
 * tiles of scanned pairs): the resident grid claims tiles by atomic
 * increments until they run out, with no block waiting on another.  Each
 * pair's result is bitwise that of qsd_apply_H on its class's path.
 * xs[i], ys[i]: device [D_i][k] in the precision's storage type; all pairs
 * share precision and k; n <= 256 qubits per pair.  Asynchronous on the
 * context's stream.  The paper evaluates one subspace at a time; this is the
 * batching of many products into one launch. */
int qsd_apply_H_batch(qsd_ctx ctx, int32_t n, const qsd_op *ops, const qsd_sub *subs,
                      int precision, int32_t k, const void *const *xs, void *const *ys);

/* As qsd_apply_H with x and y in HOST memory: copies x to the device, applies,
 * copies y back and synchronises.  Pinned host buffers copy fastest. */
int qsd_apply_H_host(qsd_ctx ctx, qsd_op op, qsd_sub sub, int precision,
                     int32_t k, const void *x_host, void *y_host);

/* Diagonal of H_S into device double [D] (real part). */
int qsd_diagonal(qsd_ctx ctx, qsd_op op, qsd_sub sub, double *d_out);

/* Target table of rows row0 .. row0+nrows-1: out is device int64
 * [nrows][n_groups] in group order; entry = -2 when no term of the group is
 * nonzero at the row (the group is skipped with no lookup, Methods "Matrix
 * evaluation"), -1 when the column is not in the subspace, else the column
 * index. */
int qsd_target_table(qsd_ctx ctx, qsd_op op, qsd_sub sub, int64_t row0,
                     int64_t nrows, int64_t *out);

/* Term table of rows row0 .. row0+nrows-1 for the terms as passed to
 * qsd_load_operator: out is device int8 [nrows][n_terms_in]; entry 0 when
 * <r|W_t|r xor F_t> is zero, else 1 + p where the element is i^p. */
int qsd_term_table(qsd_ctx ctx, qsd_op op, qsd_sub sub, int64_t row0,
                   int64_t nrows, int8_t *out);

/* FP64 Rayleigh quotient of a real vector u (device double [D]), the step
 * that refines a mixed-precision Ritz value (the Rayleigh quotient of a vector
 * with residual r is off by O(|r|^2)).  out (host double [3]) receives
 * out[0] = u^T H u / u^T u, out[1] = |H u - out[0] u| / |u| and out[2] = u^T u.
 * Uses device scratch of D + 4 * 2048 doubles held by the context (allocated on
 * first use, grown when a larger subspace comes).  Synchronises the stream.
 * Errors: QSD_ERR_COMPLEX_UNSUPPORTED, QSD_ERR_INVALID_ARG (u^T u == 0). */
int qsd_rayleigh_quotient(qsd_ctx ctx, qsd_op op, qsd_sub sub, const double *u, double *out);

/* The same Rayleigh quotient as qsd_rayleigh_quotient, for callers that
 * cannot allocate device memory: host programs whose own pool or allocator
 * owns the whole device (an allocation here would fail or fragment memory
 * they manage), and serving or real-time loops that reserve all memory up
 * front because cudaMalloc and cudaFree can synchronise the device and stall
 * other streams mid-flight.  It calls no cudaMalloc, cudaFree or allocating
 * library routine; its scratch is one fixed __device__ array of the library
 * (about 16.8 MB, held by every GPU that loads the library until the process
 * exits), so it serves subspaces of at most 2^20 rows and returns
 * QSD_ERR_CAPACITY above that.  The first call on a device resolves the
 * array's device address; make that first call before any stream capture.
 * All calls share the array and it keeps the last call's contents: calls that
 * overlap on the GPU race and must be serialised by the caller.  The paper has
 * no counterpart; it is a deployment variant of the refinement step. */
int qsd_rayleigh_quotient_noalloc(qsd_ctx ctx, qsd_op op, qsd_sub sub, const double *u, double *out);

/* ------------------------------------------------------------- eigensolver */
typedef struct {
    int32_t precision;     /* QSD_FP64, or QSD_FP32_MIXED / QSD_FP32_DOT2: FP32
                              Krylov basis and products (of that mode), FP64 dots
                              and tridiagonal, then FP64 refinement of the Ritz
                              value */
    int32_t max_steps;     /* Krylov dimension limit (>= 1) */
    double tol;            /* stop when |H u - theta u| / |theta| <= tol */
    double refine_tol;     /* mixed only: stop refining when the relative change
                              of the FP64 Rayleigh quotient is <= refine_tol */
    int32_t check_every;   /* solve the tridiagonal problem every this many steps */
    int32_t refine_steps;  /* mixed only: Krylov steps per FP64 refinement restart */
    int32_t max_refine;    /* mixed only: refinement restarts limit */
    int32_t use_graphs;    /* capture each block of check_every steps in a CUDA graph */
    uint64_t seed;         /* start vector entries U(-1,1) from SplitMix64(seed ^ i) */
    const double *v0;      /* optional device start vector [D] (overrides seed) */
    double time_limit_s;   /* 0 = none; else QSD_ERR_TIMEOUT after this wall time */
} qsd_lanczos_params;

typedef struct {
    int32_t steps;         /* Krylov steps taken (all phases) */
    int32_t refine_restarts;
    double residual;       /* |H u - theta u| / |theta| of the returned vector (FP64) */
    double energy_unrefined; /* Ritz value before FP64 refinement */
    int32_t status;        /* copy of the return code */
    int32_t applies;       /* number of H_S products */
} qsd_lanczos_info;

/* Fill *p with defaults: FP64, max_steps 300, tol 1e-9, refine_tol 1e-10,
 * check_every 10, refine_steps 30, max_refine 5, graphs on, seed 1. */
void qsd_lanczos_default_params(qsd_lanczos_params *p);

/* Lowest eigenvalue of the real symmetric H_S with a Lanczos solver on the
 * device, fully reorthogonalised: per step the three-term recurrence, then
 * one classical Gram-Schmidt pass of the residual against every earlier
 * vector with FP64 dots (complete reorthogonalisation; the recurrence is the
 * first pass for the two vectors whose coefficients cancel).  The workspace
 * (the basis of max_steps + 1 vectors of D values and a few vectors more)
 * comes from the context's pool (qsd_create).
 * *energy receives the Ritz value (FP64).  vec_out (optional, device double
 * [D]) receives the normalised Ritz vector.  info is optional.
 * Errors: QSD_ERR_NOT_HERMITIAN, QSD_ERR_COMPLEX_UNSUPPORTED,
 * QSD_ERR_NOT_CONVERGED (best estimate still written), QSD_ERR_TIMEOUT. */
int qsd_lanczos_ground_state(qsd_ctx ctx, qsd_op op, qsd_sub sub,
                             const qsd_lanczos_params *p, double *energy,
                             double *vec_out, qsd_lanczos_info *info);

/* Failure injection for tests (the paper has no counterpart): the next n
 * device allocations of the library, in any context or thread, fail with
 * QSD_ERR_OOM as if the device were out of memory, without calling CUDA; 0
 * cancels what is left.  The call that meets the failure returns
 * QSD_ERR_OOM and leaves its context usable.  Errors: QSD_ERR_INVALID_ARG
 * (n < 0). */
int qsd_inject_alloc_failures(int64_t n);

/* --------------------------------------------------------------- serving */
/* Continuous-batching ground-state server (the served loop of the build
 * target; the paper runs one eigensolve at a time).  One scheduler thread
 * admits queued requests in FIFO order when one of `max_active` slots is free
 * and the request's device footprint (Krylov basis, refinement basis,
 * diagonal and work vectors; the subspace and operator tables are the
 * caller's) fits in `budget_bytes` next to the admitted ones (a request
 * larger than the budget runs alone).  Each admitted request has its own
 * stream (small requests: a shared pack stream and packed graph replays,
 * see qsd_server_set_pack_rows) and advances asynchronously -- graph-captured chunks of Lanczos
 * steps, Ritz vector and FP64 residual, FP64 refinement restarts -- so the
 * work of all admitted requests overlaps on the device and requests that
 * arrive while others run start as soon as a slot and memory free up.
 * Results equal those of qsd_lanczos_ground_state with the same parameters.
 * op and sub may come from any context of the same device and must stay alive
 * until the request is done.  All calls are thread-safe. */
typedef struct qsd_server_s *qsd_server;

typedef struct {
    int64_t queued, active, completed, failed, admitted;
    uint64_t bytes_in_use, peak_bytes, budget_bytes;
    int64_t packed_requests;  /* requests admitted into a pack of small requests */
    int64_t packed_chunks;    /* packed chunks enqueued (each serves every waiting member) */
} qsd_server_stats;

int qsd_server_create(qsd_ctx ctx, size_t budget_bytes, int32_t max_active, qsd_server *out);
/* Queue a request; *ticket identifies it.  Errors: QSD_ERR_NOT_HERMITIAN,
 * QSD_ERR_COMPLEX_UNSUPPORTED, QSD_ERR_INVALID_ARG. */
int qsd_server_submit(qsd_server srv, qsd_op op, qsd_sub sub, const qsd_lanczos_params *p, uint64_t *ticket);
/* QSD_PENDING while running, else the request's final status with energy,
 * info and times (optional host double [3]: submit, admit, done, in seconds
 * since the server was created; admit = -1 if never admitted). */
int qsd_server_poll(qsd_server srv, uint64_t ticket, double *energy, qsd_lanczos_info *info, double *times);
/* As poll, blocking up to timeout_s seconds (<= 0: no limit); QSD_ERR_TIMEOUT
 * when the wait runs out. */
int qsd_server_wait(qsd_server srv, uint64_t ticket, double timeout_s, double *energy, qsd_lanczos_info *info,
                    double *times);
/* Request cancellation; the request ends with QSD_ERR_CANCELLED at its next
 * piece boundary (or at once while queued). */
int qsd_server_cancel(qsd_server srv, uint64_t ticket);
/* Forget a finished request (QSD_PENDING while it is not retired yet). */
int qsd_server_release(qsd_server srv, uint64_t ticket);
int qsd_server_get_stats(qsd_server srv, qsd_server_stats *stats);
/* Requests with at most `rows` rows whose product can be packed (the
 * sector-factored product, n <= 128 qubits, or a one-lane group scan of at
 * most 4096 groups, n <= 256) join the pack of their product precision:
 * their Lanczos chunks run together on the pack's stream, one CUDA-graph
 * replay per chunk whose launches serve every waiting member (the products
 * from device tile queues, as qsd_apply_H_batch; each Lanczos kernel once for
 * all members).  A graph is captured per (product classes present, steps)
 * on first use and replayed for any membership.  A member's Lanczos
 * arithmetic is bitwise that of the request alone with the same product.
 * Packed launches end with their longest member, while requests on their own
 * streams overlap one another's kernels: measured on GB300 (closed loop, 64
 * slots) packing pays for subspaces of a few thousand rows (about 1.4x the
 * solves/s at 1e3-4e3 rows), breaks even near 1e4 rows and loses above
 * (0.7x at 1e3-3e4 rows); 4096 is a good threshold.  0 (the default)
 * disables packing.  Applies to requests admitted afterwards. */
int qsd_server_set_pack_rows(qsd_server srv, int64_t rows);
const char *qsd_server_last_error(qsd_server srv);
/* Cancel what is queued or running, wait for the scheduler, free everything. */
int qsd_server_destroy(qsd_server srv);

#ifdef __cplusplus
}
#endif
#endif /* QSD_H */
