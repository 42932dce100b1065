/*
 * Plain CPU oracle for the subspace Hamiltonian-vector product.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this code; the library never does and
 * shares nothing with it (no headers, helpers, tables or constants).
 *
 * What it computes is the plain definition (Methods, "Qubit Hamiltonians"):
 *   H = sum_t c_t W_t,  W_t = (x)_q w_{t,q}  over the extended alphabet
 *   [Z, 0, 1, X, Y, -, +] -> codes 0..6,
 *   H_S[a,b] = <s_a| H |s_b> for the bit-strings s_a, s_b of the subspace S,
 *   y = H_S x.
 * Each word is evaluated factor by factor from the single-qubit matrix
 * elements <r|w|c>:
 *   Z : <0|Z|0> = 1, <1|Z|1> = -1        0 : <0|0|0> = 1
 *   1 : <1|1|1> = 1                       X : <1|X|0> = <0|X|1> = 1
 *   Y : <1|Y|0> = i, <0|Y|1> = -i         + : <1|+|0> = 1 (raising, |1><0|)
 *   - : <0|-|1> = 1 (lowering, |0><1|)
 * so a word has exactly one candidate column per row (Methods, properties
 * 1-2): the row with the bits under X, Y, +, - flipped.  The column is looked
 * up by binary search in the subspace sorted by integer value (word W-1 most
 * significant); its index is its rank (Methods, "Lower / upper triangle
 * evaluation": the subspace is integer-sorted).  No grouping, no masks, no
 * hash table: every term of every row is evaluated on its own, in FP64
 * complex arithmetic, in input term order.
 *
 * Bit-strings: W little-endian uint64 words per string, qubit q is bit q%64
 * of word q/64; arrays of strings are row-major [count][W].
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_QUBIT 2
#define ORC_ERR_REPEAT 3

enum { L_Z = 0, L_0 = 1, L_1 = 2, L_X = 3, L_Y = 4, L_LOWER = 5, L_RAISE = 6 };

/* ------------------------------------------------------------ bit-strings */
static int key_cmp(const uint64_t *a, const uint64_t *b, int W)
{
    for (int w = W - 1; w >= 0; --w) {
        if (a[w] < b[w]) return -1;
        if (a[w] > b[w]) return 1;
    }
    return 0;
}

static int get_bit(const uint64_t *s, int q) { return (int)((s[q >> 6] >> (q & 63)) & 1u); }
static void flip_bit(uint64_t *s, int q) { s[q >> 6] ^= (uint64_t)1 << (q & 63); }

/* Bottom-up merge sort of row indices by key (stable). */
static void sort_rows(int W, int64_t n, const uint64_t *words, int64_t *idx)
{
    int64_t *tmp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) idx[i] = i;
    for (int64_t width = 1; width < n; width *= 2) {
        for (int64_t lo = 0; lo < n; lo += 2 * width) {
            int64_t mid = lo + width < n ? lo + width : n;
            int64_t hi = lo + 2 * width < n ? lo + 2 * width : n;
            int64_t i = lo, j = mid, o = lo;
            while (i < mid && j < hi) {
                if (key_cmp(words + idx[j] * W, words + idx[i] * W, W) < 0) tmp[o++] = idx[j++];
                else tmp[o++] = idx[i++];
            }
            while (i < mid) tmp[o++] = idx[i++];
            while (j < hi) tmp[o++] = idx[j++];
        }
        memcpy(idx, tmp, sizeof(int64_t) * (size_t)n);
    }
    free(tmp);
}

/* Sort bit-strings by integer value and drop duplicates; returns the count. */
int64_t orc_sort_unique(int W, int64_t n_in, const uint64_t *words, uint64_t *out)
{
    if (n_in <= 0) return 0;
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)n_in);
    sort_rows(W, n_in, words, idx);
    int64_t d = 0;
    for (int64_t i = 0; i < n_in; ++i) {
        const uint64_t *k = words + idx[i] * W;
        if (d == 0 || key_cmp(out + (d - 1) * W, k, W) != 0) {
            memcpy(out + d * W, k, sizeof(uint64_t) * (size_t)W);
            ++d;
        }
    }
    free(idx);
    return d;
}

/* Rank of `key` in the sorted unique array, or -1 when absent. */
int64_t orc_find(int W, int64_t D, const uint64_t *keys, const uint64_t *key)
{
    int64_t lo = 0, hi = D - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        int c = key_cmp(keys + mid * W, key, W);
        if (c == 0) return mid;
        if (c < 0) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* ------------------------------------------------------------------ words */
/* Checks qubit range and that no qubit repeats inside a word. */
int orc_check_operator(int n, int64_t T, const int64_t *term_ptr,
                       const int32_t *op_qubit, const uint8_t *op_code)
{
    for (int64_t t = 0; t < T; ++t) {
        for (int64_t a = term_ptr[t]; a < term_ptr[t + 1]; ++a) {
            if (op_qubit[a] < 0 || op_qubit[a] >= n || op_code[a] > 6) return ORC_ERR_QUBIT;
            for (int64_t b = term_ptr[t]; b < a; ++b)
                if (op_qubit[b] == op_qubit[a]) return ORC_ERR_REPEAT;
        }
    }
    return ORC_OK;
}

/* <row| W_t |col>: writes the only column that can be nonzero into `col`
 * and returns 0 when the element is zero, else 1 with *ipow such that the
 * element equals i^(*ipow). */
static int word_element(const int32_t *qs, const uint8_t *cs, int64_t len,
                        const uint64_t *row, uint64_t *col, int W, int *ipow)
{
    int p = 0;
    memcpy(col, row, sizeof(uint64_t) * (size_t)W);
    for (int64_t a = 0; a < len; ++a) {
        int q = qs[a];
        int r = get_bit(row, q);
        switch (cs[a]) {
        case L_Z: if (r) p += 2; break;                        /* -1 on |1> */
        case L_0: if (r) return 0; break;                      /* |0><0| */
        case L_1: if (!r) return 0; break;                     /* |1><1| */
        case L_X: flip_bit(col, q); break;
        case L_Y: flip_bit(col, q); p += r ? 1 : 3; break;     /* <1|Y|0>=i, <0|Y|1>=-i */
        case L_LOWER: if (r) return 0; flip_bit(col, q); break; /* <0|-|1> */
        case L_RAISE: if (!r) return 0; flip_bit(col, q); break; /* <1|+|0> */
        default: return 0;
        }
    }
    *ipow = p & 3;
    return 1;
}

static void mul_ipow(double re, double im, int p, double *ore, double *oim)
{
    switch (p & 3) {
    case 0: *ore = re;  *oim = im;  break;
    case 1: *ore = -im; *oim = re;  break;
    case 2: *ore = -re; *oim = -im; break;
    default: *ore = im; *oim = -re; break;
    }
}

/* y = H_S x for k right-hand sides.  x, y are [D][k] row-major; x_im may be
 * NULL (real input); y_im may be NULL (imaginary part not stored). */
int orc_apply(int n, int W, int64_t T, const int64_t *term_ptr,
              const int32_t *op_qubit, const uint8_t *op_code,
              const double *coef_re, const double *coef_im,
              int64_t D, const uint64_t *keys, int k,
              const double *x_re, const double *x_im, double *y_re, double *y_im)
{
    int rc = orc_check_operator(n, T, term_ptr, op_qubit, op_code);
    if (rc) return rc;
    #pragma omp parallel
    {
        uint64_t *col = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)W);
        double *acc = (double *)malloc(sizeof(double) * 2 * (size_t)(k > 0 ? k : 1));
        #pragma omp for schedule(dynamic, 64)
        for (int64_t a = 0; a < D; ++a) {
            const uint64_t *row = keys + a * W;
            for (int j = 0; j < 2 * k; ++j) acc[j] = 0.0;
            for (int64_t t = 0; t < T; ++t) {
                int p;
                if (!word_element(op_qubit + term_ptr[t], op_code + term_ptr[t],
                                  term_ptr[t + 1] - term_ptr[t], row, col, W, &p))
                    continue;
                int64_t b = orc_find(W, D, keys, col);
                if (b < 0) continue;
                double hre, him;
                mul_ipow(coef_re[t], coef_im ? coef_im[t] : 0.0, p, &hre, &him);
                for (int j = 0; j < k; ++j) {
                    double xr = x_re[b * k + j], xi = x_im ? x_im[b * k + j] : 0.0;
                    acc[2 * j] += hre * xr - him * xi;
                    acc[2 * j + 1] += hre * xi + him * xr;
                }
            }
            for (int j = 0; j < k; ++j) {
                y_re[a * k + j] = acc[2 * j];
                if (y_im) y_im[a * k + j] = acc[2 * j + 1];
            }
        }
        free(col);
        free(acc);
    }
    return ORC_OK;
}

/* y[i] = (H_S x)[rows[i]] for a list of rows only (sampled checks at sizes
 * where the full product is too slow); y is [n_rows][k]. */
int orc_apply_rows(int n, int W, int64_t T, const int64_t *term_ptr,
                   const int32_t *op_qubit, const uint8_t *op_code,
                   const double *coef_re, const double *coef_im,
                   int64_t D, const uint64_t *keys, int k, const double *x_re,
                   int64_t n_rows, const int64_t *rows, double *y_re, double *y_im)
{
    int rc = orc_check_operator(n, T, term_ptr, op_qubit, op_code);
    if (rc) return rc;
    for (int64_t i = 0; i < n_rows; ++i)
        if (rows[i] < 0 || rows[i] >= D) return ORC_ERR_ARG;
    #pragma omp parallel
    {
        uint64_t *col = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)W);
        double *acc = (double *)malloc(sizeof(double) * 2 * (size_t)(k > 0 ? k : 1));
        #pragma omp for schedule(dynamic, 16)
        for (int64_t i = 0; i < n_rows; ++i) {
            const uint64_t *row = keys + rows[i] * W;
            for (int j = 0; j < 2 * k; ++j) acc[j] = 0.0;
            for (int64_t t = 0; t < T; ++t) {
                int p;
                if (!word_element(op_qubit + term_ptr[t], op_code + term_ptr[t],
                                  term_ptr[t + 1] - term_ptr[t], row, col, W, &p))
                    continue;
                int64_t b = orc_find(W, D, keys, col);
                if (b < 0) continue;
                double hre, him;
                mul_ipow(coef_re[t], coef_im ? coef_im[t] : 0.0, p, &hre, &him);
                for (int j = 0; j < k; ++j) {
                    acc[2 * j] += hre * x_re[b * k + j];
                    acc[2 * j + 1] += him * x_re[b * k + j];
                }
            }
            for (int j = 0; j < k; ++j) {
                y_re[i * k + j] = acc[2 * j];
                if (y_im) y_im[i * k + j] = acc[2 * j + 1];
            }
        }
        free(col);
        free(acc);
    }
    return ORC_OK;
}

/* Diagonal of H_S: the sum over terms whose candidate column is the row. */
int orc_diagonal(int n, int W, int64_t T, const int64_t *term_ptr,
                 const int32_t *op_qubit, const uint8_t *op_code,
                 const double *coef_re, const double *coef_im,
                 int64_t D, const uint64_t *keys, double *d_re, double *d_im)
{
    int rc = orc_check_operator(n, T, term_ptr, op_qubit, op_code);
    if (rc) return rc;
    #pragma omp parallel
    {
        uint64_t *col = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)W);
        #pragma omp for schedule(static)
        for (int64_t a = 0; a < D; ++a) {
            const uint64_t *row = keys + a * W;
            double sr = 0.0, si = 0.0;
            for (int64_t t = 0; t < T; ++t) {
                int p;
                if (!word_element(op_qubit + term_ptr[t], op_code + term_ptr[t],
                                  term_ptr[t + 1] - term_ptr[t], row, col, W, &p))
                    continue;
                if (key_cmp(col, row, W) != 0) continue;
                double hre, him;
                mul_ipow(coef_re[t], coef_im ? coef_im[t] : 0.0, p, &hre, &him);
                sr += hre; si += him;
            }
            d_re[a] = sr;
            if (d_im) d_im[a] = si;
        }
        free(col);
    }
    return ORC_OK;
}

/* Per (row, term) unit factor of the element <r|W_t|candidate column>:
 * 0 when the element is zero, else 1 + p where the factor is i^p.  Rows
 * row0 .. row0+nrows-1 of the sorted subspace; out is [nrows][T]. */
int orc_term_table(int n, int W, int64_t T, const int64_t *term_ptr,
                   const int32_t *op_qubit, const uint8_t *op_code,
                   int64_t D, const uint64_t *keys, int64_t row0, int64_t nrows,
                   int8_t *out)
{
    int rc = orc_check_operator(n, T, term_ptr, op_qubit, op_code);
    if (rc) return rc;
    if (row0 < 0 || row0 + nrows > D) return ORC_ERR_ARG;
    #pragma omp parallel
    {
        uint64_t *col = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)W);
        #pragma omp for schedule(static)
        for (int64_t i = 0; i < nrows; ++i) {
            const uint64_t *row = keys + (row0 + i) * W;
            for (int64_t t = 0; t < T; ++t) {
                int p;
                int nz = word_element(op_qubit + term_ptr[t], op_code + term_ptr[t],
                                      term_ptr[t + 1] - term_ptr[t], row, col, W, &p);
                out[i * T + t] = (int8_t)(nz ? 1 + p : 0);
            }
        }
        free(col);
    }
    return ORC_OK;
}

/* The off-diagonal structure of a word: the bits it flips (X, Y, +, -). */
static void flip_set(const int32_t *qs, const uint8_t *cs, int64_t len, uint64_t *f, int W)
{
    memset(f, 0, sizeof(uint64_t) * (size_t)W);
    for (int64_t a = 0; a < len; ++a)
        if (cs[a] >= L_X) flip_bit(f, qs[a]);
}

static int popcount_words(const uint64_t *f, int W)
{
    int c = 0;
    for (int w = 0; w < W; ++w) c += __builtin_popcountll(f[w]);
    return c;
}

/* Distinct nonempty flip sets of the terms with a nonzero coefficient,
 * ordered by (number of flipped bits, then integer value).  Writes at most
 * max_groups sets into groups ([G][W]) and returns G, or -1 on overflow. */
int64_t orc_groups(int W, int64_t T, const int64_t *term_ptr, const int32_t *op_qubit,
                   const uint8_t *op_code, const double *coef_re, const double *coef_im,
                   int64_t max_groups, uint64_t *groups)
{
    uint64_t *all = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(T > 0 ? T : 1) * (size_t)(W + 1));
    int64_t m = 0;
    int W1 = W + 1;
    for (int64_t t = 0; t < T; ++t) {
        if (coef_re[t] == 0.0 && (!coef_im || coef_im[t] == 0.0)) continue;
        uint64_t *f = all + m * W1;
        flip_set(op_qubit + term_ptr[t], op_code + term_ptr[t], term_ptr[t + 1] - term_ptr[t], f, W);
        int c = popcount_words(f, W);
        if (c == 0) continue;
        f[W] = (uint64_t)c;  /* most significant "word": the weight */
        ++m;
    }
    uint64_t *uniq = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(m > 0 ? m : 1) * (size_t)W1);
    int64_t g = orc_sort_unique(W1, m, all, uniq);
    int64_t ret = g;
    if (g > max_groups) ret = -1;
    else
        for (int64_t i = 0; i < g; ++i) memcpy(groups + i * W, uniq + i * W1, sizeof(uint64_t) * (size_t)W);
    free(all);
    free(uniq);
    return ret;
}

/* Per (row, group) target: for each group of orc_groups() order, -2 when no
 * term with that flip set is nonzero at the row (no lookup is needed), -1
 * when the candidate column is not in the subspace, else its index. */
int orc_target_table(int n, int W, int64_t T, const int64_t *term_ptr,
                     const int32_t *op_qubit, const uint8_t *op_code,
                     const double *coef_re, const double *coef_im,
                     int64_t D, const uint64_t *keys, int64_t G, const uint64_t *groups,
                     int64_t row0, int64_t nrows, int64_t *out)
{
    int rc = orc_check_operator(n, T, term_ptr, op_qubit, op_code);
    if (rc) return rc;
    if (row0 < 0 || row0 + nrows > D) return ORC_ERR_ARG;
    #pragma omp parallel
    {
        uint64_t *col = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)W);
        uint64_t *f = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)W);
        #pragma omp for schedule(static)
        for (int64_t i = 0; i < nrows; ++i) {
            const uint64_t *row = keys + (row0 + i) * W;
            int64_t *o = out + i * G;
            for (int64_t g = 0; g < G; ++g) o[g] = -2;
            for (int64_t t = 0; t < T; ++t) {
                if (coef_re[t] == 0.0 && (!coef_im || coef_im[t] == 0.0)) continue;
                int p;
                const int32_t *qs = op_qubit + term_ptr[t];
                const uint8_t *cs = op_code + term_ptr[t];
                int64_t len = term_ptr[t + 1] - term_ptr[t];
                flip_set(qs, cs, len, f, W);
                if (popcount_words(f, W) == 0) continue;
                if (!word_element(qs, cs, len, row, col, W, &p)) continue;
                /* find the group of this flip set (linear scan: plain) */
                for (int64_t g = 0; g < G; ++g) {
                    if (key_cmp(groups + g * W, f, W) == 0) {
                        o[g] = orc_find(W, D, keys, col);
                        break;
                    }
                }
            }
        }
        free(col);
        free(f);
    }
    return ORC_OK;
}

/* ------------------------------------------------ one row, any bit-string */
/* Row `row` of H over the whole Hilbert space (not a subspace): every
 * distinct column reached by a term with a nonzero coefficient and a nonzero
 * element, with the summed element, in ascending integer order; the diagonal
 * (column == row) is always listed.  cols is [T + 1][W], re/im [T + 1].
 * Returns the number of entries. */
typedef struct { const uint64_t *col; double re, im; } rowent_t;
static int rowent_W;

static int rowent_cmp(const void *a, const void *b)
{
    const uint64_t *x = ((const rowent_t *)a)->col, *y = ((const rowent_t *)b)->col;
    for (int w = rowent_W - 1; w >= 0; --w)
        if (x[w] != y[w]) return x[w] < y[w] ? -1 : 1;
    return 0;
}

int64_t orc_row_elements(int n, int W, int64_t T, const int64_t *term_ptr, const int32_t *op_qubit,
                         const uint8_t *op_code, const double *coef_re, const double *coef_im,
                         const uint64_t *row, uint64_t *cols, double *re, double *im)
{
    int rc = orc_check_operator(n, T, term_ptr, op_qubit, op_code);
    if (rc) return -(int64_t)rc;
    uint64_t *tmp = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(T + 1) * (size_t)W);
    rowent_t *ent = (rowent_t *)malloc(sizeof(rowent_t) * (size_t)(T + 1));
    int64_t m = 0;
    memcpy(tmp, row, sizeof(uint64_t) * (size_t)W);
    ent[m].col = tmp; ent[m].re = 0.0; ent[m].im = 0.0; ++m;
    for (int64_t t = 0; t < T; ++t) {
        int p;
        if (coef_re[t] == 0.0 && (!coef_im || coef_im[t] == 0.0)) continue;
        uint64_t *c = tmp + (size_t)m * W;
        if (!word_element(op_qubit + term_ptr[t], op_code + term_ptr[t], term_ptr[t + 1] - term_ptr[t],
                          row, c, W, &p))
            continue;
        mul_ipow(coef_re[t], coef_im ? coef_im[t] : 0.0, p, &ent[m].re, &ent[m].im);
        ent[m].col = c;
        ++m;
    }
    rowent_W = W;
    qsort(ent, (size_t)m, sizeof(rowent_t), rowent_cmp);
    int64_t u = 0;
    for (int64_t i = 0; i < m; ++i) {
        if (u > 0 && rowent_cmp(&ent[u - 1], &ent[i]) == 0) {
            ent[u - 1].re += ent[i].re;
            ent[u - 1].im += ent[i].im;
        } else {
            ent[u++] = ent[i];
        }
    }
    for (int64_t i = 0; i < u; ++i) {
        memcpy(cols + (size_t)i * W, ent[i].col, sizeof(uint64_t) * (size_t)W);
        re[i] = ent[i].re;
        im[i] = ent[i].im;
    }
    free(ent);
    free(tmp);
    return u;
}

/* --------------------------------------------------------------- CSR form */
/* Entries of row a: the diagonal (always), plus every column in S that at
 * least one term reaches with a nonzero element.  Columns ascending; values
 * are sums over the terms (numeric zeros kept). */
typedef struct { int64_t col; double re, im; } entry_t;

static int entry_cmp(const void *a, const void *b)
{
    int64_t x = ((const entry_t *)a)->col, y = ((const entry_t *)b)->col;
    return (x > y) - (x < y);
}

static int64_t row_entries(int W, int64_t T, const int64_t *term_ptr, const int32_t *op_qubit,
                           const uint8_t *op_code, const double *coef_re, const double *coef_im,
                           int64_t D, const uint64_t *keys, int64_t a, entry_t *buf, uint64_t *col)
{
    const uint64_t *row = keys + a * W;
    int64_t m = 0;
    buf[m].col = a; buf[m].re = 0.0; buf[m].im = 0.0; ++m;
    for (int64_t t = 0; t < T; ++t) {
        int p;
        /* a word whose coefficient is exactly zero is not a term of H */
        if (coef_re[t] == 0.0 && (!coef_im || coef_im[t] == 0.0))
            continue;
        if (!word_element(op_qubit + term_ptr[t], op_code + term_ptr[t],
                          term_ptr[t + 1] - term_ptr[t], row, col, W, &p))
            continue;
        int64_t b = orc_find(W, D, keys, col);
        if (b < 0) continue;
        double hre, him;
        mul_ipow(coef_re[t], coef_im ? coef_im[t] : 0.0, p, &hre, &him);
        buf[m].col = b; buf[m].re = hre; buf[m].im = him; ++m;
    }
    qsort(buf, (size_t)m, sizeof(entry_t), entry_cmp);
    int64_t u = 0;
    for (int64_t i = 0; i < m; ++i) {
        if (u > 0 && buf[u - 1].col == buf[i].col) {
            buf[u - 1].re += buf[i].re;
            buf[u - 1].im += buf[i].im;
        } else {
            buf[u++] = buf[i];
        }
    }
    return u;
}

/* Pass 1: number of stored entries per row (row_nnz[D]). */
int orc_csr_count(int n, int W, int64_t T, const int64_t *term_ptr, const int32_t *op_qubit,
                  const uint8_t *op_code, const double *coef_re, const double *coef_im,
                  int64_t D, const uint64_t *keys, int64_t *row_nnz)
{
    int rc = orc_check_operator(n, T, term_ptr, op_qubit, op_code);
    if (rc) return rc;
    #pragma omp parallel
    {
        entry_t *buf = (entry_t *)malloc(sizeof(entry_t) * (size_t)(T + 1));
        uint64_t *col = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)W);
        #pragma omp for schedule(dynamic, 64)
        for (int64_t a = 0; a < D; ++a)
            row_nnz[a] = row_entries(W, T, term_ptr, op_qubit, op_code, coef_re, coef_im, D, keys, a, buf, col);
        free(buf);
        free(col);
    }
    return ORC_OK;
}

/* Pass 2: columns and values given indptr[D+1] from pass 1. */
int orc_csr_fill(int n, int W, int64_t T, const int64_t *term_ptr, const int32_t *op_qubit,
                 const uint8_t *op_code, const double *coef_re, const double *coef_im,
                 int64_t D, const uint64_t *keys, const int64_t *indptr,
                 int64_t *indices, double *data_re, double *data_im)
{
    int rc = orc_check_operator(n, T, term_ptr, op_qubit, op_code);
    if (rc) return rc;
    #pragma omp parallel
    {
        entry_t *buf = (entry_t *)malloc(sizeof(entry_t) * (size_t)(T + 1));
        uint64_t *col = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)W);
        #pragma omp for schedule(dynamic, 64)
        for (int64_t a = 0; a < D; ++a) {
            int64_t m = row_entries(W, T, term_ptr, op_qubit, op_code, coef_re, coef_im, D, keys, a, buf, col);
            for (int64_t i = 0; i < m; ++i) {
                indices[indptr[a] + i] = buf[i].col;
                data_re[indptr[a] + i] = buf[i].re;
                if (data_im) data_im[indptr[a] + i] = buf[i].im;
            }
        }
        free(buf);
        free(col);
    }
    return ORC_OK;
}

/* ------------------------------------------------------------ eigensolver */
/* Number of eigenvalues of the symmetric tridiagonal matrix (diagonal a[m],
 * off-diagonal b[1..m-1]) that are smaller than x (Sylvester's law of
 * inertia on the LDL^T pivots). */
static int sturm_count(int m, const double *a, const double *b, double x)
{
    int c = 0;
    double q = 1.0;
    for (int i = 0; i < m; ++i) {
        double bb = i ? b[i] * b[i] : 0.0;
        q = a[i] - x - (i ? bb / q : 0.0);
        if (q == 0.0) q = -1e-300;
        if (q < 0.0) ++c;
    }
    return c;
}

/* Smallest eigenvalue of the tridiagonal matrix by bisection. */
double orc_tridiag_min(int m, const double *a, const double *b)
{
    double lo = a[0], hi = a[0];
    for (int i = 0; i < m; ++i) {
        double r = (i ? fabs(b[i]) : 0.0) + (i + 1 < m ? fabs(b[i + 1]) : 0.0);
        if (a[i] - r < lo) lo = a[i] - r;
        if (a[i] + r > hi) hi = a[i] + r;
    }
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (sturm_count(m, a, b, mid) >= 1) hi = mid; else lo = mid;
    }
    return 0.5 * (lo + hi);
}

static uint64_t splitmix64(uint64_t *state)
{
    /* SplitMix64 (Steele, Lea & Flood, 2014): Weyl increment + finaliser */
    uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Lanczos with full reorthogonalisation (classical Gram-Schmidt applied
 * twice) on H_S, which must be real symmetric (the real part of H_S x is
 * used), from a start vector of U(-1,1) entries
 * drawn with SplitMix64 from `seed` (entry i uses state seed ^ i), or from v0
 * when given.  Stops when the lowest Ritz value changed by at most
 * tol*|theta| over the last 5 steps, when beta vanishes, or after m_max
 * steps.  Returns the lowest Ritz value in *energy and the step count. */
int orc_lanczos(int n, int W, int64_t T, const int64_t *term_ptr, const int32_t *op_qubit,
                const uint8_t *op_code, const double *coef_re, const double *coef_im,
                int64_t D, const uint64_t *keys,
                int m_max, double tol, uint64_t seed, const double *v0,
                double *energy, int *steps)
{
    if (D <= 0 || m_max <= 0) return ORC_ERR_ARG;
    if (m_max > D) m_max = (int)D;
    double *V = (double *)malloc(sizeof(double) * (size_t)D * (size_t)(m_max + 1));
    double *w = (double *)malloc(sizeof(double) * (size_t)D);
    double *h = (double *)malloc(sizeof(double) * (size_t)(m_max + 1));
    double *al = (double *)calloc((size_t)m_max + 1, sizeof(double));
    double *be = (double *)calloc((size_t)m_max + 2, sizeof(double));
    double nrm = 0.0;
    for (int64_t i = 0; i < D; ++i) {
        double v;
        if (v0) v = v0[i];
        else {
            uint64_t s = seed ^ (uint64_t)i;
            v = 2.0 * ((double)(splitmix64(&s) >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
        }
        V[i] = v;
        nrm += v * v;
    }
    nrm = sqrt(nrm);
    for (int64_t i = 0; i < D; ++i) V[i] /= nrm;
    double theta = 0.0, hist[5] = {0};
    int j, rc = ORC_OK;
    for (j = 0; j < m_max; ++j) {
        double *vj = V + (size_t)j * D;
        rc = orc_apply(n, W, T, term_ptr, op_qubit, op_code, coef_re, coef_im, D, keys, 1, vj, NULL, w, NULL);
        if (rc) break;
        for (int pass = 0; pass < 2; ++pass) {
            for (int i = 0; i <= j; ++i) {
                double s = 0.0;
                const double *vi = V + (size_t)i * D;
                for (int64_t r = 0; r < D; ++r) s += vi[r] * w[r];
                h[i] = s;
            }
            for (int i = 0; i <= j; ++i) {
                const double *vi = V + (size_t)i * D;
                for (int64_t r = 0; r < D; ++r) w[r] -= h[i] * vi[r];
            }
            al[j] += h[j];
        }
        double b = 0.0;
        for (int64_t r = 0; r < D; ++r) b += w[r] * w[r];
        b = sqrt(b);
        be[j + 1] = b;
        theta = orc_tridiag_min(j + 1, al, be);
        for (int s = 4; s > 0; --s) hist[s] = hist[s - 1];
        hist[0] = theta;
        if (b <= 1e-14 * (fabs(theta) > 1.0 ? fabs(theta) : 1.0)) { ++j; break; }
        if (j >= 5) {
            double dmax = 0.0;
            for (int s = 1; s < 5; ++s) dmax = fmax(dmax, fabs(hist[s] - hist[0]));
            if (dmax <= tol * fabs(theta)) { ++j; break; }
        }
        double *vn = V + (size_t)(j + 1) * D;
        for (int64_t r = 0; r < D; ++r) vn[r] = w[r] / b;
    }
    *energy = theta;
    *steps = j;
    free(V); free(w); free(h); free(al); free(be);
    return rc;
}
