/*
 * Plain CPU oracle for CSR sparse matrix-matrix multiplication.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file; only the test suite, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code with the CUDA library.
 *
 * What it computes is the plain definition of the product (paper, Sec. 2):
 * for A (m x k) and B (k x n) in CSR, C = A B in CSR, with
 *   C_ij = sum over k in A_i of a_ik * b_kj.
 * Row i is formed the obvious way (row-wise Gustavson): for each k of row i of
 * A in stored (ascending) order, for each j of row k of B in stored
 * (ascending) order, append the pair (j, a_ik * b_kj) to a list; sort the list
 * by j, keeping list order among equal j (a library qsort over the key
 * (j, list position)); then add up each run of equal j in list order.  The
 * output pattern is structural: an entry exists wherever some product lands,
 * even if the values cancel to zero.  Columns come out ascending.
 *
 * Beside each value it returns S_ij = sum |a_ik| |b_kj| in double, the scale
 * of the entry used by the tolerance |dC_ij| <= tol * S_ij.
 *
 * Two value precisions:
 *   *_f64: double products, double sums.
 *   *_f32: float products, float sums (working precision of float data).
 * Compile with -ffp-contract=off: each product and each sum rounds once.
 *
 * The same machinery gives the ordered sum of several CSR matrices of one
 * shape (the merge of partial products, paper Sec. 4.4 / Alg. 1 line
 * "C_ijk += partial"): the list of row i is the concatenation of row i of each
 * part, in part order, and runs of equal j are added in that order.
 *
 * Parallelism: rows are independent; an OpenMP loop over rows gives identical
 * results for any thread count.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t col;
    int64_t seq; /* position in the row's product list */
} okey;

static int okey_cmp(const void* x, const void* y) {
    const okey* a = (const okey*)x;
    const okey* b = (const okey*)y;
    if (a->col != b->col) return a->col < b->col ? -1 : 1;
    if (a->seq != b->seq) return a->seq < b->seq ? -1 : 1;
    return 0;
}

static int cmp_i32(const void* x, const void* y) {
    int32_t a = *(const int32_t*)x, b = *(const int32_t*)y;
    return (a > b) - (a < b);
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Number of intermediate products of each row: u_i = sum_{k in A_i} |B_k|. */
void oracle_row_products(int64_t m, const int64_t* arp, const int32_t* acol,
                         const int64_t* brp, int64_t* u) {
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        int64_t s = 0;
        for (int64_t e = arp[i]; e < arp[i + 1]; ++e) s += brp[acol[e] + 1] - brp[acol[e]];
        u[i] = s;
    }
}

/* ---------------------------------------------------------------- product */

/* nnz of each row of C = A B (number of distinct j). */
int oracle_spgemm_counts(int64_t m, const int64_t* arp, const int32_t* acol,
                         const int64_t* brp, const int32_t* bcol, int64_t* counts) {
    int err = 0;
    #pragma omp parallel
    {
        int32_t* buf = NULL;
        int64_t cap = 0;
        #pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < m; ++i) {
            int64_t u = 0;
            for (int64_t e = arp[i]; e < arp[i + 1]; ++e) u += brp[acol[e] + 1] - brp[acol[e]];
            if (u > cap) {
                free(buf);
                cap = u;
                buf = (int32_t*)malloc((size_t)cap * sizeof(int32_t));
                if (!buf) { cap = 0; err = 1; continue; }
            }
            int64_t n = 0;
            for (int64_t e = arp[i]; e < arp[i + 1]; ++e) {
                int32_t k = acol[e];
                for (int64_t f = brp[k]; f < brp[k + 1]; ++f) buf[n++] = bcol[f];
            }
            qsort(buf, (size_t)n, sizeof(int32_t), cmp_i32);
            int64_t c = 0;
            for (int64_t t = 0; t < n; ++t)
                if (t == 0 || buf[t] != buf[t - 1]) ++c;
            counts[i] = c;
        }
        free(buf);
    }
    return err;
}

#define DEFINE_SPGEMM_FILL(NAME, T)                                                          \
int NAME(int64_t m, const int64_t* arp, const int32_t* acol, const T* aval,                  \
         const int64_t* brp, const int32_t* bcol, const T* bval,                             \
         const int64_t* crp, int32_t* ccol, T* cval, double* cabs) {                         \
    int err = 0;                                                                             \
    _Pragma("omp parallel")                                                                  \
    {                                                                                        \
        okey* key = NULL; T* prod = NULL; double* mag = NULL;                                \
        int64_t cap = 0;                                                                     \
        _Pragma("omp for schedule(dynamic, 64)")                                             \
        for (int64_t i = 0; i < m; ++i) {                                                    \
            int64_t u = 0;                                                                   \
            for (int64_t e = arp[i]; e < arp[i + 1]; ++e)                                    \
                u += brp[acol[e] + 1] - brp[acol[e]];                                        \
            if (u > cap) {                                                                   \
                free(key); free(prod); free(mag);                                            \
                cap = u;                                                                     \
                key = (okey*)malloc((size_t)cap * sizeof(okey));                             \
                prod = (T*)malloc((size_t)cap * sizeof(T));                                  \
                mag = (double*)malloc((size_t)cap * sizeof(double));                         \
                if (!key || !prod || !mag) { cap = 0; err = 1; continue; }                   \
            }                                                                                \
            int64_t n = 0;                                                                   \
            for (int64_t e = arp[i]; e < arp[i + 1]; ++e) {                                  \
                int32_t k = acol[e];                                                         \
                T a = aval[e];                                                               \
                for (int64_t f = brp[k]; f < brp[k + 1]; ++f) {                              \
                    key[n].col = bcol[f];                                                    \
                    key[n].seq = n;                                                          \
                    prod[n] = a * bval[f];                                                   \
                    mag[n] = fabs((double)a) * fabs((double)bval[f]);                        \
                    ++n;                                                                     \
                }                                                                            \
            }                                                                                \
            qsort(key, (size_t)n, sizeof(okey), okey_cmp);                                   \
            int64_t out = crp[i];                                                            \
            for (int64_t t = 0; t < n;) {                                                    \
                int32_t j = key[t].col;                                                      \
                T s = prod[key[t].seq];                                                      \
                double sm = mag[key[t].seq];                                                 \
                int64_t r = t + 1;                                                           \
                while (r < n && key[r].col == j) {                                           \
                    s = s + prod[key[r].seq];                                                \
                    sm = sm + mag[key[r].seq];                                               \
                    ++r;                                                                     \
                }                                                                            \
                if (out >= crp[i + 1]) { err = 2; break; }                                   \
                ccol[out] = j; cval[out] = s;                                                \
                if (cabs) cabs[out] = sm;                                                    \
                ++out;                                                                       \
                t = r;                                                                       \
            }                                                                                \
            if (out != crp[i + 1]) err = 2;                                                  \
        }                                                                                    \
        free(key); free(prod); free(mag);                                                    \
    }                                                                                        \
    return err;                                                                              \
}

DEFINE_SPGEMM_FILL(oracle_spgemm_fill_f64, double)
DEFINE_SPGEMM_FILL(oracle_spgemm_fill_f32, float)

/* ------------------------------------------------------ ordered sum (merge) */

/* nnz of each row of  sum_p C_p  (union of the row patterns). */
int oracle_csr_sum_counts(int32_t nparts, int64_t m, const int64_t* const* rps,
                          const int32_t* const* cols, int64_t* counts) {
    int err = 0;
    #pragma omp parallel
    {
        int32_t* buf = NULL;
        int64_t cap = 0;
        #pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < m; ++i) {
            int64_t u = 0;
            for (int32_t p = 0; p < nparts; ++p) u += rps[p][i + 1] - rps[p][i];
            if (u > cap) {
                free(buf);
                cap = u;
                buf = (int32_t*)malloc((size_t)cap * sizeof(int32_t));
                if (!buf) { cap = 0; err = 1; continue; }
            }
            int64_t n = 0;
            for (int32_t p = 0; p < nparts; ++p)
                for (int64_t f = rps[p][i]; f < rps[p][i + 1]; ++f) buf[n++] = cols[p][f];
            qsort(buf, (size_t)n, sizeof(int32_t), cmp_i32);
            int64_t c = 0;
            for (int64_t t = 0; t < n; ++t)
                if (t == 0 || buf[t] != buf[t - 1]) ++c;
            counts[i] = c;
        }
        free(buf);
    }
    return err;
}

#define DEFINE_SUM_FILL(NAME, T)                                                             \
int NAME(int32_t nparts, int64_t m, const int64_t* const* rps, const int32_t* const* cols,   \
         const T* const* vals, const int64_t* crp, int32_t* ccol, T* cval) {                 \
    int err = 0;                                                                             \
    _Pragma("omp parallel")                                                                  \
    {                                                                                        \
        okey* key = NULL; T* v = NULL;                                                       \
        int64_t cap = 0;                                                                     \
        _Pragma("omp for schedule(dynamic, 64)")                                             \
        for (int64_t i = 0; i < m; ++i) {                                                    \
            int64_t u = 0;                                                                   \
            for (int32_t p = 0; p < nparts; ++p) u += rps[p][i + 1] - rps[p][i];             \
            if (u > cap) {                                                                   \
                free(key); free(v);                                                          \
                cap = u;                                                                     \
                key = (okey*)malloc((size_t)cap * sizeof(okey));                             \
                v = (T*)malloc((size_t)cap * sizeof(T));                                     \
                if (!key || !v) { cap = 0; err = 1; continue; }                              \
            }                                                                                \
            int64_t n = 0;                                                                   \
            for (int32_t p = 0; p < nparts; ++p)                                             \
                for (int64_t f = rps[p][i]; f < rps[p][i + 1]; ++f) {                        \
                    key[n].col = cols[p][f]; key[n].seq = n; v[n] = vals[p][f]; ++n;         \
                }                                                                            \
            qsort(key, (size_t)n, sizeof(okey), okey_cmp);                                   \
            int64_t out = crp[i];                                                            \
            for (int64_t t = 0; t < n;) {                                                    \
                int32_t j = key[t].col;                                                      \
                T s = v[key[t].seq];                                                         \
                int64_t r = t + 1;                                                           \
                while (r < n && key[r].col == j) { s = s + v[key[r].seq]; ++r; }             \
                if (out >= crp[i + 1]) { err = 2; break; }                                   \
                ccol[out] = j; cval[out] = s; ++out;                                         \
                t = r;                                                                       \
            }                                                                                \
            if (out != crp[i + 1]) err = 2;                                                  \
        }                                                                                    \
        free(key); free(v);                                                                  \
    }                                                                                        \
    return err;                                                                              \
}

DEFINE_SUM_FILL(oracle_csr_sum_fill_f64, double)
DEFINE_SUM_FILL(oracle_csr_sum_fill_f32, float)

/* ----------------------------------------------------------------- backward
 *
 * For C = A B on fixed patterns and an upstream gradient G on the pattern of C
 * (G_ij = dL/dC_ij), the chain rule on C_ij = sum_k a_ik b_kj gives
 *   dL/da_ik = sum_{j in B_k} G_ij b_kj          for (i,k) in pattern(A)
 *   dL/db_kj = sum_{i : k in A_i} a_ik G_ij      for (k,j) in pattern(B)
 * i.e. (G B^T) sampled on A's pattern and (A^T G) sampled on B's pattern.
 * G_ij is found by binary search in the sorted row i of C.  dB is formed by
 * scattering over i in ascending order (serial, so the order is fixed).
 * Accumulation in double.
 */
static int64_t find_col(const int32_t* col, int64_t lo, int64_t hi, int32_t j) {
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (col[mid] < j) lo = mid + 1; else hi = mid;
    }
    return lo;
}

int oracle_spgemm_backward_f64(int64_t m, int64_t kdim,
                               const int64_t* arp, const int32_t* acol, const double* aval,
                               const int64_t* brp, const int32_t* bcol, const double* bval,
                               const int64_t* crp, const int32_t* ccol, const double* g,
                               double* da, double* db) {
    int err = 0;
    (void)kdim;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < m; ++i) {
        for (int64_t e = arp[i]; e < arp[i + 1]; ++e) {
            int32_t k = acol[e];
            double s = 0.0;
            for (int64_t f = brp[k]; f < brp[k + 1]; ++f) {
                int64_t pos = find_col(ccol, crp[i], crp[i + 1], bcol[f]);
                if (pos >= crp[i + 1] || ccol[pos] != bcol[f]) { err = 1; continue; }
                s += g[pos] * bval[f];
            }
            da[e] = s;
        }
    }
    memset(db, 0, sizeof(double) * (size_t)brp[kdim]);
    for (int64_t i = 0; i < m; ++i) {
        for (int64_t e = arp[i]; e < arp[i + 1]; ++e) {
            int32_t k = acol[e];
            double a = aval[e];
            for (int64_t f = brp[k]; f < brp[k + 1]; ++f) {
                int64_t pos = find_col(ccol, crp[i], crp[i + 1], bcol[f]);
                if (pos >= crp[i + 1] || ccol[pos] != bcol[f]) { err = 1; continue; }
                db[f] += a * g[pos];
            }
        }
    }
    return err;
}

/* ------------------------------------------- mixed precision (float in)
 *
 * Float inputs, each product rounded to float (as the float path does), the
 * products of an entry added in double in list order.  Used by the Markov
 * clustering expansion, whose decisions (prune, top-k) are taken in double.
 */
int oracle_spgemm_fill_f32p64(int64_t m, const int64_t* arp, const int32_t* acol, const float* aval,
                              const int64_t* brp, const int32_t* bcol, const float* bval,
                              const int64_t* crp, int32_t* ccol, double* cval) {
    int err = 0;
    #pragma omp parallel
    {
        okey* key = NULL; double* prod = NULL;
        int64_t cap = 0;
        #pragma omp for schedule(dynamic, 16)
        for (int64_t i = 0; i < m; ++i) {
            int64_t u = 0;
            for (int64_t e = arp[i]; e < arp[i + 1]; ++e) u += brp[acol[e] + 1] - brp[acol[e]];
            if (u > cap) {
                free(key); free(prod);
                cap = u;
                key = (okey*)malloc((size_t)cap * sizeof(okey));
                prod = (double*)malloc((size_t)cap * sizeof(double));
                if (!key || !prod) { cap = 0; err = 1; continue; }
            }
            int64_t n = 0;
            for (int64_t e = arp[i]; e < arp[i + 1]; ++e) {
                int32_t k = acol[e];
                float a = aval[e];
                for (int64_t f = brp[k]; f < brp[k + 1]; ++f) {
                    float p = a * bval[f];
                    key[n].col = bcol[f];
                    key[n].seq = n;
                    prod[n] = (double)p;
                    ++n;
                }
            }
            qsort(key, (size_t)n, sizeof(okey), okey_cmp);
            int64_t out = crp[i];
            for (int64_t t = 0; t < n;) {
                int32_t j = key[t].col;
                double s = prod[key[t].seq];
                int64_t r = t + 1;
                while (r < n && key[r].col == j) { s = s + prod[key[r].seq]; ++r; }
                if (out >= crp[i + 1]) { err = 2; break; }
                ccol[out] = j; cval[out] = s; ++out;
                t = r;
            }
            if (out != crp[i + 1]) err = 2;
        }
        free(key); free(prod);
    }
    return err;
}
