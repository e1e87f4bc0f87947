/*
 * FP64 CPU oracle for symmetric sparse kernels (SySTeC, arXiv 2406.09266).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into liboracle.so and is
 * loaded by the tests, by the smoke check and by the CPU-baseline leg of the
 * benchmark.  The product library never links, loads or calls it, and it shares
 * no code, header, table or constant with the CUDA path.
 *
 * Everything here is the plain definition written out, in double precision:
 *   - canonical coordinates: the upper triangle, i_1 <= i_2 <= ... <= i_N
 *     (Sec. 2.1, Def. "Canonical"; full symmetry, Def. "Symmetry");
 *   - each stored canonical entry stands for every DISTINCT permutation of its
 *     indices (Sec. 3.1: n!/m! assignments when m indices are equal; Sec. 4.1,
 *     Def. "Unique Symmetry Group" S_P|E and the symmetrised-kernel pseudocode
 *     figure: for every equivalence group E, for every sigma in S_P|E, apply the
 *     assignment with permuted indices).  The oracle enumerates those
 *     permutations literally with a next-permutation step on the sorted tuple,
 *     which visits each distinct arrangement exactly once;
 *   - MTTKRP  C[i,r] = sum A[i,k,l,..] B[k,r] B[l,r] ..        (Sec. 5.2.6)
 *   - SSYMV   y[i]   = sum_j A[i,j] x[j]                        (Sec. 5.2.1)
 *   - SYPRD   y      = sum x[i] A[i,j] x[j]                      (Sec. 5.2.3)
 *   - TTM     C[i,j,l] = sum_k A[k,j,l] B[k,i]                   (Sec. 4.2, 5.2.5)
 *   - partial symmetry: a tensor symmetric only inside parts of its modes
 *     (Sec. 2 Def. "Partial Symmetry"), each entry standing for the distinct
 *     arrangements that permute inside parts; MTTKRP per part's factor.
 *   - CP fit  ||X - sum_r b_r (x) ... (x) b_r||^2, unit weights, over the full
 *     tensor (the symmetric CPD that MTTKRP serves, Sec. 5.2.6).
 * A second, independent MTTKRP form uses per-run integer weights (the
 * diagonal-splitting / simplicial-lookup-table result of Sec. 4.2.5, 4.2.9 and
 * the split loop nests of Sec. 4.3) so the two can be checked against each other.
 *
 * Pins (tests/test_oracle_*.py): dense brute force on tiny tensors (expand the
 * canonical triangle over all N! position permutations, then a dense einsum),
 * the paper's printed multiplicities 6/3/3/1 and per-row update counts for the
 * 3-way MTTKRP, the lookup-table values [2,0,1,1,0,0,1/3], closed forms
 * N!/prod(m!) for the counts, x^T(Ax) = SYPRD, relabel and input-permutation
 * invariance; for the TTM the assignments of the paper's symmetrised TTM
 * listing cell by cell, output symmetry, and the MTTKRP obtained by one more
 * contraction.  No function here is "parity unpinned".
 *
 * Conventions: 0-based indices; coordinate arrays are (order x nnz) row-major,
 * idx[q*nnz + e]; dense factors are row-major n x R.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORC_OK 0
#define ORC_INVALID (-1)
#define ORC_NONCANONICAL (-2)
#define ORC_RANGE (-3)
#define ORC_DUPLICATE (-4)
#define ORC_NOMEM (-5)

#define ORC_MAX_ORDER 5

/* ------------------------------------------------------------------------ */
/* small helpers                                                              */
/* ------------------------------------------------------------------------ */

/* In-place ascending sort of a short tuple (insertion sort). */
static void sort_tuple(int32_t* c, int order) {
    for (int a = 1; a < order; ++a) {
        int32_t t = c[a];
        int b = a - 1;
        while (b >= 0 && c[b] > t) { c[b + 1] = c[b]; --b; }
        c[b + 1] = t;
    }
}

/* Next lexicographic permutation of a[0..k); returns 0 after the last one.
 * Starting from the ascending tuple this visits every distinct arrangement
 * of the multiset exactly once. */
static int next_perm(int32_t* a, int k) {
    int i = k - 2;
    while (i >= 0 && a[i] >= a[i + 1]) --i;
    if (i < 0) return 0;
    int j = k - 1;
    while (a[j] <= a[i]) --j;
    int32_t t = a[i]; a[i] = a[j]; a[j] = t;
    for (int l = i + 1, r = k - 1; l < r; ++l, --r) { t = a[l]; a[l] = a[r]; a[r] = t; }
    return 1;
}

typedef struct {
    int32_t c[ORC_MAX_ORDER];
    float v;
    int64_t pos;
} rec_t;

static int g_order_for_cmp = 0;

static int cmp_rec(const void* pa, const void* pb) {
    const rec_t* a = (const rec_t*)pa;
    const rec_t* b = (const rec_t*)pb;
    for (int q = 0; q < g_order_for_cmp; ++q) {
        if (a->c[q] < b->c[q]) return -1;
        if (a->c[q] > b->c[q]) return 1;
    }
    /* equal coordinates: keep input order so the surviving duplicate is the first */
    if (a->pos < b->pos) return -1;
    if (a->pos > b->pos) return 1;
    return 0;
}

static void load_tuple(const int32_t* idx, int order, int64_t nnz, int64_t e, int32_t* c) {
    for (int q = 0; q < order; ++q) c[q] = idx[(int64_t)q * nnz + e];
}

/* ------------------------------------------------------------------------ */
/* Canonicalisation (Sec. 2.1 Def. Canonical, upper triangle)                 */
/* ------------------------------------------------------------------------ */

/* Sort every tuple ascending, check 0 <= c < n, sort the entries
 * lexicographically and resolve duplicates: policy 0 rejects any repeated
 * multiset; policy 1 keeps the first copy and rejects copies whose value bits
 * differ.  Output arrays have room for nnz entries. */
int orc_canonicalize(int order, int64_t n, int64_t nnz, const int32_t* idx, const float* val,
                     int dup_policy, int32_t* cidx, float* cval, int64_t* nnz_out) {
    if (order < 1 || order > ORC_MAX_ORDER || n <= 0 || nnz < 0) return ORC_INVALID;
    *nnz_out = 0;
    if (nnz == 0) return ORC_OK;
    rec_t* r = (rec_t*)malloc(sizeof(rec_t) * (size_t)nnz);
    if (!r) return ORC_NOMEM;
    for (int64_t e = 0; e < nnz; ++e) {
        load_tuple(idx, order, nnz, e, r[e].c);
        for (int q = 0; q < order; ++q)
            if (r[e].c[q] < 0 || r[e].c[q] >= n) { free(r); return ORC_RANGE; }
        sort_tuple(r[e].c, order);
        r[e].v = val[e];
        r[e].pos = e;
    }
    g_order_for_cmp = order;
    qsort(r, (size_t)nnz, sizeof(rec_t), cmp_rec);
    int64_t m = 0;
    for (int64_t e = 0; e < nnz; ++e) {
        if (m > 0) {
            int same = 1;
            for (int q = 0; q < order; ++q)
                if (r[e].c[q] != cidx[(int64_t)q * nnz + (m - 1)]) { same = 0; break; }
            if (same) {
                if (dup_policy != 1) { free(r); return ORC_DUPLICATE; }
                uint32_t ba, bb;
                memcpy(&ba, &r[e].v, 4);
                memcpy(&bb, &cval[m - 1], 4);
                if (ba != bb) { free(r); return ORC_DUPLICATE; }
                continue;
            }
        }
        for (int q = 0; q < order; ++q) cidx[(int64_t)q * nnz + m] = r[e].c[q];
        cval[m] = r[e].v;
        ++m;
    }
    free(r);
    /* compact the rows if duplicates were dropped (rows are nnz apart) */
    if (m != nnz)
        for (int q = 1; q < order; ++q)
            memmove(cidx + (int64_t)q * m, cidx + (int64_t)q * nnz, sizeof(int32_t) * (size_t)m);
    *nnz_out = m;
    return ORC_OK;
}

/* Checks that a coordinate list is canonical, sorted and duplicate free. */
int orc_check_canonical(int order, int64_t n, int64_t nnz, const int32_t* cidx) {
    int32_t prev[ORC_MAX_ORDER], c[ORC_MAX_ORDER];
    for (int64_t e = 0; e < nnz; ++e) {
        load_tuple(cidx, order, nnz, e, c);
        for (int q = 0; q < order; ++q) {
            if (c[q] < 0 || c[q] >= n) return ORC_RANGE;
            if (q > 0 && c[q - 1] > c[q]) return ORC_NONCANONICAL;
        }
        if (e > 0) {
            int cmp = 0;
            for (int q = 0; q < order && !cmp; ++q) cmp = (c[q] > prev[q]) - (c[q] < prev[q]);
            if (cmp == 0) return ORC_DUPLICATE;
            if (cmp < 0) return ORC_NONCANONICAL;
        }
        memcpy(prev, c, sizeof(c));
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Counts (integers, compared bit-exactly)                                    */
/* ------------------------------------------------------------------------ */

/* Number of distinct permutations of a canonical tuple, by enumeration. */
int64_t orc_distinct_perms(int order, const int32_t* c_in) {
    int32_t c[ORC_MAX_ORDER];
    memcpy(c, c_in, sizeof(int32_t) * (size_t)order);
    sort_tuple(c, order);
    int64_t k = 0;
    do { ++k; } while (next_perm(c, order));
    return k;
}

/* Equality pattern of a canonical tuple: bit q set when c_q == c_{q+1}. */
static int pattern_of(const int32_t* c, int order) {
    int p = 0;
    for (int q = 0; q + 1 < order; ++q)
        if (c[q] == c[q + 1]) p |= 1 << q;
    return p;
}

/* counts[p] = entries with equality pattern p (p < 16); *expanded = sum of the
 * distinct-permutation counts (nonzeros of the full tensor); *root_fibers =
 * distinct c_1; *l2_fibers = distinct (c_1, c_2); *normsq = ||X||^2 over the
 * full tensor = sum over entries of (#perms) * v^2. */
int orc_counts(int order, int64_t nnz, const int32_t* cidx, const float* cval, int64_t* counts,
               int64_t* expanded, int64_t* root_fibers, int64_t* l2_fibers, double* normsq) {
    if (order < 1 || order > ORC_MAX_ORDER) return ORC_INVALID;
    for (int p = 0; p < 16; ++p) counts[p] = 0;
    *expanded = 0; *root_fibers = 0; *l2_fibers = 0; *normsq = 0.0;
    int32_t c[ORC_MAX_ORDER], prev[ORC_MAX_ORDER];
    for (int64_t e = 0; e < nnz; ++e) {
        load_tuple(cidx, order, nnz, e, c);
        counts[pattern_of(c, order)] += 1;
        int64_t k = orc_distinct_perms(order, c);
        *expanded += k;
        *normsq += (double)k * (double)cval[e] * (double)cval[e];
        if (e == 0 || c[0] != prev[0]) *root_fibers += 1;
        if (order >= 2 && (e == 0 || c[0] != prev[0] || c[1] != prev[1])) *l2_fibers += 1;
        memcpy(prev, c, sizeof(c));
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* MTTKRP, definitional form                                                  */
/* ------------------------------------------------------------------------ */

/* M[pi_1, r] += v * prod_{q >= 2} B[pi_q, r] for every distinct permutation pi
 * of every canonical entry; this is the full-tensor MTTKRP restricted to its
 * nonzeros.  Mabs (nullable) receives sum |terms| per output element.
 * row_mask (nullable, length n) limits the work to selected output rows. */
static void mttkrp_enum_range(int order, int64_t nnz, const int32_t* cidx, const float* cval, const double* B,
                              int R, double* M, double* Mabs, const uint8_t* row_mask, int64_t e0, int64_t e1) {
    int32_t c[ORC_MAX_ORDER];
    for (int64_t e = e0; e < e1; ++e) {
        load_tuple(cidx, order, nnz, e, c);
        sort_tuple(c, order);
        double v = (double)cval[e];
        do {
            int64_t i = c[0];
            if (row_mask && !row_mask[i]) continue;
            for (int r = 0; r < R; ++r) {
                double t = v;
                for (int q = 1; q < order; ++q) t *= B[(int64_t)c[q] * R + r];
                M[i * R + r] += t;
                if (Mabs) Mabs[i * R + r] += fabs(t);
            }
        } while (next_perm(c, order));
    }
}

int orc_mttkrp_enum(int order, int64_t n, int64_t nnz, const int32_t* cidx, const float* cval,
                    const double* B, int R, double* M, double* Mabs, const uint8_t* row_mask) {
    if (order < 2 || order > ORC_MAX_ORDER || R <= 0) return ORC_INVALID;
    memset(M, 0, sizeof(double) * (size_t)n * (size_t)R);
    if (Mabs) memset(Mabs, 0, sizeof(double) * (size_t)n * (size_t)R);
    mttkrp_enum_range(order, nnz, cidx, cval, B, R, M, Mabs, row_mask, 0, nnz);
    return ORC_OK;
}

/* The same definitional MTTKRP on `threads` POSIX threads (the timing baseline
 * on all host cores): thread t takes the contiguous entries
 * [nnz t / T, nnz (t + 1) / T) into a private FP64 output, and the private
 * outputs are added into M in thread order, so the result does not depend on
 * scheduling. */
struct enum_job {
    int order;
    int64_t n, nnz, e0, e1;
    const int32_t* cidx;
    const float* cval;
    const double* B;
    int R;
    double* M;
};

static void* enum_job_run(void* arg) {
    struct enum_job* j = (struct enum_job*)arg;
    mttkrp_enum_range(j->order, j->nnz, j->cidx, j->cval, j->B, j->R, j->M, NULL, NULL, j->e0, j->e1);
    return NULL;
}

int orc_mttkrp_enum_threads(int order, int64_t n, int64_t nnz, const int32_t* cidx, const float* cval,
                            const double* B, int R, double* M, int threads) {
    if (order < 2 || order > ORC_MAX_ORDER || R <= 0 || threads < 1 || threads > 1024) return ORC_INVALID;
    const size_t cells = (size_t)n * (size_t)R;
    memset(M, 0, sizeof(double) * cells);
    struct enum_job* jobs = (struct enum_job*)calloc((size_t)threads, sizeof(struct enum_job));
    pthread_t* tid = (pthread_t*)calloc((size_t)threads, sizeof(pthread_t));
    int* started = (int*)calloc((size_t)threads, sizeof(int));
    if (!jobs || !tid || !started) {
        free(jobs);
        free(tid);
        free(started);
        return ORC_NOMEM;
    }
    int rc = ORC_OK;
    for (int t = 0; t < threads; ++t) {
        struct enum_job* j = &jobs[t];
        j->order = order;
        j->n = n;
        j->nnz = nnz;
        j->e0 = nnz * t / threads;
        j->e1 = nnz * (t + 1) / threads;
        j->cidx = cidx;
        j->cval = cval;
        j->B = B;
        j->R = R;
        j->M = (double*)calloc(cells > 0 ? cells : 1, sizeof(double));
        if (!j->M) {
            rc = ORC_NOMEM;
            break;
        }
    }
    for (int t = 0; t < threads && rc == ORC_OK; ++t)
        if (pthread_create(&tid[t], NULL, enum_job_run, &jobs[t]) == 0) started[t] = 1;
        else enum_job_run(&jobs[t]);  /* no thread: run it here */
    for (int t = 0; t < threads; ++t)
        if (started[t]) pthread_join(tid[t], NULL);
    if (rc == ORC_OK)
        for (int t = 0; t < threads; ++t)
            for (size_t k = 0; k < cells; ++k) M[k] += jobs[t].M[k];
    for (int t = 0; t < threads; ++t) free(jobs[t].M);
    free(jobs);
    free(tid);
    free(started);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Mode-1 TTM (Sec. 4.2, TTM listing; Sec. 5.2.5)                            */
/* ------------------------------------------------------------------------ */

/* C[j_2, .., j_N, r] = sum_k A[k, j_2, .., j_N] B[k, r] over the full tensor:
 * for every distinct permutation pi of every canonical entry,
 * C[pi_2, .., pi_N, r] += v * B[pi_1, r].  C is dense, row-major
 * n^(N-1) x R (the rank index fastest), and covers every output position,
 * including the non-canonical ones.  Cabs (nullable) receives sum |terms|.
 * row_slot (nullable, length n) restricts the work to the first output index
 * j_2 with row_slot[j_2] >= 0 and stores that slice at slot row_slot[j_2]
 * (C is then nslots x n^(N-2) x R). */
int orc_ttm_enum(int order, int64_t n, int64_t nnz, const int32_t* cidx, const float* cval, const double* B,
                 int R, const int32_t* row_slot, int64_t nslots, double* C, double* Cabs) {
    if (order < 2 || order > ORC_MAX_ORDER || R <= 0) return ORC_INVALID;
    int64_t cells = row_slot ? nslots : n;
    for (int q = 2; q < order; ++q) cells *= n;
    memset(C, 0, sizeof(double) * (size_t)cells * (size_t)R);
    if (Cabs) memset(Cabs, 0, sizeof(double) * (size_t)cells * (size_t)R);
    int32_t c[ORC_MAX_ORDER];
    for (int64_t e = 0; e < nnz; ++e) {
        load_tuple(cidx, order, nnz, e, c);
        sort_tuple(c, order);
        double v = (double)cval[e];
        do {
            int64_t cell = row_slot ? row_slot[c[1]] : c[1];
            if (cell < 0) continue;
            for (int q = 2; q < order; ++q) cell = cell * n + c[q];
            for (int r = 0; r < R; ++r) {
                double t = v * B[(int64_t)c[0] * R + r];
                C[cell * R + r] += t;
                if (Cabs) Cabs[cell * R + r] += fabs(t);
            }
        } while (next_perm(c, order));
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* MTTKRP, per-run weight form                                                */
/* ------------------------------------------------------------------------ */

static int64_t fact(int k) { int64_t f = 1; for (int a = 2; a <= k; ++a) f *= a; return f; }

/* For a canonical entry with distinct values u_1 < .. < u_d of multiplicities
 * m_1..m_d, the permutations whose first index is u_t number
 * W_t = (N-1)! / ((m_t - 1)! prod_{s != t} m_s!), and each contributes
 * v * prod_s B[u_s]^(m_s - [s == t]).  Written from the run structure, not by
 * enumeration. */
int orc_mttkrp_runs(int order, int64_t n, int64_t nnz, const int32_t* cidx, const float* cval,
                    const double* B, int R, double* M) {
    if (order < 2 || order > ORC_MAX_ORDER || R <= 0) return ORC_INVALID;
    memset(M, 0, sizeof(double) * (size_t)n * (size_t)R);
    int32_t c[ORC_MAX_ORDER], u[ORC_MAX_ORDER];
    int m[ORC_MAX_ORDER];
    for (int64_t e = 0; e < nnz; ++e) {
        load_tuple(cidx, order, nnz, e, c);
        sort_tuple(c, order);
        int d = 0;
        for (int q = 0; q < order; ++q) {
            if (d > 0 && u[d - 1] == c[q]) m[d - 1] += 1;
            else { u[d] = c[q]; m[d] = 1; ++d; }
        }
        double v = (double)cval[e];
        for (int t = 0; t < d; ++t) {
            int64_t den = fact(m[t] - 1);
            for (int s = 0; s < d; ++s) if (s != t) den *= fact(m[s]);
            double W = (double)(fact(order - 1) / den);
            for (int r = 0; r < R; ++r) {
                double p = W * v;
                for (int s = 0; s < d; ++s) {
                    int ex = m[s] - (s == t ? 1 : 0);
                    for (int a = 0; a < ex; ++a) p *= B[(int64_t)u[s] * R + r];
                }
                M[(int64_t)u[t] * R + r] += p;
            }
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* SSYMV and SYPRD over an upper-triangle CSR                                 */
/* ------------------------------------------------------------------------ */

/* Validates the upper CSR: rowptr monotone from 0, cols in [row, n) strictly
 * increasing within a row. */
int orc_check_upper_csr(int64_t n, const int32_t* rowptr, const int32_t* col) {
    if (n < 0 || rowptr[0] != 0) return ORC_INVALID;
    for (int64_t i = 0; i < n; ++i) {
        if (rowptr[i + 1] < rowptr[i]) return ORC_INVALID;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            if (col[p] < 0 || col[p] >= n) return ORC_RANGE;
            if (col[p] < i) return ORC_NONCANONICAL;
            if (p > rowptr[i] && col[p] <= col[p - 1]) return ORC_NONCANONICAL;
        }
    }
    return ORC_OK;
}

/* y[pi_1] += a * x[pi_2] for each distinct permutation pi of each stored (i, j). */
int orc_ssymv_enum(int64_t n, const int32_t* rowptr, const int32_t* col, const float* val,
                   const double* x, double* y, double* yabs) {
    int rc = orc_check_upper_csr(n, rowptr, col);
    if (rc) return rc;
    memset(y, 0, sizeof(double) * (size_t)n);
    if (yabs) memset(yabs, 0, sizeof(double) * (size_t)n);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            int32_t c[2] = {(int32_t)i, col[p]};
            double a = (double)val[p];
            do {
                double t = a * x[c[1]];
                y[c[0]] += t;
                if (yabs) yabs[c[0]] += fabs(t);
            } while (next_perm(c, 2));
        }
    return ORC_OK;
}

/* s = sum over distinct permutations pi of stored (i, j) of x[pi_1] a x[pi_2]. */
int orc_syprd_enum(int64_t n, const int32_t* rowptr, const int32_t* col, const float* val,
                   const double* x, double* s, double* sabs) {
    int rc = orc_check_upper_csr(n, rowptr, col);
    if (rc) return rc;
    double acc = 0.0, aabs = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            int32_t c[2] = {(int32_t)i, col[p]};
            double a = (double)val[p];
            do {
                double t = x[c[0]] * a * x[c[1]];
                acc += t;
                aabs += fabs(t);
            } while (next_perm(c, 2));
        }
    *s = acc;
    if (sabs) *sabs = aabs;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Bellman-Ford relaxation step over the symmetric matrix (Sec. 5.2.2)        */
/* ------------------------------------------------------------------------ */

/* y[pi_1] = min(y[pi_1], a + d[pi_2]) over distinct permutations; y starts at d. */
int orc_bellman_enum(int64_t n, const int32_t* rowptr, const int32_t* col, const float* val,
                     const double* d, double* y) {
    int rc = orc_check_upper_csr(n, rowptr, col);
    if (rc) return rc;
    for (int64_t i = 0; i < n; ++i) y[i] = d[i];
    for (int64_t i = 0; i < n; ++i)
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            int32_t c[2] = {(int32_t)i, col[p]};
            double a = (double)val[p];
            do {
                double t = a + d[c[1]];
                if (t < y[c[0]]) y[c[0]] = t;
            } while (next_perm(c, 2));
        }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* CP-fit residual                                                            */
/* ------------------------------------------------------------------------ */

/* res = ||X||^2 - 2 <X, Mcp> + ||Mcp||^2 where X is the full symmetric tensor
 * and Mcp = sum_r b_r (x) ... (x) b_r (unit weights).  Each inner product is
 * summed over the distinct permutations of every stored entry; ||Mcp||^2 =
 * sum_{r,s} (b_r . b_s)^N.  abs_terms (nullable) receives the sum of absolute
 * values of all terms, the denominator of the componentwise error. */
int orc_cpfit(int order, int64_t n, int64_t nnz, const int32_t* cidx, const float* cval,
              const double* B, int R, double* res, double* abs_terms, double* parts) {
    if (order < 2 || order > ORC_MAX_ORDER || R <= 0) return ORC_INVALID;
    double xx = 0.0, xm = 0.0, xm_abs = 0.0;
    int32_t c[ORC_MAX_ORDER];
    for (int64_t e = 0; e < nnz; ++e) {
        load_tuple(cidx, order, nnz, e, c);
        sort_tuple(c, order);
        double v = (double)cval[e];
        do {
            xx += v * v;
            for (int r = 0; r < R; ++r) {
                double t = v;
                for (int q = 0; q < order; ++q) t *= B[(int64_t)c[q] * R + r];
                xm += t;
                xm_abs += fabs(t);
            }
        } while (next_perm(c, order));
    }
    double mm = 0.0, mm_abs = 0.0;
    for (int r = 0; r < R; ++r)
        for (int s = 0; s < R; ++s) {
            double g = 0.0, ga = 0.0;
            for (int64_t i = 0; i < n; ++i) {
                g += B[i * R + r] * B[i * R + s];
                ga += fabs(B[i * R + r] * B[i * R + s]);
            }
            double gp = 1.0, gap = 1.0;
            for (int q = 0; q < order; ++q) { gp *= g; gap *= ga; }
            mm += gp;
            mm_abs += gap;
        }
    *res = xx - 2.0 * xm + mm;
    if (abs_terms) *abs_terms = xx + 2.0 * xm_abs + mm_abs;
    if (parts) { parts[0] = xx; parts[1] = xm; parts[2] = mm; }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Expanded (non-symmetric) tensor                                            */
/* ------------------------------------------------------------------------ */

static int g_exp_order = 0;
static int cmp_exp(const void* pa, const void* pb) {
    const rec_t* a = (const rec_t*)pa;
    const rec_t* b = (const rec_t*)pb;
    for (int q = 0; q < g_exp_order; ++q) {
        if (a->c[q] < b->c[q]) return -1;
        if (a->c[q] > b->c[q]) return 1;
    }
    return 0;
}

/* Writes every distinct permutation of every canonical entry (the nonzeros of
 * the full tensor), sorted lexicographically.  eidx is (order x cap). */
int orc_expand(int order, int64_t nnz, const int32_t* cidx, const float* cval, int64_t cap,
               int32_t* eidx, float* evals, int64_t* count) {
    if (order < 1 || order > ORC_MAX_ORDER) return ORC_INVALID;
    int64_t k = 0;
    int32_t c[ORC_MAX_ORDER];
    for (int64_t e = 0; e < nnz; ++e) {
        load_tuple(cidx, order, nnz, e, c);
        sort_tuple(c, order);
        do { ++k; } while (next_perm(c, order));
    }
    *count = k;
    if (k > cap) return ORC_NOMEM;
    rec_t* r = (rec_t*)malloc(sizeof(rec_t) * (size_t)(k > 0 ? k : 1));
    if (!r) return ORC_NOMEM;
    int64_t w = 0;
    for (int64_t e = 0; e < nnz; ++e) {
        load_tuple(cidx, order, nnz, e, c);
        sort_tuple(c, order);
        do {
            memcpy(r[w].c, c, sizeof(c));
            r[w].v = cval[e];
            r[w].pos = w;
            ++w;
        } while (next_perm(c, order));
    }
    g_exp_order = order;
    qsort(r, (size_t)k, sizeof(rec_t), cmp_exp);
    for (int64_t e = 0; e < k; ++e) {
        for (int q = 0; q < order; ++q) eidx[(int64_t)q * cap + e] = r[e].c[q];
        evals[e] = r[e].v;
    }
    free(r);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Partial symmetry (Sec. 2, Def. "Partial Symmetry"; Sec. 4.1)              */
/* ------------------------------------------------------------------------ */
/* The N modes are split into consecutive parts of sizes part[0..nparts); the
 * modes of part p range over [0, dim[p]).  The tensor is unchanged by any
 * permutation that moves positions only inside their part, so the canonical
 * coordinate has its indices non-decreasing inside every part, and a stored
 * entry stands for every distinct arrangement obtained by permuting inside
 * parts. */

static int parts_valid(int order, int nparts, const int32_t* part, const int64_t* dim) {
    if (order < 1 || order > ORC_MAX_ORDER || nparts < 1 || nparts > order) return 0;
    int total = 0;
    for (int p = 0; p < nparts; ++p) {
        if (part[p] < 1 || dim[p] < 1) return 0;
        total += part[p];
    }
    return total == order;
}

static void sort_within_parts(int32_t* c, int nparts, const int32_t* part) {
    int q = 0;
    for (int p = 0; p < nparts; ++p) {
        sort_tuple(c + q, part[p]);
        q += part[p];
    }
}

/* Next arrangement that permutes positions only inside their parts, the last
 * part varying fastest: a part that has been through all its distinct
 * arrangements goes back to ascending order and the next part to the left
 * advances.  Starting from the canonical tuple this visits every distinct
 * arrangement once; returns 0 after the last. */
static int next_part_perm(int32_t* c, int order, int nparts, const int32_t* part) {
    int start = order;
    for (int p = nparts - 1; p >= 0; --p) {
        start -= part[p];
        if (next_perm(c + start, part[p])) return 1;
        sort_tuple(c + start, part[p]);
    }
    return 0;
}

/* Canonicalisation: sort inside every part, check each index against its
 * part's dimension, sort entries lexicographically, resolve duplicates as
 * orc_canonicalize does. */
int orc_pcanonicalize(int order, int nparts, const int32_t* part, const int64_t* dim, int64_t nnz,
                      const int32_t* idx, const float* val, int dup_policy, int32_t* cidx, float* cval,
                      int64_t* nnz_out) {
    if (!parts_valid(order, nparts, part, dim) || nnz < 0) return ORC_INVALID;
    *nnz_out = 0;
    if (nnz == 0) return ORC_OK;
    int64_t mdim[ORC_MAX_ORDER];
    for (int p = 0, q = 0; p < nparts; ++p)
        for (int t = 0; t < part[p]; ++t) mdim[q++] = dim[p];
    rec_t* r = (rec_t*)malloc(sizeof(rec_t) * (size_t)nnz);
    if (!r) return ORC_NOMEM;
    for (int64_t e = 0; e < nnz; ++e) {
        load_tuple(idx, order, nnz, e, r[e].c);
        for (int q = 0; q < order; ++q)
            if (r[e].c[q] < 0 || r[e].c[q] >= mdim[q]) { free(r); return ORC_RANGE; }
        sort_within_parts(r[e].c, nparts, part);
        r[e].v = val[e];
        r[e].pos = e;
    }
    g_order_for_cmp = order;
    qsort(r, (size_t)nnz, sizeof(rec_t), cmp_rec);
    int64_t m = 0;
    for (int64_t e = 0; e < nnz; ++e) {
        if (m > 0) {
            int same = 1;
            for (int q = 0; q < order; ++q)
                if (r[e].c[q] != cidx[(int64_t)q * nnz + (m - 1)]) { same = 0; break; }
            if (same) {
                if (dup_policy != 1) { free(r); return ORC_DUPLICATE; }
                uint32_t ba, bb;
                memcpy(&ba, &r[e].v, 4);
                memcpy(&bb, &cval[m - 1], 4);
                if (ba != bb) { free(r); return ORC_DUPLICATE; }
                continue;
            }
        }
        for (int q = 0; q < order; ++q) cidx[(int64_t)q * nnz + m] = r[e].c[q];
        cval[m] = r[e].v;
        ++m;
    }
    free(r);
    if (m != nnz)
        for (int q = 1; q < order; ++q)
            memmove(cidx + (int64_t)q * m, cidx + (int64_t)q * nnz, sizeof(int32_t) * (size_t)m);
    *nnz_out = m;
    return ORC_OK;
}

/* *expanded = number of full-tensor nonzeros (arrangements, by enumeration);
 * *normsq = ||X||^2 over the full tensor. */
int orc_pcounts(int order, int nparts, const int32_t* part, int64_t nnz, const int32_t* cidx, const float* cval,
                int64_t* expanded, double* normsq) {
    *expanded = 0;
    *normsq = 0.0;
    int32_t c[ORC_MAX_ORDER];
    for (int64_t e = 0; e < nnz; ++e) {
        load_tuple(cidx, order, nnz, e, c);
        sort_within_parts(c, nparts, part);
        int64_t k = 0;
        do { ++k; } while (next_part_perm(c, order, nparts, part));
        *expanded += k;
        *normsq += (double)k * (double)cval[e] * (double)cval[e];
    }
    return ORC_OK;
}

/* MTTKRP for the factor of part out_part: with f the first mode of that part,
 * M[x_f, r] += v * prod_{q != f} F_{part of q}[x_q, r] for every arrangement x
 * of every canonical entry (permutations inside parts only) — the full-tensor
 * MTTKRP restricted to its nonzeros; any mode of the part gives the same M.
 * F holds the parts' factors one after the other, part p as a row-major
 * dim[p] x R block.  M is dim[out_part] x R; Mabs (nullable) gets sum |terms|. */
int orc_pmttkrp_enum(int order, int nparts, const int32_t* part, const int64_t* dim, int64_t nnz,
                     const int32_t* cidx, const float* cval, const double* F, int R, int out_part, double* M,
                     double* Mabs) {
    if (!parts_valid(order, nparts, part, dim) || R <= 0 || out_part < 0 || out_part >= nparts) return ORC_INVALID;
    const double* fq[ORC_MAX_ORDER];
    int f = 0;
    {
        const double* base = F;
        int q = 0;
        for (int p = 0; p < nparts; ++p) {
            if (p == out_part) f = q;
            for (int t = 0; t < part[p]; ++t) fq[q++] = base;
            base += dim[p] * (int64_t)R;
        }
    }
    memset(M, 0, sizeof(double) * (size_t)dim[out_part] * (size_t)R);
    if (Mabs) memset(Mabs, 0, sizeof(double) * (size_t)dim[out_part] * (size_t)R);
    int32_t c[ORC_MAX_ORDER];
    for (int64_t e = 0; e < nnz; ++e) {
        load_tuple(cidx, order, nnz, e, c);
        sort_within_parts(c, nparts, part);
        const double v = (double)cval[e];
        do {
            const int64_t i = c[f];
            for (int r = 0; r < R; ++r) {
                double t = v;
                for (int q = 0; q < order; ++q)
                    if (q != f) t *= fq[q][(int64_t)c[q] * R + r];
                M[i * R + r] += t;
                if (Mabs) Mabs[i * R + r] += fabs(t);
            }
        } while (next_part_perm(c, order, nparts, part));
    }
    return ORC_OK;
}

/* Mode-1 TTM of a partially symmetric order-3 tensor (Sec. 2.1, Def.
 * "Partial Symmetry"; the TTM of Sec. 4.2 and Sec. 5.2.5 with the contracted
 * factor of the first mode's part):
 *   C[j_2, j_3, r] = sum_k A[k, j_2, j_3] B[k, r]
 * over the full tensor, i.e. for every distinct inside-part arrangement pi of
 * every canonical entry, C[pi_2, pi_3, r] += v * B[pi_1, r].  B is
 * dim(part of mode 1) x R; C is dense row-major d_2 x d_3 x R (d_q the range of
 * mode q), the rank index fastest.  Cabs (nullable) receives sum |terms|. */
int orc_pttm_enum(int nparts, const int32_t* part, const int64_t* dim, int64_t nnz, const int32_t* cidx,
                  const float* cval, const double* B, int R, double* C, double* Cabs) {
    const int order = 3;
    if (!parts_valid(order, nparts, part, dim) || R <= 0) return ORC_INVALID;
    int64_t dq[3];
    {
        int q = 0;
        for (int p = 0; p < nparts; ++p)
            for (int t = 0; t < part[p]; ++t) dq[q++] = dim[p];
    }
    const size_t cells = (size_t)dq[1] * (size_t)dq[2] * (size_t)R;
    memset(C, 0, sizeof(double) * cells);
    if (Cabs) memset(Cabs, 0, sizeof(double) * cells);
    int32_t c[ORC_MAX_ORDER];
    for (int64_t e = 0; e < nnz; ++e) {
        load_tuple(cidx, order, nnz, e, c);
        sort_within_parts(c, nparts, part);
        const double v = (double)cval[e];
        do {
            const int64_t o = ((int64_t)c[1] * dq[2] + c[2]) * R;
            for (int r = 0; r < R; ++r) {
                const double t = v * B[(int64_t)c[0] * R + r];
                C[o + r] += t;
                if (Cabs) Cabs[o + r] += fabs(t);
            }
        } while (next_part_perm(c, order, nparts, part));
    }
    return ORC_OK;
}


/* Every arrangement of every canonical entry (permutations inside parts),
 * sorted lexicographically: the tensor with no symmetry left.  eidx is
 * order x cap; *count receives the number of arrangements. */
int orc_pexpand(int order, int nparts, const int32_t* part, int64_t nnz, const int32_t* cidx, const float* cval,
                int64_t cap, int32_t* eidx, float* evals, int64_t* count) {
    int64_t k = 0;
    int32_t c[ORC_MAX_ORDER];
    for (int64_t e = 0; e < nnz; ++e) {
        load_tuple(cidx, order, nnz, e, c);
        sort_within_parts(c, nparts, part);
        do { ++k; } while (next_part_perm(c, order, nparts, part));
    }
    *count = k;
    if (k > cap) return ORC_NOMEM;
    rec_t* r = (rec_t*)malloc(sizeof(rec_t) * (size_t)(k > 0 ? k : 1));
    if (!r) return ORC_NOMEM;
    int64_t w = 0;
    for (int64_t e = 0; e < nnz; ++e) {
        load_tuple(cidx, order, nnz, e, c);
        sort_within_parts(c, nparts, part);
        do {
            memcpy(r[w].c, c, sizeof(c));
            r[w].v = cval[e];
            r[w].pos = w;
            ++w;
        } while (next_part_perm(c, order, nparts, part));
    }
    g_order_for_cmp = order;
    qsort(r, (size_t)k, sizeof(rec_t), cmp_rec);
    for (int64_t e = 0; e < k; ++e) {
        for (int q = 0; q < order; ++q) eidx[(int64_t)q * cap + e] = r[e].c[q];
        evals[e] = r[e].v;
    }
    free(r);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Symmetric CP-ALS update (the shared-factor update the MTTKRP serves,      */
/* Sec. 5.2.6: one factor for all modes)                                     */
/* ------------------------------------------------------------------------ */

/* B_new = M H^{-1} with M the full-tensor MTTKRP of X with B (by enumeration),
 * H = (B^T B) raised elementwise to the power N-1, plus ridge on the diagonal.
 * H is factorised by Cholesky (H = L L^T) and every row solved by forward and
 * back substitution.  Returns the 1-based column of a non-positive pivot in
 * *info (0 = success). */
int orc_cp_als_step(int order, int64_t n, int64_t nnz, const int32_t* cidx, const float* cval, const double* B,
                    int R, double ridge, double* B_new, int* info) {
    if (order < 2 || order > ORC_MAX_ORDER || R <= 0) return ORC_INVALID;
    double* M = (double*)malloc(sizeof(double) * (size_t)n * (size_t)R);
    double* H = (double*)malloc(sizeof(double) * (size_t)R * (size_t)R);
    double* y = (double*)malloc(sizeof(double) * (size_t)R);
    if (!M || !H || !y) { free(M); free(H); free(y); return ORC_NOMEM; }
    int rc = orc_mttkrp_enum(order, n, nnz, cidx, cval, B, R, M, NULL, NULL);
    if (rc) { free(M); free(H); free(y); return rc; }
    for (int r = 0; r < R; ++r)
        for (int s = 0; s < R; ++s) {
            double g = 0.0;
            for (int64_t i = 0; i < n; ++i) g += B[i * R + r] * B[i * R + s];
            double h = 1.0;
            for (int q = 0; q < order - 1; ++q) h *= g;
            H[r * R + s] = h + (r == s ? ridge : 0.0);
        }
    /* Cholesky, lower triangle in place */
    *info = 0;
    for (int j = 0; j < R; ++j) {
        double d = H[j * R + j];
        for (int k = 0; k < j; ++k) d -= H[j * R + k] * H[j * R + k];
        if (!(d > 0.0)) { *info = j + 1; break; }
        d = sqrt(d);
        H[j * R + j] = d;
        for (int i = j + 1; i < R; ++i) {
            double t = H[i * R + j];
            for (int k = 0; k < j; ++k) t -= H[i * R + k] * H[j * R + k];
            H[i * R + j] = t / d;
        }
    }
    if (*info == 0) {
        for (int64_t i = 0; i < n; ++i) {
            /* solve L y = m_i, then L^T b = y */
            for (int r = 0; r < R; ++r) {
                double t = M[i * R + r];
                for (int k = 0; k < r; ++k) t -= H[r * R + k] * y[k];
                y[r] = t / H[r * R + r];
            }
            for (int r = R - 1; r >= 0; --r) {
                double t = y[r];
                for (int k = r + 1; k < R; ++k) t -= H[k * R + r] * B_new[i * R + k];
                B_new[i * R + r] = t / H[r * R + r];
            }
        }
    } else {
        memset(B_new, 0, sizeof(double) * (size_t)n * (size_t)R);
    }
    free(M); free(H); free(y);
    return ORC_OK;
}
