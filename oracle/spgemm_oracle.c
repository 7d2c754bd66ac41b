/*
 * CPU oracle for CSR SpGEMM (Liu & Vinter, "A Framework for General Sparse
 * Matrix-Matrix Multiplication on GPUs and Heterogeneous Processors").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * CUDA library is checked against.  It shares no code, header, table or
 * helper with the CUDA path, and only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it.
 *
 * What it computes (plain definitions, written out):
 *   - oracle_rows_count / oracle_rows_fill: C = A*B row by row, following
 *     Gustavson's row-wise formulation (Algorithm 1, Section 2.1) with a dense
 *     sparse accumulator plus a "mark" vector (the Matlab/SPA algorithm of
 *     Gilbert et al., Section 2.2).  Row i of C collects a_ij * b_jk for every
 *     stored a_ij in row i of A (visited in stored order) and every stored b_jk
 *     in row j of B (visited in stored order).  Every column reached is a
 *     structural entry of C even when its value cancels to 0.0, because the
 *     method never considers cancellation (Section 3.1).  Columns of each
 *     output row are emitted in ascending order without duplicates (the CSR
 *     convention of Section 3.2).  The fill pass also returns
 *     den_ij = sum_k |a_ik * b_kj|, the denominator of the value tolerance.
 *   - oracle_upper_bound: u_i = sum over stored a_ij of nnz(b_j*)  (Algorithm 2).
 *   - oracle_binning: the 38-bin assignment and temporary-row sizes of
 *     Algorithm 3 (Section 4.1), serially, in row order.
 *
 * Build with -ffp-contract=off so that every product and every sum is one
 * separately rounded IEEE operation.  Row pointers are int64, columns int32,
 * values double.  OpenMP (optional) parallelises over independent rows only;
 * the arithmetic inside a row is the same serial loop either way.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/*
 * ORACLE_MUTANT != 0 builds a deliberately wrong oracle, used only by the
 * oracle's own tests to show that the pins catch plausible mistakes:
 *   1 = a dropped term (the last product of each A row is skipped),
 *   2 = a wrong sign (duplicates are subtracted instead of added),
 *   3 = a wrong index (products land one column to the right, modulo n).
 * The default build (0) is the oracle.
 */
#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

typedef struct {
    int64_t *mark;   /* mark[j] == stamp  <=> column j already in the row */
    double *acc;     /* accumulated value of column j */
    double *den;     /* accumulated |a*b| of column j */
    int32_t *list;   /* columns touched, in first-touch order */
} spa_t;

static int spa_init(spa_t *s, int64_t ncols, int want_values) {
    size_t n = (size_t)(ncols > 0 ? ncols : 1);
    s->mark = (int64_t *)malloc(n * sizeof(int64_t));
    s->list = (int32_t *)malloc(n * sizeof(int32_t));
    s->acc = want_values ? (double *)malloc(n * sizeof(double)) : NULL;
    s->den = want_values ? (double *)malloc(n * sizeof(double)) : NULL;
    if (!s->mark || !s->list || (want_values && (!s->acc || !s->den))) return -1;
    for (size_t j = 0; j < n; ++j) s->mark[j] = -1;
    return 0;
}

static void spa_free(spa_t *s) {
    free(s->mark); free(s->list); free(s->acc); free(s->den);
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Number of structural entries of row i of C (the boolean product row). */
static int64_t row_count(int64_t i, const int64_t *arp, const int32_t *acol,
                         const int64_t *brp, const int32_t *bcol, spa_t *s) {
    int64_t n = 0;
    for (int64_t p = arp[i]; p < arp[i + 1]; ++p) {
        int32_t j = acol[p];
        for (int64_t q = brp[j]; q < brp[j + 1]; ++q) {
            int32_t k = bcol[q];
            if (s->mark[k] != i) { s->mark[k] = i; ++n; }
        }
    }
    return n;
}

/*
 * rows == NULL selects all rows 0..nsel-1; otherwise rows[0..nsel) lists the
 * rows to evaluate (any order, duplicates allowed).  counts[t] receives
 * nnz(c_{rows[t]*}).
 */
int oracle_rows_count(int64_t ncols_b,
                      const int64_t *arp, const int32_t *acol,
                      const int64_t *brp, const int32_t *bcol,
                      const int64_t *rows, int64_t nsel, int64_t *counts, int nthreads) {
    int err = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel reduction(| : err)
#endif
    {
        spa_t s;
        if (spa_init(&s, ncols_b, 0) != 0) {
            err = 1;
        } else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
            for (int64_t t = 0; t < nsel; ++t) {
                int64_t i = rows ? rows[t] : t;
                /* stamps must be unique per evaluated row within this thread */
                counts[t] = row_count(i, arp, acol, brp, bcol, &s);
                /* reset marks touched by this row so a repeated row id works */
                for (int64_t p = arp[i]; p < arp[i + 1]; ++p) {
                    int32_t j = acol[p];
                    for (int64_t q = brp[j]; q < brp[j + 1]; ++q) s.mark[bcol[q]] = -1;
                }
            }
            spa_free(&s);
        }
    }
    (void)nthreads;
    return err;
}

/*
 * Fills the selected rows.  out_off[t] is the first output slot of selected row
 * t (the caller computes it from oracle_rows_count); the row's columns go to
 * out_col[out_off[t] ...] ascending, its values to out_val and the tolerance
 * denominators sum|a*b| to out_den (out_den may be NULL).
 */
int oracle_rows_fill(int64_t ncols_b,
                     const int64_t *arp, const int32_t *acol, const double *aval,
                     const int64_t *brp, const int32_t *bcol, const double *bval,
                     const int64_t *rows, int64_t nsel, const int64_t *out_off,
                     int32_t *out_col, double *out_val, double *out_den, int nthreads) {
    int err = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel reduction(| : err)
#endif
    {
        spa_t s;
        if (spa_init(&s, ncols_b, 1) != 0) {
            err = 1;
        } else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
            for (int64_t t = 0; t < nsel; ++t) {
                int64_t i = rows ? rows[t] : t;
                int64_t n = 0;
                /* Algorithm 1: for each a_ij in row i, for each b_jk in row j */
                for (int64_t p = arp[i]; p < arp[i + 1]; ++p) {
                    int32_t j = acol[p];
                    double a = aval[p];
                    for (int64_t q = brp[j]; q < brp[j + 1]; ++q) {
                        int32_t k = bcol[q];
                        double v = a * bval[q];
#if ORACLE_MUTANT == 1
                        if (p == arp[i + 1] - 1 && q == brp[j + 1] - 1 && arp[i + 1] - arp[i] > 1) continue;
#elif ORACLE_MUTANT == 3
                        k = (int32_t)((k + 1) % ncols_b);
#endif
                        if (s.mark[k] != i) {      /* c_ik not yet in c_i*: insert */
                            s.mark[k] = i;
                            s.acc[k] = v;
                            s.den[k] = fabs(v);
                            s.list[n++] = k;
                        } else {                   /* c_ik += a_ij * b_jk */
#if ORACLE_MUTANT == 2
                            s.acc[k] = s.acc[k] - v;
#else
                            s.acc[k] = s.acc[k] + v;
#endif
                            s.den[k] = s.den[k] + fabs(v);
                        }
                    }
                }
                qsort(s.list, (size_t)n, sizeof(int32_t), cmp_i32);
                int64_t o = out_off[t];
                for (int64_t r = 0; r < n; ++r) {
                    int32_t k = s.list[r];
                    out_col[o + r] = k;
                    out_val[o + r] = s.acc[k];
                    if (out_den) out_den[o + r] = s.den[k];
                    s.mark[k] = -1;
                }
            }
            spa_free(&s);
        }
    }
    (void)nthreads;
    return err;
}

/* Algorithm 2: u_i <- sum over stored a_ij of nnz(b_j*). */
void oracle_upper_bound(int64_t m, const int64_t *arp, const int32_t *acol,
                        const int64_t *brp, int64_t *u) {
    for (int64_t i = 0; i < m; ++i) {
        int64_t s = 0;
        for (int64_t p = arp[i]; p < arp[i + 1]; ++p) {
            int32_t j = acol[p];
            s += brp[j + 1] - brp[j];
        }
        u[i] = s;
    }
}

/*
 * Algorithm 3 (stage 2 on a CPU core).  For each row, in row order, assign a
 * bin and the size of the row in the temporary matrix C~:
 *   u = 0       -> bin 0,  size 0
 *   u = 1       -> bin 1,  size 1
 *   2..32       -> bin u,  size u
 *   33..64      -> bin 33, size u
 *   65..128     -> bin 34, size u
 *   129..256    -> bin 35, size u
 *   257..512    -> bin 36, size u
 *   > 512       -> bin 37, size 256
 * bin_rows receives the row indices grouped by bin (bin 0 first), in row order
 * within each bin; bin_count[38] the bin sizes; the return value is nnz(C~).
 */
int64_t oracle_binning(int64_t m, const int64_t *u, int32_t *bin, int64_t *size,
                       int64_t *bin_count, int32_t *bin_rows) {
    for (int b = 0; b < 38; ++b) bin_count[b] = 0;
    int64_t total = 0;
    for (int64_t i = 0; i < m; ++i) {
        int64_t ui = u[i];
        int b;
        int64_t sz;
        if (ui == 0) { b = 0; sz = 0; }
        else if (ui == 1) { b = 1; sz = 1; }
        else if (ui >= 2 && ui <= 32) { b = (int)ui; sz = ui; }
        else if (ui >= 33 && ui <= 64) { b = 33; sz = ui; }
        else if (ui >= 65 && ui <= 128) { b = 34; sz = ui; }
        else if (ui >= 129 && ui <= 256) { b = 35; sz = ui; }
        else if (ui >= 257 && ui <= 512) { b = 36; sz = ui; }
        else { b = 37; sz = 256; }
        bin[i] = b;
        size[i] = sz;
        bin_count[b] += 1;
        total += sz;
    }
    /* "insert i to bin_b": the bins are one array of size m in 38 segments */
    int64_t start[39];
    start[0] = 0;
    for (int b = 0; b < 38; ++b) start[b + 1] = start[b] + bin_count[b];
    for (int64_t i = 0; i < m; ++i) bin_rows[start[bin[i]]++] = (int32_t)i;
    return total;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
