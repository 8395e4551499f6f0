/*
 * ORACLE (test infrastructure only: used by tests/ and the CPU baseline of the
 * benchmark; never by the product path).
 *
 * NInv of Section 2.2 in plain C on all host threads (OpenMP): the CPU baseline
 * variant with every core busy.  It computes what oracle.core.ninv computes:
 *
 *   W = sum_{t=0}^{m} E^t, E = I - L (Eq. (6) truncated after the m-th power),
 *   by Horner steps in column form, W_t[:, j] = e_j + sum_k E_kj W_{t-1}[:, k]
 *   over the rows k of column j of E (no value dropping);
 *   N_ij = (W^T D^{-1} W)_ij for (i, j) in S_lo (Eq. (8)), as the dot product of
 *   column i of W with column j of Y = D^{-1} W (D has 1x1 and 2x2 blocks).
 *
 * The columns of one Horner step, and the entries of the product, are
 * independent: each is one thread's work.  Sums run in a different order from
 * the sparse-matrix products of oracle.core.ninv, so the two agree to rounding.
 * Storage: L strictly lower CSC with sorted rows; W and Y column-compressed with
 * sorted rows; N in S_lo CSR order.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int64_t *cp;
    int32_t *r;
    double *v;
} csc_t;

static void csc_free(csc_t *a) {
    free(a->cp); free(a->r); free(a->v);
    a->cp = NULL; a->r = NULL; a->v = NULL;
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

int oracle_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Per-thread work arrays: a dense accumulator, membership tags and a row list. */
typedef struct {
    double *acc;
    int64_t *tag;
    int32_t *rows;
} work_t;

static int work_alloc(work_t *w, int64_t n) {
    w->acc = (double *)calloc((size_t)n + 1, sizeof(double));
    w->tag = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    w->rows = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    if (!w->acc || !w->tag || !w->rows) return -1;
    for (int64_t i = 0; i <= n; ++i) w->tag[i] = -1;
    return 0;
}

static void work_free(work_t *w) { free(w->acc); free(w->tag); free(w->rows); }

/* struct of W_t[:, j]: {j} and the rows of W_{t-1}[:, k] for k in struct(E[:, j]);
 * returns the count, rows left (unsorted) in w->rows, tags set to `stamp`. */
static int64_t gather_struct(int64_t j, int64_t stamp, const int64_t *Lcp, const int32_t *Lr, const csc_t *Wp,
                             work_t *w) {
    int64_t c = 0;
    w->tag[j] = stamp; w->rows[c++] = (int32_t)j;
    for (int64_t q = Lcp[j]; q < Lcp[j + 1]; ++q) {
        int64_t k = Lr[q];
        for (int64_t p = Wp->cp[k]; p < Wp->cp[k + 1]; ++p) {
            int32_t r = Wp->r[p];
            if (w->tag[r] != stamp) { w->tag[r] = stamp; w->rows[c++] = r; }
        }
    }
    return c;
}

/* W_t = I + W_{t-1} E in column form; returns 0 or -1 (allocation). */
static int horner_step(int64_t n, const int64_t *Lcp, const int32_t *Lr, const double *Lv, const csc_t *Wp,
                       csc_t *Wn, int64_t stamp_base) {
    Wn->cp = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    if (!Wn->cp) return -1;
    int err = 0;
#pragma omp parallel
    {
        work_t w;
        int own = work_alloc(&w, n);
        if (own != 0) {
#pragma omp atomic write
            err = -1;
        }
#pragma omp for schedule(dynamic, 64)
        for (int64_t j = 0; j < n; ++j) {
            if (own != 0) continue;
            Wn->cp[j + 1] = gather_struct(j, stamp_base + j, Lcp, Lr, Wp, &w);
        }
#pragma omp single
        {
            Wn->cp[0] = 0;
            for (int64_t j = 0; j < n; ++j) Wn->cp[j + 1] += Wn->cp[j];
            Wn->r = (int32_t *)malloc(((size_t)Wn->cp[n] + 1) * sizeof(int32_t));
            Wn->v = (double *)malloc(((size_t)Wn->cp[n] + 1) * sizeof(double));
            if (!Wn->r || !Wn->v) err = -1;
        }
        if (err == 0 && own == 0) {
#pragma omp for schedule(dynamic, 64)
            for (int64_t j = 0; j < n; ++j) {
                int64_t c = gather_struct(j, stamp_base + n + j, Lcp, Lr, Wp, &w);
                qsort(w.rows, (size_t)c, sizeof(int32_t), cmp_i32);
                w.acc[j] = 1.0;
                for (int64_t q = Lcp[j]; q < Lcp[j + 1]; ++q) {
                    int64_t k = Lr[q];
                    double e = -Lv[q];
                    for (int64_t p = Wp->cp[k]; p < Wp->cp[k + 1]; ++p) w.acc[Wp->r[p]] += e * Wp->v[p];
                }
                int64_t o = Wn->cp[j];
                for (int64_t t = 0; t < c; ++t) {
                    int32_t r = w.rows[t];
                    Wn->r[o + t] = r;
                    Wn->v[o + t] = w.acc[r];
                    w.acc[r] = 0.0;
                }
            }
        }
        work_free(&w);
    }
    return err;
}

/* Returns 0, -1 (allocation) or -2 (singular pivot block). */
int oracle_ninv_threads(int64_t n, const int64_t *Lcp, const int32_t *Lr, const double *Lv,
                        const int8_t *pivot_start, const double *d_diag, const double *d_off, int m,
                        const int64_t *Srp, const int32_t *Sc, double *N) {
    int rc = 0;
    csc_t W = {0}, Y = {0};
    double *dinv = NULL;   /* per row r: D^{-1}(r, r) and D^{-1}(partner, r) */
    double *dpart = NULL;
    int64_t *partner = NULL;
    /* W_0 = I */
    W.cp = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    W.r = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    W.v = (double *)malloc(((size_t)n + 1) * sizeof(double));
    if (!W.cp || !W.r || !W.v) { rc = -1; goto out; }
    for (int64_t j = 0; j <= n; ++j) W.cp[j] = j;
    for (int64_t j = 0; j < n; ++j) { W.r[j] = (int32_t)j; W.v[j] = 1.0; }
    for (int t = 1; t <= m; ++t) {
        csc_t Wn = {0};
        if (horner_step(n, Lcp, Lr, Lv, &W, &Wn, (int64_t)2 * n * t) != 0) { csc_free(&Wn); rc = -1; goto out; }
        csc_free(&W);
        W = Wn;
    }
    /* D^{-1} by rows: dinv[r] = D^{-1}(r, r), dpart[r] = D^{-1}(partner(r), r) */
    dinv = (double *)malloc(((size_t)n + 1) * sizeof(double));
    dpart = (double *)malloc(((size_t)n + 1) * sizeof(double));
    partner = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    if (!dinv || !dpart || !partner) { rc = -1; goto out; }
    for (int64_t j = 0; j < n;) {
        if (j + 1 < n && !pivot_start[j + 1]) {
            double a = d_diag[j], b = d_off[j], d = d_diag[j + 1];
            double det = a * d - b * b;
            if (det == 0.0) { rc = -2; goto out; }
            dinv[j] = d / det; dinv[j + 1] = a / det;
            dpart[j] = -b / det; dpart[j + 1] = -b / det;
            partner[j] = j + 1; partner[j + 1] = j;
            j += 2;
        } else {
            if (d_diag[j] == 0.0) { rc = -2; goto out; }
            dinv[j] = 1.0 / d_diag[j]; dpart[j] = 0.0; partner[j] = -1;
            j += 1;
        }
    }
    /* Y = D^{-1} W: column j has the rows of W[:, j] and their 2x2 partners */
    Y.cp = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    if (!Y.cp) { rc = -1; goto out; }
    {
        int err = 0;
#pragma omp parallel
        {
            work_t w;
            int own = work_alloc(&w, n);
            if (own != 0) {
#pragma omp atomic write
                err = -1;
            }
#pragma omp for schedule(dynamic, 64)
            for (int64_t j = 0; j < n; ++j) {
                if (own != 0) continue;
                int64_t c = 0;
                for (int64_t p = W.cp[j]; p < W.cp[j + 1]; ++p) {
                    int64_t r = W.r[p];
                    if (w.tag[r] != j) { w.tag[r] = j; ++c; }
                    if (partner[r] >= 0 && w.tag[partner[r]] != j) { w.tag[partner[r]] = j; ++c; }
                }
                Y.cp[j + 1] = c;
            }
#pragma omp single
            {
                Y.cp[0] = 0;
                for (int64_t j = 0; j < n; ++j) Y.cp[j + 1] += Y.cp[j];
                Y.r = (int32_t *)malloc(((size_t)Y.cp[n] + 1) * sizeof(int32_t));
                Y.v = (double *)malloc(((size_t)Y.cp[n] + 1) * sizeof(double));
                if (!Y.r || !Y.v) err = -1;
                for (int64_t i = 0; i <= n; ++i) w.tag[i] = -1;
            }
            if (err == 0 && own == 0) {
                for (int64_t i = 0; i <= n; ++i) w.tag[i] = -1;
#pragma omp for schedule(dynamic, 64)
                for (int64_t j = 0; j < n; ++j) {
                    int64_t c = 0;
                    for (int64_t p = W.cp[j]; p < W.cp[j + 1]; ++p) {
                        int64_t r = W.r[p];
                        double v = W.v[p];
                        if (w.tag[r] != j) { w.tag[r] = j; w.rows[c++] = (int32_t)r; }
                        w.acc[r] += dinv[r] * v;
                        if (partner[r] >= 0) {
                            int64_t q = partner[r];
                            if (w.tag[q] != j) { w.tag[q] = j; w.rows[c++] = (int32_t)q; }
                            w.acc[q] += dpart[r] * v;
                        }
                    }
                    qsort(w.rows, (size_t)c, sizeof(int32_t), cmp_i32);
                    int64_t o = Y.cp[j];
                    for (int64_t t = 0; t < c; ++t) {
                        int32_t r = w.rows[t];
                        Y.r[o + t] = r;
                        Y.v[o + t] = w.acc[r];
                        w.acc[r] = 0.0;
                    }
                }
            }
            work_free(&w);
        }
        if (err != 0) { rc = err; goto out; }
    }
    /* N_ij = W[:, i] . Y[:, j] on S_lo (sorted merge) */
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t e = Srp[i]; e < Srp[i + 1]; ++e) {
            int64_t j = Sc[e];
            int64_t a = W.cp[i], ae = W.cp[i + 1], b = Y.cp[j], be = Y.cp[j + 1];
            double s = 0.0;
            while (a < ae && b < be) {
                int32_t ra = W.r[a], rb = Y.r[b];
                if (ra == rb) { s += W.v[a] * Y.v[b]; ++a; ++b; }
                else if (ra < rb) ++a;
                else ++b;
            }
            N[e] = s;
        }
    }
out:
    csc_free(&W); csc_free(&Y);
    free(dinv); free(dpart); free(partner);
    return rc;
}
