/*
 * Incomplete LDL^T factorisation with a drop tolerance and adjacent 1x1/2x2
 * pivots, plus a solve with the resulting factors.
 *
 * This produces the INPUTS of the selected-inverse path (the paper takes the
 * factors of a block ILDL as given: Section 2, Eq. (1) "A ~ L D L^T" with L
 * block unit lower triangular and D block diagonal).  It computes nothing of
 * the selected inverse itself.
 *
 * Algorithm: left-looking (Crout) column elimination in the given order.
 *   Column j of the current Schur complement is
 *       w = A(j:n, j) - sum_{pivot blocks P < j} L(j:n, P) D_P L(j, P)^T .
 *   Pivot test (Bunch-Kaufman restricted to the adjacent pair, no interchange):
 *       1x1 if |w_jj| >= alpha |w_{j+1,j}|, else the 2x2 block {j, j+1}.
 *   New factor column(s):  L(r, P) = w(r, P) D_P^{-1}  for r past the block, and
 *   an entry is dropped when |L(r, p)| < tau (tau = 0 keeps every structural
 *   entry).  A 1x1 pivot with |d| < static_piv is replaced by +-static_piv; a 2x2
 *   block with |det| < static_piv^2 has static_piv added (with sign) to its
 *   diagonal.  Both replacements are counted.
 *
 * Storage: the input is the lower triangle (diagonal included) of a symmetric
 * matrix in CSC with sorted rows; the output L is strictly lower CSC with sorted
 * rows; D is returned as d_diag[n] and d_off[n] (d_off[j] = D(j+1, j) when j
 * starts a 2x2 block, else 0) with pivot_start[n] (1 = a block starts here).
 * A 2x2 block never stores L(j+1, j) (it is zero: the block of L is I).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int64_t n;
    int64_t nnz;
    int64_t cap;
    int64_t *colptr; /* n+1 */
    int32_t *row;
    double *val;
    int8_t *pivot_start;
    double *d_diag;
    double *d_off;
    int64_t n_static;
    int64_t n_2x2;
} ildl_result;

static int grow(ildl_result *R, int64_t need) {
    if (R->nnz + need <= R->cap) return 0;
    int64_t cap = R->cap ? R->cap : 1024;
    while (cap < R->nnz + need) cap *= 2;
    int32_t *r = (int32_t *)realloc(R->row, (size_t)cap * sizeof(int32_t));
    if (!r) return -1;
    R->row = r;
    double *v = (double *)realloc(R->val, (size_t)cap * sizeof(double));
    if (!v) return -1;
    R->val = v;
    R->cap = cap;
    return 0;
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

typedef struct {
    double *w;
    int64_t *mark;
    int32_t *list;
    int64_t cnt;
} work_col;

static inline void acc(work_col *W, int64_t stamp, int32_t r, double x) {
    if (W->mark[r] != stamp) {
        W->mark[r] = stamp;
        W->w[r] = 0.0;
        W->list[W->cnt++] = r;
    }
    W->w[r] += x;
}

typedef struct {
    int64_t n;
    const int64_t *Acp;
    const int32_t *Ar;
    const double *Av;
    ildl_result *R;
    int64_t *ptr;     /* first entry of column k with row >= current column */
    int32_t *head;    /* linked lists of columns keyed by ptr row */
    int32_t *next;
    int64_t *blkmark;
} state;

/* Schur complement column c (rows >= c) into W. */
static void schur_column(state *S, int64_t c, work_col *W) {
    ildl_result *R = S->R;
    W->cnt = 0;
    for (int64_t p = S->Acp[c]; p < S->Acp[c + 1]; ++p) {
        int32_t r = S->Ar[p];
        if (r >= c) acc(W, c, r, S->Av[p]);
    }
    acc(W, c, (int32_t)c, 0.0);
    for (int32_t k = S->head[c]; k != -1; k = S->next[k]) {
        int64_t b = R->pivot_start[k] ? k : k - 1;
        if (S->blkmark[b] == c) continue;
        S->blkmark[b] = c;
        int two = (b + 1 < c) && !R->pivot_start[b + 1];
        if (!two) {
            int64_t q0 = S->ptr[b];
            double coef = R->d_diag[b] * R->val[q0];
            for (int64_t q = q0; q < R->colptr[b + 1]; ++q) acc(W, c, R->row[q], -R->val[q] * coef);
        } else {
            int64_t k0 = b, k1 = b + 1;
            int64_t p0 = S->ptr[k0], p1 = S->ptr[k1];
            double l0 = (p0 < R->colptr[k0 + 1] && R->row[p0] == c) ? R->val[p0] : 0.0;
            double l1 = (p1 < R->colptr[k1 + 1] && R->row[p1] == c) ? R->val[p1] : 0.0;
            double c0 = R->d_diag[k0] * l0 + R->d_off[k0] * l1;
            double c1 = R->d_off[k0] * l0 + R->d_diag[k1] * l1;
            for (int64_t q = p0; q < R->colptr[k0 + 1]; ++q) acc(W, c, R->row[q], -R->val[q] * c0);
            for (int64_t q = p1; q < R->colptr[k1 + 1]; ++q) acc(W, c, R->row[q], -R->val[q] * c1);
        }
    }
}

/* Move every column whose current row is c on to its next row. */
static void advance(state *S, int64_t c) {
    ildl_result *R = S->R;
    int32_t k = S->head[c];
    S->head[c] = -1;
    while (k != -1) {
        int32_t nk = S->next[k];
        int64_t p = ++S->ptr[k];
        if (p < R->colptr[k + 1]) {
            int32_t r = R->row[p];
            S->next[k] = S->head[r];
            S->head[r] = k;
        }
        k = nk;
    }
}

static void link_new_column(state *S, int64_t k) {
    ildl_result *R = S->R;
    S->ptr[k] = R->colptr[k];
    if (R->colptr[k] < R->colptr[k + 1]) {
        int32_t r = R->row[R->colptr[k]];
        S->next[k] = S->head[r];
        S->head[r] = (int32_t)k;
    }
}

int ildl_factor(int64_t n, const int64_t *Acp, const int32_t *Ar, const double *Av, double tau,
                double alpha, double static_piv, int allow_2x2, ildl_result *R) {
    memset(R, 0, sizeof(*R));
    R->n = n;
    R->colptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    R->pivot_start = (int8_t *)calloc((size_t)n + 1, 1);
    R->d_diag = (double *)calloc((size_t)n + 1, sizeof(double));
    R->d_off = (double *)calloc((size_t)n + 1, sizeof(double));
    work_col W1 = {0}, W2 = {0};
    int32_t *ulist = NULL;
    int64_t *umark = NULL;
    state S = {0};
    int rc = -1;
    S.n = n; S.Acp = Acp; S.Ar = Ar; S.Av = Av; S.R = R;
    S.ptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    S.head = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    S.next = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    S.blkmark = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    W1.w = (double *)malloc(((size_t)n + 1) * sizeof(double));
    W1.mark = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    W1.list = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    W2.w = (double *)malloc(((size_t)n + 1) * sizeof(double));
    W2.mark = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    W2.list = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    ulist = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    umark = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    if (!R->colptr || !R->pivot_start || !R->d_diag || !R->d_off || !S.ptr || !S.head || !S.next ||
        !S.blkmark || !W1.w || !W1.mark || !W1.list || !W2.w || !W2.mark || !W2.list || !ulist || !umark)
        goto done;
    for (int64_t i = 0; i <= n; ++i) {
        S.head[i] = -1; S.next[i] = -1; S.blkmark[i] = -1;
        W1.mark[i] = -1; W2.mark[i] = -1; umark[i] = -1;
    }
    int64_t j = 0;
    while (j < n) {
        R->colptr[j] = R->nnz;
        R->pivot_start[j] = 1; /* set before any Schur column reads the block layout */
        schur_column(&S, j, &W1);
        double a = W1.w[j];
        double s = (j + 1 < n && W1.mark[j + 1] == j) ? W1.w[j + 1] : 0.0;
        int two = allow_2x2 && (j + 1 < n) && (fabs(a) < alpha * fabs(s));
        if (!two) {
            advance(&S, j);
            double d = a;
            if (fabs(d) < static_piv) { d = (d >= 0.0 ? 1.0 : -1.0) * static_piv; R->n_static++; }
            R->pivot_start[j] = 1;
            R->d_diag[j] = d;
            int64_t m = 0;
            for (int64_t t = 0; t < W1.cnt; ++t)
                if (W1.list[t] > j) W1.list[m++] = W1.list[t];
            qsort(W1.list, (size_t)m, sizeof(int32_t), cmp_i32);
            if (grow(R, m)) goto done;
            for (int64_t t = 0; t < m; ++t) {
                int32_t r = W1.list[t];
                double l = W1.w[r] / d;
                if (fabs(l) >= tau) { R->row[R->nnz] = r; R->val[R->nnz] = l; R->nnz++; }
            }
            R->colptr[j + 1] = R->nnz;
            link_new_column(&S, j);
            j += 1;
        } else {
            advance(&S, j);
            schur_column(&S, j + 1, &W2);
            advance(&S, j + 1);
            double c = W2.w[j + 1];
            double det = a * c - s * s;
            if (fabs(det) < static_piv * static_piv) {
                a += (a >= 0.0 ? 1.0 : -1.0) * static_piv;
                c += (c >= 0.0 ? 1.0 : -1.0) * static_piv;
                det = a * c - s * s;
                R->n_static++;
            }
            double i00 = c / det, i01 = -s / det, i11 = a / det;
            R->pivot_start[j] = 1;
            R->pivot_start[j + 1] = 0;
            R->d_diag[j] = a;
            R->d_diag[j + 1] = c;
            R->d_off[j] = s;
            R->n_2x2++;
            int64_t m = 0;
            for (int64_t t = 0; t < W1.cnt; ++t) {
                int32_t r = W1.list[t];
                if (r > j + 1 && umark[r] != j) { umark[r] = j; ulist[m++] = r; }
            }
            for (int64_t t = 0; t < W2.cnt; ++t) {
                int32_t r = W2.list[t];
                if (r > j + 1 && umark[r] != j) { umark[r] = j; ulist[m++] = r; }
            }
            qsort(ulist, (size_t)m, sizeof(int32_t), cmp_i32);
            if (grow(R, 2 * m)) goto done;
            /* column j */
            for (int64_t t = 0; t < m; ++t) {
                int32_t r = ulist[t];
                double x0 = (W1.mark[r] == j) ? W1.w[r] : 0.0;
                double x1 = (W2.mark[r] == j + 1) ? W2.w[r] : 0.0;
                double l = x0 * i00 + x1 * i01;
                if (fabs(l) >= tau) { R->row[R->nnz] = r; R->val[R->nnz] = l; R->nnz++; }
            }
            R->colptr[j + 1] = R->nnz;
            for (int64_t t = 0; t < m; ++t) {
                int32_t r = ulist[t];
                double x0 = (W1.mark[r] == j) ? W1.w[r] : 0.0;
                double x1 = (W2.mark[r] == j + 1) ? W2.w[r] : 0.0;
                double l = x0 * i01 + x1 * i11;
                if (fabs(l) >= tau) { R->row[R->nnz] = r; R->val[R->nnz] = l; R->nnz++; }
            }
            R->colptr[j + 2] = R->nnz;
            link_new_column(&S, j);
            link_new_column(&S, j + 1);
            j += 2;
        }
    }
    R->colptr[n] = R->nnz;
    rc = 0;
done:
    free(S.ptr); free(S.head); free(S.next); free(S.blkmark);
    free(W1.w); free(W1.mark); free(W1.list);
    free(W2.w); free(W2.mark); free(W2.list);
    free(ulist); free(umark);
    return rc;
}

void ildl_free(ildl_result *R) {
    free(R->colptr); free(R->row); free(R->val);
    free(R->pivot_start); free(R->d_diag); free(R->d_off);
    memset(R, 0, sizeof(*R));
}

/* Solve (L D L^T) X = B in place for nrhs right-hand sides stored column after
 * column with leading dimension ldx.  L strictly lower CSC (unit diagonal). */
int ldl_solve(int64_t n, const int64_t *Lcp, const int32_t *Lr, const double *Lv,
              const int8_t *pivot_start, const double *d_diag, const double *d_off, double *X,
              int64_t nrhs, int64_t ldx) {
    for (int64_t c = 0; c < nrhs; ++c) {
        double *x = X + c * ldx;
        for (int64_t j = 0; j < n; ++j) {
            double xj = x[j];
            if (xj != 0.0)
                for (int64_t q = Lcp[j]; q < Lcp[j + 1]; ++q) x[Lr[q]] -= Lv[q] * xj;
        }
        for (int64_t j = 0; j < n;) {
            if (j + 1 < n && !pivot_start[j + 1]) {
                double a = d_diag[j], b = d_off[j], d = d_diag[j + 1];
                double det = a * d - b * b;
                double x0 = x[j], x1 = x[j + 1];
                x[j] = (d * x0 - b * x1) / det;
                x[j + 1] = (a * x1 - b * x0) / det;
                j += 2;
            } else {
                x[j] /= d_diag[j];
                j += 1;
            }
        }
        for (int64_t j = n - 1; j >= 0; --j) {
            double s = x[j];
            for (int64_t q = Lcp[j]; q < Lcp[j + 1]; ++q) s -= Lv[q] * x[Lr[q]];
            x[j] = s;
        }
    }
    return 0;
}
