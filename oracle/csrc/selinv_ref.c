/*
 * ORACLE (test infrastructure only: used by tests/, the smoke check and the CPU
 * baseline of the benchmark; never by the product path).
 *
 * Plain FP64 selected inversion by the scalar Takahashi recurrence at pivot-block
 * granularity, Section 2.1, Eqs. (4)-(5):
 *     G21 <- -G22 L21 ,   G11 <- D11^{-1} - L21^T G21 ,
 * processed from the last pivot block to the first, where block 1 is one pivot
 * block P of D (1x1 or 2x2) and block 2 is everything after it.  Section 2.1
 * restricts G21 to the pattern S and throws away whatever falls outside it:
 * here, when G22 is read its entries outside S count as zero, and X = G21 is
 * stored only where (r, p) is in S.
 *
 * Reading for a 2x2 block whose two columns have different row structure: X is
 * formed on the union U of both structures and G11 uses that unrestricted X, so
 * G11 stays symmetric; the discard happens only when X is stored.
 *
 * Storage: L strictly lower CSC with sorted rows (unit diagonal implied); the
 * result G is written in S_lo CSR order (row i: columns j <= i, sorted), the
 * same layout as the library output.  Entry lookup is a binary search in the
 * row of S_lo: slow and obviously correct.
 */
#include <stdint.h>
#include <stdlib.h>

static int64_t find_pos(const int64_t *Srp, const int32_t *Sc, int64_t r, int64_t c) {
    int64_t lo = Srp[r], hi = Srp[r + 1] - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        int32_t v = Sc[mid];
        if (v == c) return mid;
        if (v < c) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

static double g_read(const int64_t *Srp, const int32_t *Sc, const double *G, int64_t a, int64_t b) {
    int64_t r = a > b ? a : b, c = a > b ? b : a;
    int64_t p = find_pos(Srp, Sc, r, c);
    return p < 0 ? 0.0 : G[p];
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Per-block scratch of the recurrence: U (row set), mark (membership tags), Lu
 * and X (|U| x 2 panels).  One per thread in the level-set variant. */
typedef struct {
    int32_t *U;
    int64_t *mark;
    double *Lu, *X;
} block_scratch;

static int scratch_alloc(block_scratch *w, int64_t n) {
    w->U = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    w->mark = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    w->Lu = (double *)malloc(2 * ((size_t)n + 1) * sizeof(double));
    w->X = (double *)malloc(2 * ((size_t)n + 1) * sizeof(double));
    if (!w->U || !w->mark || !w->Lu || !w->X) return -1;
    for (int64_t i = 0; i <= n; ++i) w->mark[i] = -1;
    return 0;
}

static void scratch_free(block_scratch *w) {
    free(w->U); free(w->mark); free(w->Lu); free(w->X);
}

/* One step of the recurrence for the pivot block P = {b, ..., j} (1x1 or 2x2).
 * Returns 0, or -2 for a singular pivot block. */
static int selinv_block(int64_t b, int64_t j, const int64_t *Lcp, const int32_t *Lr, const double *Lv,
                        const double *d_diag, const double *d_off, const int64_t *Srp, const int32_t *Sc,
                        double *G, block_scratch *ws) {
    int32_t *U = ws->U;
    int64_t *mark = ws->mark;
    double *Lu = ws->Lu, *X = ws->X;
    int w = (int)(j - b + 1);
    /* U = union of the column structures of P, rows below the block */
    int64_t u = 0;
    for (int t = 0; t < w; ++t)
        for (int64_t q = Lcp[b + t]; q < Lcp[b + t + 1]; ++q) {
            int32_t r = Lr[q];
            if (r > j && mark[r] != b) { mark[r] = b; U[u++] = r; }
        }
    qsort(U, (size_t)u, sizeof(int32_t), cmp_i32);
    /* Lu[k][t] = L(U[k], b+t) (0 where not stored) */
    for (int64_t k = 0; k < u; ++k) { Lu[2 * k] = 0.0; Lu[2 * k + 1] = 0.0; }
    for (int t = 0; t < w; ++t) {
        int64_t k = 0;
        for (int64_t q = Lcp[b + t]; q < Lcp[b + t + 1]; ++q) {
            int32_t r = Lr[q];
            if (r <= j) continue;
            while (U[k] < r) ++k;
            Lu[2 * k + t] = Lv[q];
        }
    }
    /* X = -G~_UU Lu (G~ = G on S, 0 elsewhere) */
    for (int64_t k = 0; k < u; ++k) {
        double s0 = 0.0, s1 = 0.0;
        for (int64_t m = 0; m < u; ++m) {
            double g = g_read(Srp, Sc, G, U[k], U[m]);
            s0 += g * Lu[2 * m];
            s1 += g * Lu[2 * m + 1];
        }
        X[2 * k] = -s0;
        X[2 * k + 1] = -s1;
    }
    /* D_P^{-1} */
    double i00, i01, i11;
    if (w == 1) {
        if (d_diag[b] == 0.0) return -2;
        i00 = 1.0 / d_diag[b]; i01 = 0.0; i11 = 0.0;
    } else {
        double a = d_diag[b], c = d_off[b], d = d_diag[b + 1];
        double det = a * d - c * c;
        if (det == 0.0) return -2;
        i00 = d / det; i01 = -c / det; i11 = a / det;
    }
    /* G_PP = D_P^{-1} - Lu^T X */
    double g00 = i00, g10 = i01, g11 = i11;
    for (int64_t k = 0; k < u; ++k) {
        g00 -= Lu[2 * k] * X[2 * k];
        g10 -= Lu[2 * k + 1] * X[2 * k];
        g11 -= Lu[2 * k + 1] * X[2 * k + 1];
    }
    /* store X on S (r in struct(p)) and G_PP */
    for (int t = 0; t < w; ++t)
        for (int64_t q = Lcp[b + t]; q < Lcp[b + t + 1]; ++q) {
            int32_t r = Lr[q];
            if (r <= j) continue;
            int64_t lo = 0, hi = u - 1, k = -1;
            while (lo <= hi) {
                int64_t mid = lo + (hi - lo) / 2;
                if (U[mid] == r) { k = mid; break; }
                if (U[mid] < r) lo = mid + 1; else hi = mid - 1;
            }
            int64_t p = find_pos(Srp, Sc, r, b + t);
            if (p >= 0 && k >= 0) G[p] = X[2 * k + t];
        }
    G[find_pos(Srp, Sc, b, b)] = g00;
    if (w == 2) {
        G[find_pos(Srp, Sc, b + 1, b)] = g10;
        G[find_pos(Srp, Sc, b + 1, b + 1)] = g11;
    }
    return 0;
}

/* Returns 0 on success, -1 on allocation failure, -2 on a singular pivot block.
 * Processes the pivot blocks from the last one down to the block that starts at
 * or after stop_col (stop_col = 0: all of them); the entries of earlier blocks
 * are left untouched.  A partial run times a bounded sample of the recurrence. */
int oracle_selinv(int64_t n, const int64_t *Lcp, const int32_t *Lr, const double *Lv,
                  const int8_t *pivot_start, const double *d_diag, const double *d_off,
                  const int64_t *Srp, const int32_t *Sc, double *G, int64_t stop_col) {
    block_scratch ws;
    int rc = scratch_alloc(&ws, n);
    if (rc == 0) {
        int64_t j = n - 1;
        while (j >= 0) {
            /* pivot block P = {b} or {b, b+1} ending at j */
            int64_t b = pivot_start[j] ? j : j - 1;
            if (b < stop_col) break;
            rc = selinv_block(b, j, Lcp, Lr, Lv, d_diag, d_off, Srp, Sc, G, &ws);
            if (rc != 0) break;
            j = b - 1;
        }
    }
    scratch_free(&ws);
    return rc;
}

/* The same recurrence scheduled by level sets over all host threads (OpenMP):
 * the CPU baseline variant with every core busy.  The block of P reads G only
 * on C_P x C_P, whose entries the blocks owning the columns of C_P write, so
 *   level(P) = 0 if C_P is empty, else 1 + max level of the blocks owning C_P,
 * and the blocks of one level are independent: each writes only its own
 * columns.  Levels run in increasing order; every block does exactly the
 * arithmetic of oracle_selinv, so the results are identical to it.  Returns the
 * same codes; *nlevels receives the number of levels. */
int oracle_selinv_levels(int64_t n, const int64_t *Lcp, const int32_t *Lr, const double *Lv,
                         const int8_t *pivot_start, const double *d_diag, const double *d_off,
                         const int64_t *Srp, const int32_t *Sc, double *G, int64_t *nlevels) {
    int64_t *blk_of = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));   /* column -> block start */
    int64_t *level = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));    /* by block start */
    int64_t *order = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    int64_t *lstart = NULL;
    int rc = 0;
    if (!blk_of || !level || !order) { rc = -1; goto out; }
    for (int64_t c = 0; c < n; ++c) blk_of[c] = (pivot_start[c] || c == 0) ? c : c - 1;
    int64_t maxlev = -1, nblk = 0;
    for (int64_t j = n - 1; j >= 0;) {
        int64_t b = pivot_start[j] ? j : j - 1;
        int64_t lv = 0;
        for (int64_t t = b; t <= j; ++t)
            for (int64_t q = Lcp[t]; q < Lcp[t + 1]; ++q) {
                int64_t r = Lr[q];
                if (r > j && level[blk_of[r]] + 1 > lv) lv = level[blk_of[r]] + 1;
            }
        level[b] = lv;
        if (lv > maxlev) maxlev = lv;
        ++nblk;
        j = b - 1;
    }
    /* blocks grouped by level (counting sort), each group in decreasing start order */
    lstart = (int64_t *)calloc((size_t)maxlev + 2, sizeof(int64_t));
    if (!lstart) { rc = -1; goto out; }
    for (int64_t j = n - 1; j >= 0;) {
        int64_t b = pivot_start[j] ? j : j - 1;
        ++lstart[level[b] + 1];
        j = b - 1;
    }
    for (int64_t l = 0; l <= maxlev; ++l) lstart[l + 1] += lstart[l];
    {
        int64_t *fill = (int64_t *)malloc(((size_t)maxlev + 1) * sizeof(int64_t));
        if (!fill) { rc = -1; goto out; }
        for (int64_t l = 0; l <= maxlev; ++l) fill[l] = lstart[l];
        for (int64_t j = n - 1; j >= 0;) {
            int64_t b = pivot_start[j] ? j : j - 1;
            order[fill[level[b]]++] = b;
            j = b - 1;
        }
        free(fill);
    }
    *nlevels = maxlev + 1;
    {
        int err = 0;
#pragma omp parallel
        {
            block_scratch ws;
            int own = scratch_alloc(&ws, n);
            if (own != 0) {
#pragma omp atomic write
                err = -1;
            }
            for (int64_t l = 0; l <= maxlev; ++l) {
                /* every thread runs every level loop; the implicit barrier of the
                   worksharing loop separates the levels */
#pragma omp for schedule(dynamic, 1)
                for (int64_t e = lstart[l]; e < lstart[l + 1]; ++e) {
                    int cur;
#pragma omp atomic read
                    cur = err;
                    if (own != 0 || cur != 0) continue;
                    int64_t b = order[e];
                    int64_t j = (b + 1 < n && !pivot_start[b + 1]) ? b + 1 : b;
                    int r = selinv_block(b, j, Lcp, Lr, Lv, d_diag, d_off, Srp, Sc, G, &ws);
                    if (r != 0) {
#pragma omp atomic write
                        err = r;
                    }
                }
            }
            scratch_free(&ws);
        }
        rc = err;
    }
    (void)nblk;
out:
    free(blk_of); free(level); free(order); free(lstart);
    return rc;
}

/* The recurrence on a given list of pivot blocks, in the order listed (each block
 * by its first column), reading and writing G in place: the blocks whose G entries
 * a listed block reads must already be in G.  Used to check a partition of the
 * recurrence (some blocks computed elsewhere and copied into G first).  Returns 0,
 * -1 (allocation) or -2 (singular pivot block). */
int oracle_selinv_blocks(int64_t n, const int64_t *Lcp, const int32_t *Lr, const double *Lv,
                         const int8_t *pivot_start, const double *d_diag, const double *d_off,
                         const int64_t *Srp, const int32_t *Sc, double *G, const int64_t *blocks, int64_t nblocks) {
    block_scratch ws;
    int rc = scratch_alloc(&ws, n);
    for (int64_t e = 0; e < nblocks && rc == 0; ++e) {
        int64_t b = blocks[e];
        int64_t j = (b + 1 < n && !pivot_start[b + 1]) ? b + 1 : b;
        rc = selinv_block(b, j, Lcp, Lr, Lv, d_diag, d_off, Srp, Sc, G, &ws);
    }
    scratch_free(&ws);
    return rc;
}
