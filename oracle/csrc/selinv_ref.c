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

/* Returns 0 on success, -1 on allocation failure, -2 on a singular pivot block.
 * Processes the pivot blocks from the last one down to the block that starts at
 * or after stop_col (stop_col = 0: all of them); the entries of earlier blocks
 * are left untouched.  A partial run times a bounded sample of the recurrence. */
int oracle_selinv(int64_t n, const int64_t *Lcp, const int32_t *Lr, const double *Lv,
                  const int8_t *pivot_start, const double *d_diag, const double *d_off,
                  const int64_t *Srp, const int32_t *Sc, double *G, int64_t stop_col) {
    int32_t *U = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    int64_t *mark = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    double *Lu = (double *)malloc(2 * ((size_t)n + 1) * sizeof(double));
    double *X = (double *)malloc(2 * ((size_t)n + 1) * sizeof(double));
    int rc = 0;
    if (!U || !mark || !Lu || !X) { rc = -1; goto out; }
    for (int64_t i = 0; i <= n; ++i) mark[i] = -1;
    int64_t j = n - 1;
    while (j >= 0) {
        /* pivot block P = {b} or {b, b+1} ending at j */
        int64_t b = pivot_start[j] ? j : j - 1;
        if (b < stop_col) break;
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
            if (d_diag[b] == 0.0) { rc = -2; goto out; }
            i00 = 1.0 / d_diag[b]; i01 = 0.0; i11 = 0.0;
        } else {
            double a = d_diag[b], c = d_off[b], d = d_diag[b + 1];
            double det = a * d - c * c;
            if (det == 0.0) { rc = -2; goto out; }
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
        j = b - 1;
    }
out:
    free(U); free(mark); free(Lu); free(X);
    return rc;
}
