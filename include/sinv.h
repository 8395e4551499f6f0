/*
 * libsinv -- selected inverse of a sparse symmetric matrix on S = pattern(L+D+L^T)
 * from given incomplete LDL^T factors, on one NVIDIA B300 (sm_103a).
 *
 * Method: Akter, Bollhoefer, Schenk, "Scalable Approximate Selected Inversion
 * Based on Single-Level Incomplete LDL^T Factorization and Spectral Corrections
 * for Large Sparse Systems".  Section numbers below refer to that paper.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - n is the matrix order; indices are 0-based.  Column indices are int32,
 *    row pointers int64.
 *  - L is strictly lower triangular CSR (unit diagonal implied, not stored):
 *    row i holds the columns j < i of its stored entries, strictly increasing.
 *    A stored entry is structurally nonzero even when its value is 0.
 *  - D is block diagonal with 1x1 and 2x2 blocks.  pivot_start[j] = 1 when a
 *    block starts at j; the block is 2x2 iff pivot_start[j+1] = 0.  Packed
 *    values D_val list the blocks in order: d for a 1x1 block, (d11, d21, d22)
 *    for a 2x2 block, so D_val has n + (#2x2 blocks) entries.  The two columns
 *    of a 2x2 block are coupled only through D: L(j+1, j) must not be stored.
 *  - S_lo is the lower part of S (Section 1): row i holds the stored columns of
 *    L row i, then i-1 if (i-1, i) is a 2x2 block, then i.  Every value array
 *    "on S" (G_S, N_S, M_S, X_S) has |S_lo| entries in this CSR order.
 *  - Numeric calls take DEVICE pointers, are asynchronous on the given stream,
 *    and keep no pointer after their stream work completes.  The caller owns
 *    every buffer it passes; the handle owns everything it allocates.  Every
 *    pointer and the stream belong to the handle's device (the `device` of
 *    sinv_symbolic_opts); the call makes that device current itself.
 *  - Every call returns a status and never aborts or throws across the ABI.
 *    Errors found on the device (a singular pivot, a wait that timed out) are
 *    recorded in a handle-owned status word and returned (and cleared) by
 *    the next sinv_sync_status, which synchronises with the stream.  The
 *    handle is not thread safe: one host thread drives it at a time.
 */
#ifndef SINV_H
#define SINV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SINV_OK = 0,
    SINV_ERR_INVALID_ARG = 1,   /* null pointer, negative size, bad enum      */
    SINV_ERR_PATTERN = 2,       /* unsorted / duplicate / out-of-range / not
                                   strictly lower / bad pivot layout          */
    SINV_ERR_SINGULAR_PIVOT = 3,/* a D block with zero determinant            */
    SINV_ERR_OOM = 4,           /* host or device allocation failed           */
    SINV_ERR_CUDA = 5,          /* a CUDA runtime call failed                 */
    SINV_ERR_TIMEOUT = 6,       /* a bounded device wait gave up              */
    SINV_ERR_UNSUPPORTED = 7    /* size or option outside what is built       */
} sinv_status;

/* Arithmetic of a numeric call.  Inputs and outputs stay FP64 in every form. */
typedef enum {
    SINV_FP64 = 0,      /* native FP64 throughout                                  */
    SINV_FP32 = 1,      /* FP32 products and sums; pivot inverses and the diagonal
                           accumulation of each pivot block in FP64                */
    SINV_FP32X2 = 2,    /* FP64-class results with the NInv product on S run on the
                           FP32 pipes: every FP64 operand is split into an FP32
                           high part and an FP32 low part, a product keeps the
                           high-by-high product exactly plus both cross terms, and
                           sums carry their rounding error (error-free two-sum).
                           The other steps, whose sums go through shared-memory
                           atomics or wait on a dependency chain, run FP64 (so
                           sinv_selinv and sinv_lowrank_correct treat it as
                           SINV_FP64, and so does NInv when it runs in hash form).
                           Values of W or D^{-1}W at or above 2^100 in magnitude
                           are reported as SINV_ERR_UNSUPPORTED by the next
                           sinv_sync_status.                                       */
    SINV_TF32_FP32ACC = 3,  /* sinv_selinv only (Section 2.1, Eqs. (4)-(5)): the
                           supernodes of the leading levels whose row set C is a
                           contiguous range of rows run on the tensor cores
                           (tcgen05): G~_CC L_CJ with every operand split into a
                           TF32 high and a TF32 low part, the high-by-high
                           products and the cross terms in two FP32 accumulators
                           added in FP64; L_JJ^{-1}, the pivot inverses, the sum
                           of L_CJ^T G~ L_CJ over C and G_JJ in FP64.  The other
                           supernodes run SINV_FP64.  Stated error: normwise
                           1e-6 against the FP64 oracle.  Other calls return
                           SINV_ERR_UNSUPPORTED (no dense contraction there).   */
    SINV_BF16_FP32ACC = 4   /* the same with BF16 high and low parts; stated error:
                           normwise 1e-5.                                          */
} sinv_precision;

typedef struct sinv_handle_s *sinv_handle;

typedef struct {
    int32_t supernode_cap;  /* max columns per supernode (1 disables merging); 0 = 4  */
    int32_t device;         /* CUDA device ordinal the handle lives on; -1 = host-only
                               analysis (no CUDA call; numeric calls then fail with
                               SINV_ERR_INVALID_ARG)                                  */
    int64_t wait_limit;     /* polls before a device wait gives up; 0 = default       */
    int64_t big_pairs;      /* supernodes with at least this many entries of S in
                               C x C are processed by a whole CTA; 0 = default 1024   */
    int64_t ninv_index_bytes; /* device memory the map form of NInv may hold (the
                               positions of every product in the series pattern,
                               built by the first sinv_ninv of an m): 0 = half of
                               the free memory at that time, > 0 = this many bytes,
                               < 0 = never.  Without maps (also when a column of the
                               pattern is too long for them) the hash form runs:
                               same results, slower                                  */
    int64_t selinv_pair_bytes; /* memory the SelInv pair lists may take (8 B for every
                               pair of C_J x C_J in S, over all supernodes J): 0 = 8 GB,
                               > 0 = this many bytes, < 0 = none.  Past it the scan
                               form runs: every supernode reads G~_CC by scanning its
                               rows of S_lo from the diagonal down to the first row of
                               C_J, looking each column up in a hash table of C_J.
                               Same arithmetic per pair; the plan then holds O(nnz L). */
} sinv_symbolic_opts;

/* Symbolic analysis (host).  Validates the pattern of L and the pivot layout,
 * builds S_lo, the pivot blocks, the supernode partition, the dependency levels
 * and every index map the numeric calls use, and uploads them to the device.
 *   L_rowptr [n+1], L_col [nnzL], pivot_start [n]: HOST memory, read only.
 *   opts may be NULL (defaults).  *out receives a new handle (destroy with
 *   sinv_destroy).  Pattern of S: Section 1; the supernodal ordering of the
 *   Takahashi recurrence: Section 2.1 and Fig. 2 (block elimination tree). */
sinv_status sinv_symbolic(int64_t n, const int64_t *L_rowptr, const int32_t *L_col,
                          const int8_t *pivot_start, const sinv_symbolic_opts *opts,
                          sinv_handle *out);

/* Batched analysis: nmat matrices (sizes n[b], each with its own L pattern and
 * pivot layout, HOST arrays) analysed as one block-diagonal matrix.  Every numeric
 * call then processes all matrices together: one persistent SelInv launch runs the
 * supernodes of all matrices in one level-major schedule (matrices of uneven size
 * fill each other's idle levels), and each NInv step is one launch over all
 * columns.  Value arrays are the concatenations of the per-matrix arrays in matrix
 * order (L_val, D_val, and every array on S); sinv_batch_layout gives the offsets.
 * An entry of matrix b must lie inside its own block (SINV_ERR_PATTERN otherwise).
 * This is the batching of many independent problems; the paper solves one matrix
 * at a time. */
sinv_status sinv_batch_symbolic(int32_t nmat, const int64_t *n, const int64_t *const *L_rowptr,
                                const int32_t *const *L_col, const int8_t *const *pivot_start,
                                const sinv_symbolic_opts *opts, sinv_handle *out);
/* nmat (0 for a handle from sinv_symbolic) and, for arrays that are not NULL,
 * nmat+1 offsets of each matrix's rows, L entries, packed D values and S_lo entries. */
sinv_status sinv_batch_layout(sinv_handle h, int32_t *nmat, int64_t *n_off, int64_t *L_off, int64_t *D_off,
                              int64_t *S_off);

/* One call over all matrices of a batch handle, with every matrix in its own
 * buffers: the persistent, graph-capturable batched run of Section 2.1 (SelInv)
 * and Section 2.2 (NInv) over many matrices of uneven size.  The matrices'
 * L and D values are gathered into the handle's concatenated layout (one
 * launch each), SelInv runs as one persistent launch over the supernodes of all
 * matrices (level by level), NInv as one set of launches, and the results are
 * scattered back (one launch each).  Every step is a kernel launch on `stream`;
 * the per-matrix pointers travel as kernel arguments, so the whole call can be
 * captured in a CUDA graph and replayed.
 *   h: from sinv_batch_symbolic with nmat matrices.  L_vals[b], D_vals[b]: host
 *   arrays of nmat device pointers to matrix b's own L values (CSR order) and
 *   packed D.  G_outs: host array of nmat device pointers (|S_lo| of matrix b,
 *   S_lo order), or NULL to skip SelInv; an entry may be NULL to skip that
 *   matrix's copy.  m, N_outs: NInv with m terms into N_outs the same way, or
 *   N_outs NULL to skip it.  prec as for sinv_selinv (the tensor-core forms
 *   apply to SelInv only; NInv then returns SINV_ERR_UNSUPPORTED).
 *   The first call allocates the concatenated buffers (|L| + |D| + 2 |S_lo|
 *   doubles, handle-owned): make it before any stream capture.
 *   Errors: SINV_ERR_INVALID_ARG (not a batch handle, nmat mismatch, missing
 *   pointers), SINV_ERR_OOM, and those of sinv_selinv / sinv_ninv. */
sinv_status sinv_batch_run(sinv_handle h, int32_t nmat, const double *const *L_vals, const double *const *D_vals,
                           sinv_precision prec, double *const *G_outs, int m, double *const *N_outs, void *stream);

/* S_lo on the device (handle-owned, valid until sinv_destroy) and its size. */
sinv_status sinv_get_pattern(sinv_handle h, const int64_t **S_rowptr, const int32_t **S_col,
                             int64_t *nnzS_lo);

/* Copies S_lo into caller-owned HOST arrays S_rowptr [n+1] and S_col [|S_lo|]. */
sinv_status sinv_get_pattern_host(sinv_handle h, int64_t *S_rowptr, int32_t *S_col);

/* Selected inverse on S (Section 2.1, Eqs. (4)-(5)): for every pivot block
 * from the last to the first, G21 = -G22 L21 restricted to S (entries of G22
 * outside S read as zero), G11 = D11^{-1} - L21^T G21.  Supernodes of
 * consecutive pivot blocks with nested structure are processed as one dense
 * step; supernodes are scheduled by a persistent kernel in dependency order.
 *   L_val [nnzL] (CSR order of L), D_val (packed), G_S [|S_lo|]: device.
 * Singular D blocks: SINV_ERR_SINGULAR_PIVOT (reported by sinv_sync_status). */
sinv_status sinv_selinv(sinv_handle h, const double *L_val, const double *D_val,
                        sinv_precision prec, double *G_S, void *stream);

/* NInv on S (Section 2.2, Eqs. (6) and (8)): W = sum_{t=0}^{m} E^t with
 * L = I - E, by m Horner steps W <- I + E W on the fixed pattern of the
 * truncated series, then N = W^T D^{-1} W evaluated on S only.  0 <= m <= 30.
 *   L_val, D_val, N_S [|S_lo|]: device.  m > 30: SINV_ERR_UNSUPPORTED.
 * The first call for an m builds that pattern (host) and its position maps
 * (device, see sinv_symbolic_opts.ninv_index_bytes) and synchronises the
 * stream; later calls with the same m only launch kernels (make the first one
 * before capturing a stream into a CUDA graph).  In the map form the FP64 and
 * SINV_FP32X2 results repeat bit for bit (the Horner steps sum in exact fixed
 * point); the FP32 form and the hash form sum with floating-point atomics, so
 * their repeated calls agree to rounding. */
sinv_status sinv_ninv(sinv_handle h, const double *L_val, const double *D_val, int m,
                      sinv_precision prec, double *N_S, void *stream);

/* NInv with the inverse tolerance delta sparsifying the series (Section 2.2:
 * larger delta, sparser L^inv): the Horner steps run in column form,
 * W <- I + W E (column j of W from the columns k of struct(j)), and after every
 * step the off-diagonal entries of W with |w| < delta are set to zero; the product
 * W^T D^{-1} W is then evaluated exactly on S, as in sinv_ninv.  delta = 0 is
 * sinv_ninv.  The kernels keep the structural pattern of the full series, so a
 * larger delta changes the values, not the work.  delta < 0 or NaN:
 * SINV_ERR_INVALID_ARG.  Everything else as sinv_ninv. */
sinv_status sinv_ninv_drop(sinv_handle h, const double *L_val, const double *D_val, int m, double delta,
                           sinv_precision prec, double *N_S, void *stream);

/* NInv on S for every truncation t = 0..m of the series at once (Eq. (6) cut after
 * t terms, then Eq. (8)): N_stack[t * |S_lo| + e] (device, (m+1) x |S_lo| doubles).
 * The last slice equals sinv_ninv(m); t = 0 gives D^{-1} on S.  The per-order
 * differences are inputs of the learned correction. */
sinv_status sinv_ninv_stack(sinv_handle h, const double *L_val, const double *D_val, int m,
                            sinv_precision prec, double *N_stack, void *stream);

/* NInv on its own pattern (Section 2.2, Eqs. (6) and (8)): the inverse
 * tolerance delta sparsifies both W = L^inv and the product W^T D^{-1} W, so
 * the result is a sparse approximate inverse whose pattern depends only on the
 * sizes of the entries (not on S).  W is built by the m Horner steps of
 * sinv_ninv_drop (off-diagonal |w| < delta dropped after every step), each
 * step's survivors appended per column (no structural pattern of the series is
 * built: a step whose output passes its first size guess is rerun into a
 * buffer of the size it counted), so the next step only streams the
 * survivors; the product is
 * formed by columns through the rows of W and keeps the diagonal and the
 * entries with |N_ij| >= delta sqrt(|N_ii N_jj|) (the reading of "delta
 * controls the sparsity of the product").  The result is the lower triangle
 * N_lo in CSC (column j: rows i >= j, in no particular order), kept by the
 * handle until the next call: sinv_ninv_own_size gives its size and the size
 * of W after every step (nnz_W_steps[t], t = 0..m), sinv_ninv_own_copy copies
 * it into caller-owned device buffers (colptr n+1, rows and values nnz).
 * Synchronous on `stream` (sizes are read back after every step).
 * delta = 0 keeps every structural entry (the product's pattern then grows
 * like (L^{-1})^T L^{-1}).  For n = 0 the result is empty (colptr {0}, every
 * nnz_W_steps[t] = 0) and L_val, D_val may be NULL.  Errors: SINV_ERR_INVALID_ARG (m < 0, delta < 0,
 * NaN), SINV_ERR_UNSUPPORTED (m > 30), SINV_ERR_OOM (device memory for the
 * series, its hash tables or the product), SINV_ERR_CUDA. */
sinv_status sinv_ninv_own(sinv_handle h, const double *L_val, const double *D_val, int m, double delta,
                          void *stream);
sinv_status sinv_ninv_own_size(sinv_handle h, int64_t *nnz_N_lo, int64_t *nnz_W_steps, int32_t max_steps);
sinv_status sinv_ninv_own_copy(sinv_handle h, int64_t *N_colptr, int32_t *N_row, double *N_val, void *stream);

/* Mix on NInv's own pattern (Section 2.3): with S_eps = {(i, j) in S_lo : |G_ij| >
 * eps}, the result is G on S_eps and the last sinv_ninv_own result N elsewhere on
 * N's pattern, so its pattern is the union of N's and S_eps (lower triangle, CSC,
 * rows of a column in no particular order: N's rows first, then the rows of S_eps
 * that N lacks).  The paper computes N for Mix with a loose inverse tolerance
 * (delta = 1e-1), so the result has about NInv's fill and SelInv's large entries.
 *   G_S [|S_lo|]: device, SelInv on S_lo (S_lo CSR order).  eps: any value but NaN
 *   (+inf gives N, a negative value all of S).  Synchronous on `stream` (the result
 *   is sized on the host); the result is handle-owned until the next call:
 *   sinv_mix_own_size gives its number of entries, sinv_mix_own_copy copies it to
 *   caller-owned device arrays (n+1 column pointers, then rows and values).
 *   G_S may be NULL when S is empty (n = 0; the result is then empty).
 *   Errors: SINV_ERR_INVALID_ARG (no sinv_ninv_own result, null G_S, NaN eps),
 *   SINV_ERR_OOM, SINV_ERR_CUDA. */
sinv_status sinv_mix_own(sinv_handle h, const double *G_S, double eps, void *stream);
sinv_status sinv_mix_own_size(sinv_handle h, int64_t *nnz);
sinv_status sinv_mix_own_copy(sinv_handle h, int64_t *M_colptr, int32_t *M_row, double *M_val, void *stream);
/* The rank-k correction of Eq. (9) added in place to the handle-owned result of
 * sinv_mix_own: M_ij += sum_l lambda_l V_il V_jl on its pattern.  Arguments, forms
 * and limits as for sinv_lowrank_correct (V [n x k] row-major and lambda [k] on
 * the device, 0 <= k <= 256, SINV_FP64 or SINV_FP32).
 *   Errors: SINV_ERR_INVALID_ARG (no sinv_mix_own result, bad arguments),
 *   SINV_ERR_UNSUPPORTED (k > 256, tensor-core forms), SINV_ERR_OOM, SINV_ERR_CUDA. */
sinv_status sinv_lowrank_correct_mix_own(sinv_handle h, int k, const double *V, const double *lambda,
                                         sinv_precision prec, void *stream);

/* Mix-SPAI on the Mix pattern (Section 2.4: the refinement keeps the pattern of
 * the Mix built on NInv's loose-tolerance pattern).  sinv_spai_analyse_mix_own
 * replaces the handle's SPAI plan by one on the pattern of the current
 * sinv_mix_own result (read back to the host; A as for sinv_spai_analyse, HOST
 * arrays), and sinv_spai_mix_own runs the refinement, writing Y_P [|P_lo|]
 * (device) in the order of sinv_spai_pattern.  X_M: start values on the Mix
 * pattern in the order of sinv_mix_own_copy (device), or NULL for the handle's
 * current Mix values.  Other arguments and errors as for sinv_spai_analyse /
 * sinv_spai; sinv_spai_mix_own also returns SINV_ERR_INVALID_ARG when the plan was
 * not built from the current Mix result. */
sinv_status sinv_spai_analyse_mix_own(sinv_handle h, int64_t nnzA, const int64_t *A_rowptr, const int32_t *A_col,
                                      int warp_entries);
sinv_status sinv_spai_mix_own(sinv_handle h, const double *A_val, const double *X_M, int iters, double *Y_P,
                              void *stream);

/* Mix (Section 2.3): M_ij = G_ij where |G_ij| > eps, else N_ij, on S.
 *   G_S, N_S, M_S [|S_lo|]: device (M_S may alias G_S or N_S). */
sinv_status sinv_mix(sinv_handle h, const double *G_S, const double *N_S, double eps,
                     double *M_S, void *stream);

/* Low-rank spectral correction on S (Section 2.5, Eq. (9); its diagonal is
 * the update formula of Section 2.6): X_ij += sum_{l<k} lambda_l V_il V_jl for
 * (i, j) in S_lo.
 *   V [n*k] row-major, lambda [k], X_S [|S_lo|] in/out: device.  k <= 256. */
sinv_status sinv_lowrank_correct(sinv_handle h, int k, const double *V, const double *lambda,
                                 sinv_precision prec, double *X_S, void *stream);

/* SPAI refinement on a fixed pattern P (Section 2.4; Mix-SPAI is this step
 * applied to the Mix values).  P is S, or S widened to every (i, j) whose
 * distance in the graph of A is at most `power` (a larger candidate pattern,
 * which the least-squares fit needs to beat the start values: see the
 * documentation).  For every column j, with J_j = {i : (i, j) in P}, `iters`
 * steps of Jacobi-preconditioned conjugate gradients on the normal equations
 * (A_J^T A_J) m = A_J^T e_j  of  min ||A m - e_j||_2  over m supported on J_j,
 * started from X on S and zero on the rest of P; then Y = (M + M^T) / 2 on P_lo.
 * A column stops early only when its preconditioned residual r.z is exactly
 * zero or the curvature p.Bp is not positive.  FP64 throughout.
 *
 * sinv_spai_analyse: the pattern of A, HOST arrays, n x n CSR with
 *   A_rowptr[n+1] (starts at 0, ends at nnzA) and A_col[nnzA]; rows need not be
 *   sorted; no duplicates; structurally symmetric.  power >= 0 (0: P = S; at
 *   most 8).  Builds P, the column lists of P, the entry offsets and the two
 *   work tiers (a warp per column in shared memory, a CTA per column with a
 *   global scratch block) and uploads them; it synchronises the device.  On a
 *   host-only handle it builds the plan and the pattern only.  A new analysis
 *   replaces the previous one.
 *   warp_entries: the most entries of A a column may stage to be solved by a warp
 *   (0 = the default and maximum, 704; a column also needs |J_j| <= 128 and at
 *   most 256 distinct rows of A); smaller values move columns to the CTA tier.
 *   Errors: SINV_ERR_INVALID_ARG (power < 0, warp_entries < 0), SINV_ERR_PATTERN
 *   (range, order of rowptr, duplicates, asymmetry), SINV_ERR_UNSUPPORTED
 *   (power > 8, nnzA or |P_lo| >= 2^31, a column staging >= 2^30 entries),
 *   SINV_ERR_OOM.
 * sinv_spai_pattern: copies P_lo (CSR, rows sorted, the diagonal last) into
 *   host arrays P_rowptr[n+1] and P_col[spai_nnz_P of sinv_get_stats].
 * sinv_spai: A_val[nnzA] (device, in the order of the analysed A_col; A must be
 *   symmetric: row k is read as column k), X_S [|S_lo|] and Y_P [|P_lo|]
 *   (device, must not overlap; X symmetric by construction, given by its lower
 *   part).  Stream ordered, no allocation, no synchronisation, graph-capturable.
 *   Y is not bit-reproducible (the order of the entries inside a row of the
 *   products comes from a counting sort with atomics).
 *   Errors: SINV_ERR_INVALID_ARG (no analysis on the device, iters < 0,
 *   X_S == Y_P). */
sinv_status sinv_spai_analyse(sinv_handle h, int64_t nnzA, const int64_t *A_rowptr, const int32_t *A_col,
                              int power, int warp_entries);
sinv_status sinv_spai_pattern(sinv_handle h, int64_t *P_rowptr, int32_t *P_col);
sinv_status sinv_spai(sinv_handle h, const double *A_val, const double *X_S, int iters, double *Y_P,
                      void *stream);

/* Spectral-correction producer (Section 2.5, Algorithm 1 step 5): the k
 * dominant eigenpairs (largest |lambda|) of E_inv = A^{-1} - A^inv by Lanczos
 * with full reorthogonalisation (classical Gram-Schmidt, twice) from the start
 * vector q0.  Each step applies E_inv: A^{-1} q by conjugate gradients from 0,
 * preconditioned with the ILDL factors (z = L^{-T} D^{-1} L^{-1} r), stopped
 * at ||r|| <= cg_tol ||q|| or after cg_maxit iterations; A^inv q is X applied
 * as the symmetric matrix given by its lower part on S.  Lanczos stops early
 * when beta < 1e-14 max(1, |alpha|).  The Ritz pairs come from the tridiagonal
 * matrix by cyclic Jacobi.  FP64 throughout.  A must be symmetric positive
 * definite for the CG solves (indefinite A: a CG breakdown ends that solve
 * early and counts in info[2]).
 *
 * sinv_einv_analyse: the pattern of A, HOST arrays (the same rules as
 *   sinv_spai_analyse).  Builds the columns of S and the dependency levels of
 *   the two triangular solves, uploads them, synchronises the device (on a
 *   host-only handle: the plan only).
 *   Errors: SINV_ERR_PATTERN, SINV_ERR_UNSUPPORTED (nnzA >= 2^31), SINV_ERR_OOM.
 * sinv_einv_lanczos: A_val[nnzA], L_val, D_val (as for sinv_selinv), X_S
 *   [|S_lo|], q0 [n]: device.  lambda [k]: HOST, the Ritz values, largest |.|
 *   first; V [n*k] row-major: device, the Ritz vectors (unit norm).  info [3]:
 *   HOST, (Lanczos steps taken m, total CG iterations, solves that stopped
 *   before cg_tol).  If m < k, the last k - m values and columns are 0.
 *   Synchronous on `stream` (every step reads its scalars on the host).
 *   1 <= k <= steps <= min(n, 256), cg_tol > 0, cg_maxit >= 1.
 *   Errors: SINV_ERR_INVALID_ARG (no analysis, bad sizes, q0 zero or not
 *   finite), SINV_ERR_UNSUPPORTED (steps > 256), SINV_ERR_OOM. */
sinv_status sinv_einv_analyse(sinv_handle h, int64_t nnzA, const int64_t *A_rowptr, const int32_t *A_col);
/* The inner solver of sinv_einv_lanczos for A^{-1} q (Section 2.5 solves these
 * with ILDL-preconditioned Krylov methods, sQMR for indefinite A):
 *   0 (default): conjugate gradients with M = L D L^T -- needs A and D positive
 *     definite;
 *   1: MINRES (Paige & Saunders) with the SPD preconditioner M = L |D| L^T, |D|
 *     the absolute value of every 1x1 / 2x2 pivot block -- for indefinite A.
 * Both apply M^{-1} with two triangular solves over the dependency levels:
 * one CTA walking the levels with a barrier between them when they hold fewer
 * than 64 rows on average, else a persistent grid with per-row flags (one
 * launch each); adding 2 to `solver` forces the persistent grid.  cg_tol of
 * sinv_einv_lanczos is then the relative residual in the norm of M^{-1} that
 * MINRES estimates, and cg_maxit its iteration limit.  Errors:
 * SINV_ERR_INVALID_ARG (unknown solver). */
sinv_status sinv_einv_set_solver(sinv_handle h, int32_t solver);
sinv_status sinv_einv_lanczos(sinv_handle h, const double *A_val, const double *L_val, const double *D_val,
                              const double *X_S, const double *q0, int steps, double cg_tol, int cg_maxit, int k,
                              double *lambda, double *V, int32_t *info, void *stream);

/* The FP32 form of sinv_lowrank_correct for callers that cannot allocate device
 * memory -- for instance code that gets all of its device memory from an
 * arena it owns, or that must not call cudaMalloc because it may synchronise
 * the device.  It needs no handle and allocates nothing: the FP32 working copy
 * of V and lambda lives in a 16 MiB array inside the library (reserved on
 * every GPU that loads the library until the process exits).  The paper has
 * no counterpart; this is a deployment variant of the correction above.
 *   S_rowptr [n+1], S_col [|S_lo|]: the pattern S_lo on the device (for example
 *   from sinv_get_pattern); V [n*k] row-major, lambda [k], X_S in/out: device.
 *   Limits: 1 <= k <= 256 (lambda .* V_i is staged in a 256-entry shared row)
 *   and n*k + k <= 4,194,304 (the array's size).  All pointers must belong to
 *   the current device.  The first call on a device looks up the array's
 *   device address; make that first call before any stream capture.  All
 *   calls on a device share the array: calls that overlap on the GPU (other
 *   streams, other threads) race, so order them on one stream.
 *   Returns: SINV_OK (also for n == 0 or k == 0, with nothing launched);
 *   SINV_ERR_INVALID_ARG for n < 0, k < 0 or a null pointer;
 *   SINV_ERR_UNSUPPORTED for k > 256 or n*k + k > 4,194,304 (checked before
 *   anything else is read, nothing is launched); SINV_ERR_CUDA when the device
 *   lookup or a launch fails. */
sinv_status sinv_lowrank_correct_noalloc(int64_t n, const int64_t *S_rowptr, const int32_t *S_col, int k,
                                         const double *V, const double *lambda, double *X_S, void *stream);

/* Learned correction from NInv towards SelInv (not in the paper: a proposed
 * addition).  A ReLU network 16 -> 64 -> 64 -> 1 maps features of an entry (i, j)
 * of S to a correction: N^_ij = N_ij + s_ij f(x_ij), s_ij = sqrt|N_ii N_jj|.  It is
 * trained on pairs the method itself produces (target (SelInv_ij - N_ij) / s_ij),
 * with BF16 weights and features, FP32 sums and Adam, by the library's own
 * forward, backward and optimiser kernels.  SelInv stays the reference: callers keep
 * the correction only where it lowers the error on held-out matrices.
 * Parameter vector (FP32, sinv_mlp_param_count() entries): W1[16x64], b1[64],
 * W2[64x64], b2[64], W3[64], b3. */
typedef struct sinv_mlp_s *sinv_mlp;
int32_t sinv_mlp_param_count(void);
/* Network on `device` with seeded He-uniform weights; max_batch bounds the
 * mini-batch of sinv_mlp_grad / sinv_mlp_train_step. */
sinv_status sinv_mlp_create(int32_t device, uint64_t seed, int64_t max_batch, sinv_mlp *out);
void sinv_mlp_destroy(sinv_mlp m);
/* Host copies of the FP32 master weights; set also resets the Adam state. */
sinv_status sinv_mlp_get_params(sinv_mlp m, float *theta);
sinv_status sinv_mlp_set_params(sinv_mlp m, const float *theta);
/* The whole training state, for a checkpoint: the FP32 weights, Adam's two moment
 * vectors (host arrays of sinv_mlp_param_count() floats each) and the number of
 * Adam steps taken.  Both calls first wait for the device's queued work.  After
 * sinv_mlp_set_state training continues exactly as it would have from the saved
 * network (the same inputs give the same weights bit for bit).
 *   Errors: SINV_ERR_INVALID_ARG (a NULL pointer, step < 0 or >= 2^31),
 *   SINV_ERR_CUDA. */
sinv_status sinv_mlp_get_state(sinv_mlp m, float *theta, float *mom1, float *mom2, int64_t *step);
sinv_status sinv_mlp_set_state(sinv_mlp m, const float *theta, const float *mom1, const float *mom2,
                               int64_t step);
/* Features of every S_lo entry from the NInv stack of sinv_ninv_stack (m <= 9):
 * X [|S_lo| x 16] BF16, scale [|S_lo|] FP32 (s_ij); all device. */
sinv_status sinv_mlp_features(sinv_handle h, const double *N_stack, int m, const double *L_val,
                              const double *D_val, void *X, float *scale, void *stream);
/* y[e] = (G[e] - N[e]) / scale[e] for count entries (device). */
sinv_status sinv_mlp_targets(sinv_mlp m, int64_t count, const double *G, const double *N, const float *scale,
                             float *y, void *stream);
/* Gradient of the mean squared error over the entries idx[0..count) (idx may be
 * NULL: entries 0..count-1) into grad [param_count] and the loss into *loss
 * (both device; grad may be NULL to keep it inside). */
sinv_status sinv_mlp_grad(sinv_mlp m, const void *X, const float *y, const int64_t *idx, int64_t count,
                          float *grad, float *loss, void *stream);
/* sinv_mlp_grad followed by one Adam step (beta 0.9 / 0.999, eps 1e-8) with rate lr. */
sinv_status sinv_mlp_train_step(sinv_mlp m, const void *X, const float *y, const int64_t *idx, int64_t count,
                                float lr, float *loss, void *stream);
/* out[e] = N[e] + scale[e] f(X[e]) for count entries (device).  Runs on the
 * tensor cores (tcgen05, BF16 operands, FP32 accumulators in tensor memory);
 * the first hidden layer is rounded to BF16 as the operand of the second.  X
 * must be 16-byte aligned (SINV_ERR_INVALID_ARG otherwise).  A completion wait
 * that runs out of polls is recorded for sinv_mlp_sync_status. */
sinv_status sinv_mlp_predict(sinv_mlp m, const void *X, const float *scale, const double *N, int64_t count,
                             double *out, void *stream);
/* Synchronizes `stream` and returns the first device error of the network's
 * asynchronous calls since the last check (SINV_ERR_TIMEOUT for a tensor-core
 * completion wait that ran out of polls), then clears it. */
sinv_status sinv_mlp_sync_status(sinv_mlp m, void *stream);

/* Wait for the handle's queued work on `stream` and return the first device
 * error recorded since the last call (then clear it). */
sinv_status sinv_sync_status(sinv_handle h, void *stream);

/* Statistics of the symbolic analysis (host values). */
typedef struct {
    int64_t n, nnz_L, nnz_S_lo, n_blocks, n_2x2, n_supernodes, n_levels;
    int64_t max_c, hit_pairs, max_width;
    int64_t nnz_W;        /* pattern of the truncated series, 0 until sinv_ninv ran */
    int32_t ninv_m;       /* m of that pattern                                        */
    int32_t pad;
    int64_t horner_products;  /* E_kj W[r,k] products of the m Horner steps            */
    int64_t product_stream;   /* entries of W streamed by the product on S             */
    int64_t selinv_flops;     /* algorithmic flops of one SelInv                        */
    int64_t selinv_bytes;     /* algorithmic bytes of one SelInv (S read once, L in, X out) */
    int64_t ninv_index_bytes; /* device bytes of the NInv position maps, 0 = hash form */
    int64_t product_hits;     /* rows shared by W[:, i] and (D^{-1} W)[:, j] over the
                                 entries (i, j) of S_lo: the multiply-adds of the
                                 product (known once the maps exist, else 0)           */
    int64_t spai_entries;     /* entries of A staged by all columns of the SPAI step
                                 (one product A_J^T A_J p streams each twice), 0 until
                                 sinv_spai_analyse ran                                 */
    int64_t spai_cols_warp;   /* columns solved by a warp in shared memory             */
    int64_t spai_cols_cta;    /* columns solved by a CTA with a global scratch block   */
    int64_t spai_nnz_P;       /* |P_lo| of the SPAI pattern, 0 until analysed          */
    int64_t einv_levels_fwd;  /* dependency levels of the solve with L (one launch each),
                                 0 until sinv_einv_analyse ran                          */
    int64_t einv_levels_bwd;  /* dependency levels of the solve with L^T                */
    int64_t tc_levels;        /* leading levels run by the tensor-core forms of SelInv  */
    int64_t tc_supernodes;    /* supernodes in them                                     */
    int64_t tc_pairs;         /* sum of |C|^2 over them (the contraction's size)        */
    int64_t tc_mirror_bytes;  /* their symmetric band copy of G                         */
    int64_t selinv_scan;      /* 1: SelInv reads C x C by scanning rows of S (scan form:
                                 no pair lists; see selinv_pair_bytes), 0: pair lists  */
    int64_t scan_rows_total;  /* sum over supernodes J of the lengths of the rows C_J of
                                 S_lo (an upper bound of the scan form's lookups)      */
} sinv_stats;
sinv_status sinv_get_stats(sinv_handle h, sinv_stats *out);

/* Supernode partition and levels (host arrays owned by the handle):
 * sn_start[n_supernodes+1] (first column of each supernode, then n),
 * sn_level[n_supernodes]. */
sinv_status sinv_get_supernodes(sinv_handle h, const int32_t **sn_start, const int32_t **sn_level,
                                int64_t *n_supernodes);

/* Per-kernel timing.  While enabled, every kernel a numeric call launches is
 * bracketed by CUDA events on the call's stream (small host overhead, no
 * device synchronisation).  sinv_trace_read waits for the recorded events,
 * and copies up to max_entries aggregated rows {kernel name, launches, total
 * milliseconds}; *count receives the number copied.  reset != 0 clears the
 * totals afterwards. */
typedef struct {
    char name[48];
    int64_t launches;
    double total_ms;
} sinv_kernel_time;
sinv_status sinv_trace_enable(sinv_handle h, int enable);
/* Per-supernode timeline of sinv_selinv, for the analysis of its dependency
 * chain (Section 2.1: a supernode starts when the supernodes owning its rows C
 * have finished).  While enabled, every sinv_selinv records device timestamps
 * (globaltimer, nanoseconds) for each supernode J; sinv_timeline_read writes
 * four per supernode into stamps[4J .. 4J+3] (host array of 4 * n_supernodes,
 * n_supernodes as in sinv_get_stats): the earliest start of any of its work
 * items, the latest moment a part saw its dependencies published, the latest
 * end of a part's contraction, and its publication.  Unset stamps read 0 (the
 * first one all ones).  The read synchronizes `stream`.  Recording adds atomic
 * operations to the kernels: time the path with the timeline disabled.
 * Errors: SINV_ERR_INVALID_ARG (not enabled, wrong count), SINV_ERR_OOM. */
sinv_status sinv_timeline_enable(sinv_handle h, int enable);
sinv_status sinv_timeline_read(sinv_handle h, uint64_t *stamps, int64_t n_supernodes, void *stream);
/* Scan form only: the lookups (row entries of S_lo examined) and the pairs of
 * C_J x C_J in S found by the last sinv_selinv made while the timeline was enabled
 * (both 0 for a handle with pair lists, or without such a call).  Synchronises
 * `stream` first. */
sinv_status sinv_selinv_scan_counts(sinv_handle h, int64_t *lookups, int64_t *pairs, void *stream);
sinv_status sinv_trace_read(sinv_handle h, sinv_kernel_time *out, int max_entries, int *count, int reset);

const char *sinv_status_string(sinv_status s);
/* Copies the handle's last error message (NUL terminated) into buf. */
sinv_status sinv_last_error(sinv_handle h, char *buf, size_t len);
void sinv_destroy(sinv_handle h);

/* Tests the bounded-wait machinery every persistent kernel uses: launches one
 * warp that waits, with the handle's poll limit, on a device flag that nothing
 * sets, and returns the status that wait reports (SINV_ERR_TIMEOUT expected). */
sinv_status sinv_debug_wait_timeout(sinv_handle h, void *stream);

/* Test support for the checked build (libsinv_checked.so, compiled with
 * -DSINV_CHECKED): points one stored SelInv pair position past the end of S_lo, so
 * that the next sinv_selinv meets an out-of-range index; the checked kernels skip
 * that access and sinv_sync_status reports SINV_ERR_CUDA ("index out of range").
 * The regular build returns SINV_ERR_UNSUPPORTED and changes nothing (its kernels
 * do not check).  SINV_ERR_UNSUPPORTED also when the handle has no pair lists. */
sinv_status sinv_debug_corrupt_plan(sinv_handle h);

#ifdef __cplusplus
}
#endif
#endif /* SINV_H */
