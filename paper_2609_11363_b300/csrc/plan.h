// Internal data layout shared by the host symbolic analysis and the kernels.
#pragma once
#include <cstdint>
#include <memory>
#include <new>
#include <string>
#include <utility>
#include <vector>

namespace sinv {

// An allocator whose resize() leaves new elements of trivial types uninitialised:
// for the largest arrays of the plan, which a parallel pass fills completely right
// after sizing them (zeroing them first took a single thread as long as the pass).
template <class T>
struct NoInitAlloc : std::allocator<T> {
    template <class U>
    struct rebind {
        using other = NoInitAlloc<U>;
    };
    NoInitAlloc() = default;
    template <class U>
    NoInitAlloc(const NoInitAlloc<U>&) noexcept {}
    template <class U>
    void construct(U* p) noexcept {
        ::new ((void*)p) U;
    }
    template <class U, class... A>
    void construct(U* p, A&&... a) {
        ::new ((void*)p) U(std::forward<A>(a)...);
    }
};
template <class T>
using FillVec = std::vector<T, NoInitAlloc<T>>;

// One supernode: consecutive pivot blocks [s0, s0 + w) processed as one dense
// step of the Takahashi recurrence.  C is the sorted set of rows below the
// supernode touched by any of its columns (|C| = c).
struct SnInfo {
    int32_t s0, w, c, level;
    int64_t crow_off;  // Crow[crow_off .. +c): global row of each local row
    int64_t cw_off;    // Lmap[cw_off .. +c*w): CSR position of L(C[i], s0+t), row-major (i, t), or -1
    int64_t ww_off;    // JJl / JJs [ww_off .. +w*w): within-supernode maps, row-major (a, b)
    int64_t hit_off;   // hit arrays [hit_off .. +hit_cnt)
    int64_t hit_cnt;   // pairs (i, k) of C x C (both triangles and the diagonal) with
                       // (C[i], C[k]) in S, sorted by (i, k)
    int64_t hrow_off;  // hrow[hrow_off .. +c+1): start of row i's pairs, relative to hit_off
    // tensor-core tier (supernodes of the leading levels whose C fills most of the
    // range of rows [C[0], C[c-1]]; -1 / 0 elsewhere).  The tier works on the whole
    // range R (tc_c rows): rows of R outside C have no entry in L_CJ, so they add
    // nothing to Y's rows in C nor to Z, and their X is never stored.
    int32_t tc_c;      // |R|
    int32_t tc_tiles;  // row tiles of 128 rows of R (at least 1)
    int32_t tc_ks;     // parts of the contraction over R per row tile
    int32_t tc_ndep;     // distinct supernodes owning rows of C (the ones to wait for)
    int64_t tc_map_off;  // tc_map[tc_map_off .. + tc_c * w): CSR position of L(R[o], s0+t), or -1
    int64_t tc_dep_off;  // tc_deps[tc_dep_off .. + tc_ndep): those supernodes, latest first
    int64_t tc_t_off;  // arrival counters of the row tiles
    int64_t tc_z_off;  // Z block of w x w doubles (sum over the row tiles)
};

// A unit of the persistent SelInv schedule: either one large supernode that a
// whole CTA processes, or up to kGroup consecutive small ones, one per warp.
struct WorkItem {
    int32_t first;  // index into the processing order
    int32_t count;  // supernodes in the item; for a part of a split supernode: the number of parts
    int32_t big;    // 1: CTA-cooperative; 2: one part of a supernode split over several CTAs
    int32_t part;   // the part (big == 2)
};

struct HostPlan {
    int64_t n = 0, nnzL = 0, nnzS = 0;
    // S_lo
    std::vector<int64_t> Srp;
    FillVec<int32_t> Sc;
    std::vector<int32_t> Sdiag;   // position of (i, i) in S_lo
    FillVec<int32_t> l2s;         // S_lo position of each L entry (CSR order)
    // L by columns (struct(j)), with the CSR position of each entry
    std::vector<int64_t> Lcp;
    FillVec<int32_t> Lri;
    FillVec<int32_t> Lcsr;
    // pivot blocks
    std::vector<int8_t> pstart;
    std::vector<int32_t> dpos;    // per column: offset of its block's first value in D_val
    int64_t nD = 0, n_blocks = 0, n_2x2 = 0;
    // supernodes
    std::vector<SnInfo> sn;
    std::vector<int32_t> sn_start;   // first column of each supernode, then n
    std::vector<int32_t> sn_level;
    std::vector<int32_t> owner;      // supernode of each column
    std::vector<int32_t> order;      // processing order (level-major)
    std::vector<int32_t> Crow, Lmap, JJl, JJs;
    FillVec<uint32_t> hit_ik;        // (i << 16) | k
    FillVec<int32_t> hit_pos;        // S_lo position of (max, min) of (C[i], C[k])
    std::vector<int32_t> hrow;       // per supernode c+1 row starts
    std::vector<WorkItem> items;
    // supernodes split over several CTAs: offset of their c*w partial-sum block (-1: not split)
    std::vector<int64_t> xsum_off;
    int64_t xsum_total = 0;
    // tensor-core tier: the leading tc_levels levels, whose supernodes all have a
    // nearly contiguous C and width <= kTcWMax.  tc_items: one per (supernode, row tile,
    // part of the contraction) in processing order; items[rest_first ..] are the
    // supernodes of the later levels.  The tier reads G~ from a symmetric band
    // copy ("mirror") of rows [tc_row0, n), columns row - tc_band .. row + tc_band
    // with a margin of 64 both ways, tc_width values per row.
    int64_t tc_levels = 0, rest_first = 0, tc_sn = 0, tc_pairs = 0;
    std::vector<WorkItem> tc_items;
    int64_t tc_t_total = 0, tc_z_total = 0;
    int64_t tc_row0 = 0, tc_band = 0, tc_width = 0;
    std::vector<int32_t> tc_map;
    std::vector<int32_t> tc_deps;
    int64_t n_levels = 0, max_c = 0, max_w = 0, max_cw = 0, hit_pairs = 0;
    // scan form: no pair lists are stored; every supernode reads G~_CC by scanning
    // the rows C of S_lo backwards from the diagonal to C[0] and looking each column
    // up in a hash table of C.  hrow then holds, per supernode, the prefix over its
    // rows of the row lengths of S_lo (the work measure that splits rows over CTAs),
    // and hit_cnt a third of its total (the same scale as a pair count).
    // scan_rows_total: sum over supernodes of those lengths (an upper bound of the
    // lookups; the kernel counts the exact ones on request).
    int32_t scan = 0;
    int64_t scan_rows_total = 0;
    // algorithmic work of one SelInv: 2 w flops per pair of C x C in S, 2 c w^2 for
    // the diagonal block; bytes: each entry of S in C x C once (8 B) and L_CJ in, X out
    int64_t selinv_flops = 0, selinv_bytes = 0;
};

// Neumann-series pattern P_W = pattern(sum_{t<=m} E^t), stored by columns.
// Column j lists its rows grouped by the first power t that reaches them
// (t = 0 is row j itself), each group sorted by row; grp[j*(m+2) + t] is the
// start of group t inside column j (relative to Wcp[j]), grp[j*(m+2)+m+1] its end.
// Bit 31 of a row entry is set when that row belongs to a 2x2 block of D.
struct NinvPlan {
    int m = -1;
    int64_t nnzW = 0;
    std::vector<int64_t> Wcp;
    FillVec<int32_t> Wr;
    std::vector<int32_t> grp;
    int64_t max_col = 0;
    // algorithmic work: products E_kj W_{t-1}[r,k] of all m Horner steps, and the
    // entries of W streamed by the product on S (sum over (i,j) in S_lo of |col i|)
    int64_t horner_products = 0;
    int64_t product_stream = 0;
};

// SPAI refinement (Section 2.4) on a symmetric pattern P for a given pattern of
// A.  P = S united with {(i, j) : graph distance between i and j in A <= power}
// (power 0: P = S), lower part in CSR.  Its columns (both triangles, rows
// ascending) carry the P_lo position of each entry, the S_lo position the
// start value comes from (-1: start at 0), and the offset of the entry's row
// of A inside the column's list of A entries.  Columns are split into two
// tiers by size.
struct SpaiPlan {
    int64_t n = 0, nnzA = 0, nnzP = 0;
    int power = 0;
    std::vector<int64_t> Prp;     // P_lo, CSR with sorted rows (the diagonal last)
    std::vector<int32_t> Pc;
    std::vector<int64_t> fcp;     // n+1
    std::vector<int32_t> fri;     // |P|: rows of each column, ascending
    std::vector<int32_t> fpos;    // |P|: P_lo position of (max, min)
    std::vector<int32_t> fsrc;    // |P|: S_lo position of (max, min), -1 outside S
    std::vector<int32_t> feo;     // |P|: sum of nnz(A row) over the earlier rows of the column
    std::vector<int32_t> fE;      // n: entries of A staged by each column
    std::vector<int32_t> fR;      // n: distinct rows of A those entries touch (the table y)
    std::vector<int32_t> cols_w;  // columns a warp solves in shared memory (most entries first)
    std::vector<int32_t> cols_c;  // the rest: a CTA each, with a global scratch block
    int64_t cap_nj = 0, cap_E = 0, cap_H = 0;  // largest tier-C column: rows, entries, table (pow2 >= 2R)
    int64_t entries = 0;          // sum of fE: entries of A streamed by one B product over all columns
};

// Spectral-correction producer (Section 2.5): what the Lanczos iteration on
// E_inv = A^{-1} - A^inv needs besides the plan of S.  The columns of S (both
// triangles) apply A^inv, given on S_lo; the rows of L grouped by dependency
// level drive the forward solve with L, the columns grouped the same way the
// solve with L^T (the two triangular factors of the ILDL preconditioner).
struct EinvPlan {
    int64_t n = 0, nnzA = 0;
    std::vector<int64_t> fcp;      // n+1: columns of S
    std::vector<int32_t> fri;      // rows of each column
    std::vector<int32_t> fpos;     // S_lo position of each entry
    std::vector<int32_t> Lcol;     // nnz(L): column of every CSR entry of L
    std::vector<int32_t> fwd_rows, fwd_ptr;  // rows of level l: fwd_rows[fwd_ptr[l] .. fwd_ptr[l+1])
    std::vector<int32_t> bwd_cols, bwd_ptr;  // columns of level l of the solve with L^T
};

constexpr int kTcWMax = 32;     // widest supernode of the tensor-core tier
constexpr int kTcRowsTile = 128;  // rows of C per tensor-core tile (the MMA's M)
constexpr int kTcMaxChunks = 8;   // 32-column chunks of one part of the contraction

// Returns an empty string on success, else the reason the pattern is invalid.
// big_pairs: supernodes with at least this many pairs are processed by a whole CTA;
// group: small supernodes per work item (one per warp); levels with fewer than
// thin_level supernodes give every supernode a whole CTA.
// pair_bytes: bytes the pair lists may take (> 0), 0 for the default 8 GB, < 0 to
// take the scan form whatever the size.
std::string build_plan(int64_t n, const int64_t* L_rowptr, const int32_t* L_col,
                       const int8_t* pivot_start, int supernode_cap, int64_t big_pairs, int group,
                       int64_t thin_level, HostPlan& P, int64_t pair_bytes = 0);
std::string build_ninv_plan(const HostPlan& P, int m, NinvPlan& W);
// A: n x n CSR pattern (host), structurally symmetric; warp_j / warp_e / warp_r: the
// tier-W caps on pattern rows, staged entries and distinct rows of A.
// Prp_given / Pc_given / src_given (optional): the pattern P_lo itself (CSR, sorted
// rows, the diagonal last) and, per entry, the index of its start value.
std::string build_spai_plan(const HostPlan& P, int64_t nnzA, const int64_t* A_rowptr, const int32_t* A_col,
                            int power, int warp_j, int warp_e, int warp_r, SpaiPlan& X,
                            const int64_t* Prp_given = nullptr, const int32_t* Pc_given = nullptr,
                            const int32_t* src_given = nullptr);
// A: n x n CSR pattern (host), structurally symmetric (the same checks as above).
std::string build_einv_plan(const HostPlan& P, int64_t nnzA, const int64_t* A_rowptr, const int32_t* A_col,
                            EinvPlan& X);

}  // namespace sinv
