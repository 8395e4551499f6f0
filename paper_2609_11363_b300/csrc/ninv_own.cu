// NInv on its own pattern (Section 2.2, Eqs. (6) and (8)): the inverse tolerance
// delta sparsifies the Neumann series W = L^inv and the product W^T D^{-1} W, so
// both patterns depend on the values and fall with delta.
//
// Horner step t (column form, W_t[:, j] = e_j + sum_{k in struct(j)} E_kj
// W_{t-1}[:, k]): one CTA per column accumulates the products in a hash table
// (shared memory, or a global slice for long columns) sized by the column's bound
// 1 + sum_k |W_{t-1}[:, k]| (capped at n - j), drops the off-diagonal entries
// below delta, and appends the survivors to the step's output through a global
// cursor: column j is the segment [st[j], st[j] + ct[j]) of one contiguous array.
// A step whose survivors pass the output's capacity writes nothing past it; the
// cursor still counts every survivor, so the host grows the array to exactly that
// size and runs the step again.  No structural pattern of the series is needed.
//
// Product: with Y = D^{-1} W (rows of column j and their 2x2 partners), a first
// pass forms every diagonal N_jj = W[:, j] . Y[:, j] and a bound on the length of
// column j of N (the sum of the lengths of the rows of W that Y[:, j] touches,
// capped at n - j); the second pass accumulates N[i, j] = sum_c W[c, i] Y[c, j]
// for i >= j through the rows of W (W transposed once) in a hash table, keeps the
// diagonal and the entries with |N_ij| >= delta sqrt|N_ii N_jj|, and appends them
// the same way.  A scan and a copy give the result as CSC of the lower triangle
// (rows in hash order).
#include <algorithm>

#include "device.cuh"
#include "hash.cuh"
#include "kernels.h"

namespace sinv {

namespace {

constexpr int kOwnThreads = 256;
constexpr int kOwnWarps = kOwnThreads / 32;
constexpr int kSmemSlots = 2048;    // keys + FP64 values in shared memory: 24 KB (diagonal pass, Mix)
constexpr int kHornerSlots = 4096;  // Horner step: 48 KB of dynamic shared memory
constexpr int kProdSlots = 2048;    // product: two tables (Y and N's column), 48 KB in all

// per-CTA table: shared memory when it fits, else the given global slice
struct Table {
    int32_t* keys;
    double* vals;
    uint32_t mask;
};

__device__ __forceinline__ Table make_table(int64_t entries, int32_t* skeys, double* svals, int smem_slots,
                                            int32_t* gkeys, double* gvals) {
    Table t;
    t.mask = table_mask(entries);
    if ((int64_t)t.mask + 1 <= smem_slots) {
        t.keys = skeys;
        t.vals = svals;
    } else {
        t.keys = gkeys;
        t.vals = gvals;
    }
    for (uint32_t s = threadIdx.x; s <= t.mask; s += blockDim.x) {
        t.keys[s] = -1;
        t.vals[s] = 0.0;
    }
    return t;
}

__device__ __forceinline__ void table_add(Table& t, int32_t r, double v) {
    const uint32_t s = table_insert(t.keys, t.mask, r);
    atomicAdd(t.vals + s, v);
}

// The same into a shared-memory table that may be too small: the distinct rows it
// takes are counted, and past `limit` (half its slots) the column is marked for a
// second pass with a table sized by its bound; nothing is added after the mark.
__device__ __forceinline__ void table_add_opt(Table& t, int32_t r, double v, int32_t* n_keys, int32_t limit,
                                              volatile int32_t* over) {
    if (*over) return;
    uint32_t h = hash_row(r, t.mask);
    for (uint32_t probe = 0; probe <= t.mask; ++probe) {
        const int32_t old = atomicCAS(t.keys + h, -1, r);
        if (old == -1) {
            if (atomicAdd(n_keys, 1) >= limit) *over = 1;
            atomicAdd(t.vals + h, v);
            return;
        }
        if (old == r) {
            atomicAdd(t.vals + h, v);
            return;
        }
        h = (h + 1) & t.mask;
    }
    *over = 1;
}

__device__ __forceinline__ void atomic_max_i64(int64_t* p, int64_t v) {
    atomicMax(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v);
}

// appends the table's kept entries (keep(key, value)) of column j: counts them,
// reserves [base, base + count) through the cursor, records the segment, and
// writes the entries when they fit below cap
template <class Keep>
__device__ __forceinline__ void append_kept(const Table& t, Keep keep, int64_t j, int32_t* rOut, double* vOut,
                                            int64_t* stOut, int64_t* ctOut, int64_t cap,
                                            unsigned long long* cursor, int32_t* s_cnt, int64_t* s_base) {
    for (uint32_t s = threadIdx.x; s <= t.mask; s += blockDim.x) {
        const int32_t r = t.keys[s];
        if (r >= 0 && keep(r, t.vals[s])) atomicAdd(s_cnt, 1);
    }
    __syncthreads();
    const int64_t cnt = *s_cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        const int64_t base = (int64_t)atomicAdd(cursor, (unsigned long long)cnt);
        *s_base = base;
        stOut[j] = base;
        ctOut[j] = cnt;
        *s_cnt = 0;  // reused as the write position
    }
    __syncthreads();
    const int64_t base = *s_base;
    if (base + cnt <= cap) {
        for (uint32_t s = threadIdx.x; s <= t.mask; s += blockDim.x) {
            const int32_t r = t.keys[s];
            if (r < 0) continue;
            const double v = t.vals[s];
            if (!keep(r, v)) continue;
            const int32_t o = atomicAdd(s_cnt, 1);
            rOut[base + o] = r;
            vOut[base + o] = v;
        }
    }
    __syncthreads();
}

// the largest Horner table bound of a step: 1 + sum_{k in struct(j)} |W_{t-1}[:, k]|, capped at n - j
__global__ void own_bound(int64_t n, const int64_t* __restrict__ Lcp, const int32_t* __restrict__ Lri,
                          const int64_t* __restrict__ ctIn, int64_t* __restrict__ maxb) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < n; j += nw) {
        int64_t b = 0;
        for (int64_t q = Lcp[j] + lane; q < Lcp[j + 1]; q += 32) b += ctIn[Lri[q]];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(0xffffffffu, b, o);
        if (lane == 0) atomic_max_i64(maxb, min(b + 1, n - j));
    }
}

// the largest of x[0..n)
__global__ void own_max(int64_t n, const int64_t* __restrict__ x, int64_t* __restrict__ out) {
    int64_t m = 0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        m = max(m, x[j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomic_max_i64(out, m);
}

// W_t from W_{t-1}: columns in any order (ticket)
__global__ void __launch_bounds__(kOwnThreads) own_horner(int64_t n, const int64_t* __restrict__ Lcp,
                                                          const int32_t* __restrict__ Lri,
                                                          const int32_t* __restrict__ Lcsr,
                                                          const double* __restrict__ Lval,
                                                          const int64_t* __restrict__ stIn,
                                                          const int64_t* __restrict__ ctIn,
                                                          const int32_t* __restrict__ rIn,
                                                          const double* __restrict__ vIn, double delta,
                                                          int32_t* __restrict__ rOut, double* __restrict__ vOut,
                                                          int64_t* __restrict__ stOut, int64_t* __restrict__ ctOut,
                                                          int64_t cap, unsigned long long* cursor, int32_t* gkeys,
                                                          double* gvals, int64_t gslice, int32_t* ticket) {
    extern __shared__ __align__(16) unsigned char own_dyn[];
    int32_t* skeys = reinterpret_cast<int32_t*>(own_dyn);
    double* svals = reinterpret_cast<double*>(own_dyn + kHornerSlots * sizeof(int32_t));
    __shared__ int64_t s_j, s_base;
    __shared__ unsigned long long s_b;
    __shared__ int32_t s_cnt, s_keys, s_over;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t* gk = gkeys + (int64_t)blockIdx.x * gslice;
    double* gv = gvals + (int64_t)blockIdx.x * gslice;
    for (;;) {
        if (threadIdx.x == 0) {
            s_j = atomicAdd(ticket, 1);
            s_cnt = 0;
            s_b = 0ull;
            s_keys = 0;
            s_over = 0;
        }
        __syncthreads();
        const int64_t j = s_j;
        if (j >= n) break;
        // the column's bound: every row it can receive
        unsigned long long b = 0;
        for (int64_t q = Lcp[j] + threadIdx.x; q < Lcp[j + 1]; q += blockDim.x) b += (unsigned long long)ctIn[Lri[q]];
        atomicAdd(&s_b, b);
        __syncthreads();
        const int64_t bound = min((int64_t)s_b + 1, n - j);
        // a bound past shared memory first tries the shared table (the bound counts a
        // row once per column it comes from; the distinct rows are usually far fewer)
        const bool opt = (int64_t)table_mask(bound) + 1 > kHornerSlots;
        Table t = make_table(opt ? kHornerSlots / 2 : bound, skeys, svals, kHornerSlots, gk, gv);
        __syncthreads();
        for (int pass = 0; pass < 2; ++pass) {
            const bool o = opt && pass == 0;
            if (threadIdx.x == 0) {
                if (o) table_add_opt(t, (int32_t)j, 1.0, &s_keys, kHornerSlots / 2, &s_over);
                else table_add(t, (int32_t)j, 1.0);
            }
            for (int64_t q = Lcp[j] + wid; q < Lcp[j + 1]; q += kOwnWarps) {
                const int32_t k = Lri[q];
                const double e = -Lval[Lcsr[q]];
                const int64_t p0 = stIn[k], p1 = p0 + ctIn[k];
                for (int64_t p = p0 + lane; p < p1; p += 32) {
                    if (o) table_add_opt(t, rIn[p], e * vIn[p], &s_keys, kHornerSlots / 2, &s_over);
                    else table_add(t, rIn[p], e * vIn[p]);
                }
            }
            __syncthreads();
            if (!(o && s_over)) break;
            t = make_table(bound, skeys, svals, kHornerSlots, gk, gv);  // the second pass: sized by the bound
            __syncthreads();
        }
        const int32_t jj = (int32_t)j;
        append_kept(t, [&](int32_t r, double v) { return r == jj || fabs(v) >= delta; }, j, rOut, vOut, stOut, ctOut,
                    cap, cursor, &s_cnt, &s_base);
    }
}

// W by rows: counts over the contiguous entries, then the entries (column i and
// value) of every row, column by column
__global__ void own_row_count(int64_t nnz, const int32_t* __restrict__ r, int64_t* __restrict__ rowcnt) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(reinterpret_cast<unsigned long long*>(rowcnt + r[e]), 1ull);
}

__global__ void own_row_fill(int64_t n, const int64_t* __restrict__ st, const int64_t* __restrict__ ct,
                             const int32_t* __restrict__ r, const double* __restrict__ v, int64_t* __restrict__ fill,
                             int32_t* __restrict__ rc, double* __restrict__ rv) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        for (int64_t p = st[j]; p < st[j] + ct[j]; ++p) {
            const int64_t d = (int64_t)atomicAdd(reinterpret_cast<unsigned long long*>(fill + r[p]), 1ull);
            rc[d] = (int32_t)j;
            rv[d] = v[p];
        }
}

// Y[:, j] = D^{-1} W[:, j] in the table (rows of the column and their partners)
__device__ __forceinline__ void fill_y(Table& t, const int64_t* st, const int64_t* ct, const int32_t* r,
                                       const double* v, int64_t j, const double* dr, const double* dp,
                                       const int32_t* part) {
    for (int64_t p = st[j] + threadIdx.x; p < st[j] + ct[j]; p += blockDim.x) {
        const int32_t c = r[p];
        const double w = v[p];
        table_add(t, c, dr[c] * w);
        if (part[c] >= 0) table_add(t, part[c], dp[c] * w);
    }
}

// pass A: N_jj = W[:, j] . Y[:, j], and the bound sum over the rows c of Y[:, j] of
// the length of row c of W, capped at n - j (the rows i >= j of column j of N)
__global__ void __launch_bounds__(kOwnThreads) own_diag(int64_t n, const int64_t* __restrict__ st,
                                                        const int64_t* __restrict__ ct,
                                                        const int32_t* __restrict__ r, const double* __restrict__ v,
                                                        const int64_t* __restrict__ rp, const double* __restrict__ dr,
                                                        const double* __restrict__ dp, const int32_t* __restrict__ part,
                                                        double* __restrict__ diag, int64_t* __restrict__ bound,
                                                        int64_t* __restrict__ maxb, int32_t* gkeys, double* gvals,
                                                        int64_t gslice, int32_t* ticket) {
    __shared__ int32_t skeys[kSmemSlots];
    __shared__ double svals[kSmemSlots];
    __shared__ int64_t s_j;
    __shared__ double s_d;
    __shared__ unsigned long long s_b;
    int32_t* gk = gkeys + (int64_t)blockIdx.x * gslice;
    double* gv = gvals + (int64_t)blockIdx.x * gslice;
    for (;;) {
        if (threadIdx.x == 0) {
            s_j = atomicAdd(ticket, 1);
            s_d = 0.0;
            s_b = 0ull;
        }
        __syncthreads();
        const int64_t j = s_j;
        if (j >= n) break;
        Table t = make_table(2 * ct[j], skeys, svals, kSmemSlots, gk, gv);
        __syncthreads();
        fill_y(t, st, ct, r, v, j, dr, dp, part);
        __syncthreads();
        double s = 0.0;
        for (int64_t p = st[j] + threadIdx.x; p < st[j] + ct[j]; p += blockDim.x) {
            const int32_t slot = table_find(t.keys, t.mask, r[p]);
            if (slot >= 0) s += v[p] * t.vals[slot];
        }
        unsigned long long b = 0ull;
        for (uint32_t sl = threadIdx.x; sl <= t.mask; sl += blockDim.x) {
            const int32_t c = t.keys[sl];
            if (c >= 0) b += (unsigned long long)(rp[c + 1] - rp[c]);
        }
        atomicAdd(&s_d, s);
        atomicAdd(&s_b, b);
        __syncthreads();
        if (threadIdx.x == 0) {
            diag[j] = s_d;
            const int64_t bj = min((int64_t)s_b, n - j);
            bound[j] = bj;
            atomic_max_i64(maxb, bj);
        }
        __syncthreads();
    }
}

// pass B: column j of N (rows i >= j) with the drop, appended
__global__ void __launch_bounds__(kOwnThreads) own_product(int64_t n, const int64_t* __restrict__ st,
                                                           const int64_t* __restrict__ ct,
                                                           const int32_t* __restrict__ r,
                                                           const double* __restrict__ v,
                                                           const int64_t* __restrict__ rp,
                                                           const int32_t* __restrict__ rc,
                                                           const double* __restrict__ rv,
                                                           const double* __restrict__ dr,
                                                           const double* __restrict__ dp,
                                                           const int32_t* __restrict__ part,
                                                           const double* __restrict__ diag,
                                                           const int64_t* __restrict__ bound, double delta,
                                                           int32_t* __restrict__ nr, double* __restrict__ nv,
                                                           int64_t* __restrict__ stN, int64_t* __restrict__ ctN,
                                                           int64_t cap, unsigned long long* cursor, int32_t* gkeys,
                                                           double* gvals, int64_t gslice, int32_t* ticket) {
    extern __shared__ __align__(16) unsigned char own_dyn[];
    int32_t* skeys = reinterpret_cast<int32_t*>(own_dyn);
    int32_t* skeys2 = skeys + kProdSlots;
    double* svals = reinterpret_cast<double*>(own_dyn + 2 * kProdSlots * sizeof(int32_t));
    double* svals2 = svals + kProdSlots;
    __shared__ int64_t s_j, s_base;
    __shared__ int32_t s_cnt, s_keys, s_over;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // Y[:, j] in the first half of the CTA's slice, N's column in the second
    int32_t* gk = gkeys + (int64_t)blockIdx.x * gslice;
    double* gv = gvals + (int64_t)blockIdx.x * gslice;
    for (;;) {
        if (threadIdx.x == 0) {
            s_j = atomicAdd(ticket, 1);
            s_cnt = 0;
            s_keys = 0;
            s_over = 0;
        }
        __syncthreads();
        const int64_t j = s_j;
        if (j >= n) break;
        // N's column: a bound past shared memory first tries the shared table
        const bool opt = (int64_t)table_mask(bound[j]) + 1 > kProdSlots;
        Table ty = make_table(2 * ct[j], skeys, svals, kProdSlots, gk, gv);
        Table tn = make_table(opt ? kProdSlots / 2 : bound[j], skeys2, svals2, kProdSlots, gk + gslice / 2,
                              gv + gslice / 2);
        __syncthreads();
        fill_y(ty, st, ct, r, v, j, dr, dp, part);
        __syncthreads();
        // N[i, j] += W[c, i] Y[c, j] over the rows c of Y[:, j] and the entries of row c of W
        for (int pass = 0; pass < 2; ++pass) {
            const bool o = opt && pass == 0;
            for (uint32_t s = wid; s <= ty.mask; s += kOwnWarps) {
                const int32_t c = ty.keys[s];
                if (c < 0) continue;
                const double y = ty.vals[s];
                for (int64_t p = rp[c] + lane; p < rp[c + 1]; p += 32) {
                    const int32_t i = rc[p];
                    if (i < j) continue;
                    if (o) table_add_opt(tn, i, rv[p] * y, &s_keys, kProdSlots / 2, &s_over);
                    else table_add(tn, i, rv[p] * y);
                }
            }
            __syncthreads();
            if (!(o && s_over)) break;
            tn = make_table(bound[j], skeys2, svals2, kProdSlots, gk + gslice / 2, gv + gslice / 2);
            __syncthreads();
        }
        const double djj = diag[j];
        const int32_t jj = (int32_t)j;
        append_kept(tn, [&](int32_t i, double x) { return i == jj || fabs(x) >= delta * sqrt(fabs(diag[i] * djj)); },
                    j, nr, nv, stN, ctN, cap, cursor, &s_cnt, &s_base);
    }
}

// W_0 = I
__global__ void own_identity(int64_t n, int64_t* __restrict__ st, int64_t* __restrict__ ct, int32_t* __restrict__ r,
                             double* __restrict__ v) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        st[j] = j;
        ct[j] = 1;
        r[j] = (int32_t)j;
        v[j] = 1.0;
    }
}

// exclusive scan of cnt[0..n) into out[0..n], one CTA (out[n] = total)
__global__ void __launch_bounds__(1024) own_scan(int64_t n, const int64_t* __restrict__ cnt, int64_t* __restrict__ out) {
    __shared__ int64_t part[1024];
    const int64_t per = (n + 1023) / 1024;
    const int64_t a = (int64_t)threadIdx.x * per, b = min(n, a + per);
    int64_t s = 0;
    for (int64_t i = a; i < b; ++i) s += cnt[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t run = 0;
        for (int u = 0; u < 1024; ++u) {
            const int64_t v = part[u];
            part[u] = run;
            run += v;
        }
        out[n] = run;
    }
    __syncthreads();
    int64_t run = part[threadIdx.x];
    for (int64_t i = a; i < b; ++i) {
        out[i] = run;
        run += cnt[i];
    }
}

// copy every column's entries from its segment [off[j], ...) to [cp[j], cp[j+1])
__global__ void own_compact(int64_t n, const int64_t* __restrict__ off, const int64_t* __restrict__ cp,
                            const int32_t* __restrict__ rs, const double* __restrict__ vs, int32_t* __restrict__ rd,
                            double* __restrict__ vd) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < n; j += nw) {
        const int64_t o = off[j], d = cp[j], len = cp[j + 1] - cp[j];
        for (int64_t e = lane; e < len; e += 32) {
            rd[d + e] = rs[o + e];
            vd[d + e] = vs[o + e];
        }
    }
}

// ---- Mix on NInv's own pattern (Section 2.3) ------------------------------------
// Column j of the result: the rows of N's column j (values of N), then the rows
// of S_eps in column j that N's column lacks; where a row of S_eps is in N's
// column its value is G's.  An int table maps the rows of N's column to their
// positions in it.
__device__ __forceinline__ uint32_t mix_hash(int32_t r, uint32_t mask) { return ((uint32_t)r * 2654435761u) & mask; }

// the entries of column j of S_lo: u = 0 the diagonal, u = 1 the 2x2 partner row
// j + 1 when j opens a 2x2 block, then the rows of L's column j
__device__ __forceinline__ void s_col_entry(int64_t j, int64_t u, bool partner, const int64_t* Srp,
                                            const int32_t* Sdiag, const int64_t* Lcp, const int32_t* Lri,
                                            const int32_t* Lcsr, const int32_t* l2s, int32_t& i, int64_t& p) {
    if (u == 0) {
        i = (int32_t)j;
        p = Sdiag[j];
    } else if (partner && u == 1) {
        i = (int32_t)(j + 1);
        p = Srp[j + 2] - 2;
    } else {
        const int64_t q = Lcp[j] + u - 1 - (partner ? 1 : 0);
        i = Lri[q];
        p = l2s[Lcsr[q]];
    }
}

template <bool kFill>
__global__ void __launch_bounds__(kOwnThreads) mix_own_kernel(int64_t n, const int64_t* __restrict__ Ncp,
                                                              const int32_t* __restrict__ Nr,
                                                              const double* __restrict__ Nv,
                                                              const int64_t* __restrict__ Srp,
                                                              const int32_t* __restrict__ Sdiag,
                                                              const int64_t* __restrict__ Lcp,
                                                              const int32_t* __restrict__ Lri,
                                                              const int32_t* __restrict__ Lcsr,
                                                              const int32_t* __restrict__ l2s,
                                                              const int8_t* __restrict__ pstart,
                                                              const double* __restrict__ G, double eps,
                                                              int64_t* __restrict__ cnt_or_cp, int32_t* __restrict__ outR,
                                                              double* __restrict__ outV, int32_t* gkeys,
                                                              int64_t gslice, int32_t* ticket) {
    __shared__ int32_t skeys[kSmemSlots];
    __shared__ int32_t sidx[kSmemSlots];
    __shared__ int64_t s_j;
    __shared__ int32_t s_extra;
    int32_t* gk = gkeys + (int64_t)blockIdx.x * 2 * gslice;
    for (;;) {
        if (threadIdx.x == 0) {
            s_j = atomicAdd(ticket, 1);
            s_extra = 0;
        }
        __syncthreads();
        const int64_t j = s_j;
        if (j >= n) break;
        const int64_t c0 = Ncp[j], len = Ncp[j + 1] - c0;
        const uint32_t mask = table_mask(len);
        int32_t* keys = (int64_t)mask + 1 <= kSmemSlots ? skeys : gk;
        int32_t* idx = (int64_t)mask + 1 <= kSmemSlots ? sidx : gk + gslice;
        for (uint32_t s = threadIdx.x; s <= mask; s += blockDim.x) keys[s] = -1;
        __syncthreads();
        for (int64_t e = threadIdx.x; e < len; e += blockDim.x) {
            const int32_t r = Nr[c0 + e];
            uint32_t h = mix_hash(r, mask);
            while (atomicCAS(keys + h, -1, r) != -1) h = (h + 1) & mask;  // the rows of a column are distinct
            idx[h] = (int32_t)e;
        }
        const int64_t o = kFill ? cnt_or_cp[j] : 0;
        if (kFill)
            for (int64_t e = threadIdx.x; e < len; e += blockDim.x) {
                outR[o + e] = Nr[c0 + e];
                outV[o + e] = Nv[c0 + e];
            }
        __syncthreads();
        const bool partner = pstart[j] != 0 && j + 1 < n && pstart[j + 1] == 0;
        const int64_t ns = 1 + (partner ? 1 : 0) + (Lcp[j + 1] - Lcp[j]);
        for (int64_t u = threadIdx.x; u < ns; u += blockDim.x) {
            int32_t i;
            int64_t p;
            s_col_entry(j, u, partner, Srp, Sdiag, Lcp, Lri, Lcsr, l2s, i, p);
            const double g = G[p];
            if (!(fabs(g) > eps)) continue;
            // the row in N's column, or -1
            int32_t k = -1;
            uint32_t h = mix_hash(i, mask);
            for (uint32_t probe = 0; probe <= mask; ++probe) {
                const int32_t key = keys[h];
                if (key == i) {
                    k = idx[h];
                    break;
                }
                if (key < 0) break;
                h = (h + 1) & mask;
            }
            if (k >= 0) {
                if (kFill) outV[o + k] = g;
            } else {
                const int32_t x = atomicAdd(&s_extra, 1);
                if (kFill) {
                    outR[o + len + x] = i;
                    outV[o + len + x] = g;
                }
            }
        }
        __syncthreads();
        if (!kFill && threadIdx.x == 0) cnt_or_cp[j] = len + s_extra;
        __syncthreads();
    }
}

// the longest column of a CSC pointer array
__global__ void own_max_col(int64_t n, const int64_t* __restrict__ cp, int64_t* __restrict__ out) {
    int64_t m = 0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        m = max(m, cp[j + 1] - cp[j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomic_max_i64(out, m);
}

}  // namespace

cudaError_t own_max_col_launch(int64_t n, const int64_t* cp, int64_t* out, int num_sms, cudaStream_t s) {
    cudaMemsetAsync(out, 0, sizeof(int64_t), s);
    own_max_col<<<num_sms * 4, 256, 0, s>>>(n, cp, out);
    return cudaGetLastError();
}

cudaError_t mix_own_launch(const MixOwnArgs& a, bool fill, int64_t* cnt_or_cp, int32_t* outR, double* outV,
                           cudaStream_t s) {
    cudaMemsetAsync(a.ticket, 0, sizeof(int32_t), s);
    if (fill) {
        trace_begin("mix_own_fill", s);
        mix_own_kernel<true><<<a.grid, kOwnThreads, 0, s>>>(a.n, a.Ncp, a.Nr, a.Nv, a.Srp, a.Sdiag, a.Lcp, a.Lri,
                                                            a.Lcsr, a.l2s, a.pstart, a.G, a.eps, cnt_or_cp, outR,
                                                            outV, a.gkeys, a.gslice, a.ticket);
    } else {
        trace_begin("mix_own_count", s);
        mix_own_kernel<false><<<a.grid, kOwnThreads, 0, s>>>(a.n, a.Ncp, a.Nr, a.Nv, a.Srp, a.Sdiag, a.Lcp, a.Lri,
                                                             a.Lcsr, a.l2s, a.pstart, a.G, a.eps, cnt_or_cp, outR,
                                                             outV, a.gkeys, a.gslice, a.ticket);
    }
    trace_end(s);
    return cudaGetLastError();
}

cudaError_t own_identity_launch(int64_t n, int64_t* st, int64_t* ct, int32_t* r, double* v, int num_sms,
                                cudaStream_t s) {
    own_identity<<<num_sms * 4, 256, 0, s>>>(n, st, ct, r, v);
    return cudaGetLastError();
}

cudaError_t own_bound_launch(int64_t n, const int64_t* Lcp, const int32_t* Lri, const int64_t* ctIn, int64_t* maxb,
                             int num_sms, cudaStream_t s) {
    cudaMemsetAsync(maxb, 0, sizeof(int64_t), s);
    own_bound<<<num_sms * 8, 256, 0, s>>>(n, Lcp, Lri, ctIn, maxb);
    return cudaGetLastError();
}

cudaError_t own_max_launch(int64_t n, const int64_t* x, int64_t* out, int num_sms, cudaStream_t s) {
    cudaMemsetAsync(out, 0, sizeof(int64_t), s);
    own_max<<<num_sms * 4, 256, 0, s>>>(n, x, out);
    return cudaGetLastError();
}

cudaError_t own_horner_launch(const OwnArgs& a, const int64_t* stIn, const int64_t* ctIn, const int32_t* rIn,
                              const double* vIn, int32_t* rOut, double* vOut, int64_t* stOut, int64_t* ctOut,
                              int64_t cap, cudaStream_t s) {
    cudaMemsetAsync(a.ticket, 0, sizeof(int32_t), s);
    cudaMemsetAsync(a.cursor, 0, sizeof(unsigned long long), s);
    trace_begin("ninv_own_horner", s);
    own_horner<<<a.grid, kOwnThreads, kHornerSlots * (sizeof(int32_t) + sizeof(double)), s>>>(a.n, a.Lcp, a.Lri, a.Lcsr, a.Lval, stIn, ctIn, rIn, vIn, a.delta, rOut,
                                              vOut, stOut, ctOut, cap, a.cursor, a.gkeys, a.gvals, a.gslice, a.ticket);
    trace_end(s);
    return cudaGetLastError();
}

cudaError_t own_scan_launch(int64_t n, const int64_t* cnt, int64_t* out, cudaStream_t s) {
    own_scan<<<1, 1024, 0, s>>>(n, cnt, out);
    return cudaGetLastError();
}

cudaError_t own_compact_launch(int64_t n, const int64_t* off, const int64_t* cp, const int32_t* rs, const double* vs,
                               int32_t* rd, double* vd, int num_sms, cudaStream_t s) {
    own_compact<<<num_sms * 8, 256, 0, s>>>(n, off, cp, rs, vs, rd, vd);
    return cudaGetLastError();
}

cudaError_t own_transpose_launch(int64_t n, int64_t nnz, const int64_t* st, const int64_t* ct, const int32_t* r,
                                 const double* v, int64_t* rowcnt, int64_t* rp, int64_t* fill, int32_t* rc,
                                 double* rv, int num_sms, cudaStream_t s) {
    cudaMemsetAsync(rowcnt, 0, n * sizeof(int64_t), s);
    own_row_count<<<num_sms * 8, 256, 0, s>>>(nnz, r, rowcnt);
    own_scan<<<1, 1024, 0, s>>>(n, rowcnt, rp);
    cudaMemcpyAsync(fill, rp, n * sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
    own_row_fill<<<num_sms * 8, 256, 0, s>>>(n, st, ct, r, v, fill, rc, rv);
    return cudaGetLastError();
}

cudaError_t own_diag_launch(const OwnArgs& a, const int64_t* st, const int64_t* ct, const int32_t* r, const double* v,
                            const int64_t* rp, double* diag, int64_t* bound, int64_t* maxb, cudaStream_t s) {
    cudaMemsetAsync(a.ticket, 0, sizeof(int32_t), s);
    cudaMemsetAsync(maxb, 0, sizeof(int64_t), s);
    trace_begin("ninv_own_diag", s);
    own_diag<<<a.grid, kOwnThreads, 0, s>>>(a.n, st, ct, r, v, rp, a.dr, a.dp, a.part, diag, bound, maxb, a.gkeys,
                                            a.gvals, a.gslice, a.ticket);
    trace_end(s);
    return cudaGetLastError();
}

cudaError_t own_product_launch(const OwnArgs& a, const int64_t* st, const int64_t* ct, const int32_t* r,
                               const double* v, const int64_t* rp, const int32_t* rc, const double* rv,
                               const double* diag, const int64_t* bound, int32_t* nr, double* nv, int64_t* stN,
                               int64_t* ctN, int64_t cap, cudaStream_t s) {
    cudaMemsetAsync(a.ticket, 0, sizeof(int32_t), s);
    cudaMemsetAsync(a.cursor, 0, sizeof(unsigned long long), s);
    trace_begin("ninv_own_product", s);
    own_product<<<a.grid, kOwnThreads, 2 * kProdSlots * (sizeof(int32_t) + sizeof(double)), s>>>(a.n, st, ct, r, v, rp, rc, rv, a.dr, a.dp, a.part, diag, bound,
                                               a.delta, nr, nv, stN, ctN, cap, a.cursor, a.gkeys, a.gvals, a.gslice,
                                               a.ticket);
    trace_end(s);
    return cudaGetLastError();
}

int own_table_slots(int64_t entries) { return (int)table_mask(entries) + 1; }
int own_smem_slots() { return kSmemSlots; }
int own_horner_slots() { return kHornerSlots; }
int own_prod_slots() { return kProdSlots; }

cudaError_t own_configure() {
    cudaError_t e = cudaFuncSetAttribute(own_horner, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kHornerSlots * (sizeof(int32_t) + sizeof(double))));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(own_product, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(2 * kProdSlots * (sizeof(int32_t) + sizeof(double))));
}
int own_grid_ctas(int num_sms) { return num_sms * 4; }

}  // namespace sinv
