// NInv on its own pattern (Section 2.2, Eqs. (6) and (8)): the inverse tolerance
// delta sparsifies the Neumann series W = L^inv and the product W^T D^{-1} W, so
// both patterns depend on the values and fall with delta.
//
// Horner step t (column form, W_t[:, j] = e_j + sum_{k in struct(j)} E_kj
// W_{t-1}[:, k]): one CTA per column accumulates the products in a hash table
// (shared memory, or a global slice for long columns) over the compacted
// columns of W_{t-1}, drops the off-diagonal entries below delta and writes the
// survivors into the column's slot of the structural pattern P_W (an upper bound
// of its length); a scan and a copy then compact the step.
//
// Product: with Y = D^{-1} W (rows of column j and their 2x2 partners), a first
// pass forms every diagonal N_jj = W[:, j] . Y[:, j] and a bound on the length of
// column j of N (the sum of the lengths of the rows of W that Y[:, j] touches);
// the second pass accumulates N[i, j] = sum_c W[c, i] Y[c, j] for i >= j through
// the rows of W (W transposed once) in a hash table, keeps the diagonal and the
// entries with |N_ij| >= delta sqrt|N_ii N_jj|, and writes them into the
// column's bounded slot; a scan and a copy compact the result (CSC of the lower
// triangle, rows in hash order).
#include <algorithm>

#include "device.cuh"
#include "hash.cuh"
#include "kernels.h"

namespace sinv {

namespace {

constexpr int kOwnThreads = 256;
constexpr int kOwnWarps = kOwnThreads / 32;
constexpr int kSmemSlots = 2048;  // keys + FP64 values in shared memory: 24 KB

// per-CTA table: shared memory when it fits, else the CTA's slice of `gkeys` / `gvals`
struct Table {
    int32_t* keys;
    double* vals;
    uint32_t mask;
};

__device__ __forceinline__ Table make_table(int64_t entries, int32_t* skeys, double* svals, int32_t* gkeys,
                                            double* gvals, int64_t gslice) {
    Table t;
    t.mask = table_mask(entries);
    if ((int64_t)t.mask + 1 <= kSmemSlots) {
        t.keys = skeys;
        t.vals = svals;
    } else {
        t.keys = gkeys + (int64_t)blockIdx.x * gslice;
        t.vals = gvals + (int64_t)blockIdx.x * gslice;
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

// W_t from the compacted W_{t-1}: columns in any order (ticket), survivors into the
// structural slot [Wcp[j], Wcp[j] + cap) of the scratch arrays
__global__ void __launch_bounds__(kOwnThreads) own_horner(int64_t n, const int64_t* __restrict__ Lcp,
                                                          const int32_t* __restrict__ Lri,
                                                          const int32_t* __restrict__ Lcsr,
                                                          const double* __restrict__ Lval,
                                                          const int64_t* __restrict__ cpIn,
                                                          const int32_t* __restrict__ rIn,
                                                          const double* __restrict__ vIn,
                                                          const int64_t* __restrict__ Wcp, double delta,
                                                          int32_t* __restrict__ rOut, double* __restrict__ vOut,
                                                          int64_t* __restrict__ cnt, int32_t* gkeys, double* gvals,
                                                          int64_t gslice, int32_t* ticket) {
    __shared__ int32_t skeys[kSmemSlots];
    __shared__ double svals[kSmemSlots];
    __shared__ int64_t s_j;
    __shared__ int32_t s_cnt;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) {
            s_j = atomicAdd(ticket, 1);
            s_cnt = 0;
        }
        __syncthreads();
        const int64_t j = s_j;
        __syncthreads();
        if (j >= n) break;
        const int64_t cap = Wcp[j + 1] - Wcp[j];
        Table t = make_table(cap, skeys, svals, gkeys, gvals, gslice);
        __syncthreads();
        if (threadIdx.x == 0) table_add(t, (int32_t)j, 1.0);
        for (int64_t q = Lcp[j] + wid; q < Lcp[j + 1]; q += kOwnWarps) {
            const int32_t k = Lri[q];
            const double e = -Lval[Lcsr[q]];
            for (int64_t p = cpIn[k] + lane; p < cpIn[k + 1]; p += 32) table_add(t, rIn[p], e * vIn[p]);
        }
        __syncthreads();
        const int64_t base = Wcp[j];
        for (uint32_t s = threadIdx.x; s <= t.mask; s += blockDim.x) {
            const int32_t r = t.keys[s];
            if (r < 0) continue;
            const double v = t.vals[s];
            if (r != j && !(fabs(v) >= delta)) continue;
            const int32_t o = atomicAdd(&s_cnt, 1);
            if (o < cap) {
                rOut[base + o] = r;
                vOut[base + o] = v;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) cnt[j] = min((int64_t)s_cnt, cap);  // s_cnt <= cap: P_W holds every row a step reaches
        __syncthreads();
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

// copy every column's cnt[j] entries from its slot [off[j], ...) to [cp[j], cp[j+1])
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

// W by rows: counts, then the entries (column i and value) of every row
__global__ void own_row_count(int64_t nnz, const int32_t* __restrict__ r, int64_t* __restrict__ rowcnt) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(reinterpret_cast<unsigned long long*>(rowcnt + r[e]), 1ull);
}

__global__ void own_row_fill(int64_t n, const int64_t* __restrict__ cp, const int32_t* __restrict__ r,
                             const double* __restrict__ v, int64_t* __restrict__ fill, int32_t* __restrict__ rc,
                             double* __restrict__ rv) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        for (int64_t p = cp[j]; p < cp[j + 1]; ++p) {
            const int64_t d = (int64_t)atomicAdd(reinterpret_cast<unsigned long long*>(fill + r[p]), 1ull);
            rc[d] = (int32_t)j;
            rv[d] = v[p];
        }
}

// Y[:, j] = D^{-1} W[:, j] in the table (rows of the column and their partners)
__device__ __forceinline__ void fill_y(Table& t, const int64_t* cp, const int32_t* r, const double* v, int64_t j,
                                       const double* dr, const double* dp, const int32_t* part) {
    for (int64_t p = cp[j] + threadIdx.x; p < cp[j + 1]; p += blockDim.x) {
        const int32_t c = r[p];
        const double w = v[p];
        table_add(t, c, dr[c] * w);
        if (part[c] >= 0) table_add(t, part[c], dp[c] * w);
    }
}

// pass A: N_jj = W[:, j] . Y[:, j], and the bound sum over the rows c of Y[:, j] of
// the length of row c of W, capped at n - j (the rows i >= j of column j of N)
__global__ void __launch_bounds__(kOwnThreads) own_diag(int64_t n, const int64_t* __restrict__ cp,
                                                        const int32_t* __restrict__ r, const double* __restrict__ v,
                                                        const int64_t* __restrict__ rp, const double* __restrict__ dr,
                                                        const double* __restrict__ dp, const int32_t* __restrict__ part,
                                                        double* __restrict__ diag, int64_t* __restrict__ bound,
                                                        int32_t* gkeys, double* gvals, int64_t gslice,
                                                        int32_t* ticket) {
    __shared__ int32_t skeys[kSmemSlots];
    __shared__ double svals[kSmemSlots];
    __shared__ int64_t s_j;
    __shared__ double s_d;
    __shared__ unsigned long long s_b;
    for (;;) {
        if (threadIdx.x == 0) {
            s_j = atomicAdd(ticket, 1);
            s_d = 0.0;
            s_b = 0ull;
        }
        __syncthreads();
        const int64_t j = s_j;
        __syncthreads();
        if (j >= n) break;
        Table t = make_table(2 * (cp[j + 1] - cp[j]), skeys, svals, gkeys, gvals, gslice);
        __syncthreads();
        fill_y(t, cp, r, v, j, dr, dp, part);
        __syncthreads();
        double s = 0.0;
        for (int64_t p = cp[j] + threadIdx.x; p < cp[j + 1]; p += blockDim.x) {
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
            bound[j] = min((int64_t)s_b, n - j);
        }
        __syncthreads();
    }
}

// pass B: column j of N (rows i >= j) with the drop, into the slot [off[j], off[j] + bound[j])
__global__ void __launch_bounds__(kOwnThreads) own_product(int64_t n, const int64_t* __restrict__ cp,
                                                           const int32_t* __restrict__ r,
                                                           const double* __restrict__ v,
                                                           const int64_t* __restrict__ rp,
                                                           const int32_t* __restrict__ rc,
                                                           const double* __restrict__ rv,
                                                           const double* __restrict__ dr,
                                                           const double* __restrict__ dp,
                                                           const int32_t* __restrict__ part,
                                                           const double* __restrict__ diag,
                                                           const int64_t* __restrict__ off,
                                                           const int64_t* __restrict__ bound, double delta,
                                                           int32_t* __restrict__ nr, double* __restrict__ nv,
                                                           int64_t* __restrict__ cnt, int32_t* gkeys, double* gvals,
                                                           int64_t gslice, int32_t* ticket) {
    __shared__ int32_t skeys[kSmemSlots / 2];
    __shared__ double svals[kSmemSlots / 2];
    __shared__ int32_t skeys2[kSmemSlots / 2];
    __shared__ double svals2[kSmemSlots / 2];
    __shared__ int64_t s_j;
    __shared__ int32_t s_cnt;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) {
            s_j = atomicAdd(ticket, 1);
            s_cnt = 0;
        }
        __syncthreads();
        const int64_t j = s_j;
        __syncthreads();
        if (j >= n) break;
        // Y[:, j] in the first half of the CTA's scratch, N's column in the second
        Table ty, tn;
        {
            const int64_t ey = 2 * (cp[j + 1] - cp[j]);
            ty.mask = table_mask(ey);
            const bool sm = (int64_t)ty.mask + 1 <= kSmemSlots / 2;
            ty.keys = sm ? skeys : gkeys + (int64_t)blockIdx.x * gslice;
            ty.vals = sm ? svals : gvals + (int64_t)blockIdx.x * gslice;
            tn.mask = table_mask(bound[j]);
            const bool sm2 = (int64_t)tn.mask + 1 <= kSmemSlots / 2;
            tn.keys = sm2 ? skeys2 : gkeys + (int64_t)blockIdx.x * gslice + (gslice / 2);
            tn.vals = sm2 ? svals2 : gvals + (int64_t)blockIdx.x * gslice + (gslice / 2);
            for (uint32_t s = threadIdx.x; s <= ty.mask; s += blockDim.x) {
                ty.keys[s] = -1;
                ty.vals[s] = 0.0;
            }
            for (uint32_t s = threadIdx.x; s <= tn.mask; s += blockDim.x) {
                tn.keys[s] = -1;
                tn.vals[s] = 0.0;
            }
        }
        __syncthreads();
        fill_y(ty, cp, r, v, j, dr, dp, part);
        __syncthreads();
        // N[i, j] += W[c, i] Y[c, j] over the rows c of Y[:, j] and the entries of row c of W
        for (uint32_t s = wid; s <= ty.mask; s += kOwnWarps) {
            const int32_t c = ty.keys[s];
            if (c < 0) continue;
            const double y = ty.vals[s];
            for (int64_t p = rp[c] + lane; p < rp[c + 1]; p += 32) {
                const int32_t i = rc[p];
                if (i >= j) table_add(tn, i, rv[p] * y);
            }
        }
        __syncthreads();
        const double djj = diag[j];
        const int64_t base = off[j], cap = bound[j];
        for (uint32_t s = threadIdx.x; s <= tn.mask; s += blockDim.x) {
            const int32_t i = tn.keys[s];
            if (i < 0) continue;
            const double x = tn.vals[s];
            if (i != j && !(fabs(x) >= delta * sqrt(fabs(diag[i] * djj)))) continue;
            const int32_t o = atomicAdd(&s_cnt, 1);
            if (o < cap) {
                nr[base + o] = i;
                nv[base + o] = x;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) cnt[j] = min((int64_t)s_cnt, cap);  // s_cnt <= bound[j] by construction
        __syncthreads();
    }
}

int own_grid(int num_sms) { return num_sms * 4; }

// W_0 = I as compacted columns
__global__ void own_identity(int64_t n, int64_t* __restrict__ cp, int32_t* __restrict__ r, double* __restrict__ v) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j <= n; j += (int64_t)gridDim.x * blockDim.x) {
        cp[j] = j;
        if (j < n) {
            r[j] = (int32_t)j;
            v[j] = 1.0;
        }
    }
}

}  // namespace

cudaError_t own_identity_launch(int64_t n, int64_t* cp, int32_t* r, double* v, int num_sms, cudaStream_t st) {
    own_identity<<<num_sms * 4, 256, 0, st>>>(n, cp, r, v);
    return cudaGetLastError();
}

cudaError_t own_horner_launch(const OwnArgs& a, int t, const int64_t* cpIn, const int32_t* rIn, const double* vIn,
                              int32_t* rOut, double* vOut, int64_t* cnt, cudaStream_t st) {
    (void)t;
    cudaMemsetAsync(a.ticket, 0, sizeof(int32_t), st);
    trace_begin("ninv_own_horner", st);
    own_horner<<<own_grid(a.num_sms), kOwnThreads, 0, st>>>(a.n, a.Lcp, a.Lri, a.Lcsr, a.Lval, cpIn, rIn, vIn, a.Wcp,
                                                            a.delta, rOut, vOut, cnt, a.gkeys, a.gvals, a.gslice,
                                                            a.ticket);
    trace_end(st);
    return cudaGetLastError();
}

cudaError_t own_scan_launch(int64_t n, const int64_t* cnt, int64_t* out, cudaStream_t st) {
    own_scan<<<1, 1024, 0, st>>>(n, cnt, out);
    return cudaGetLastError();
}

cudaError_t own_compact_launch(int64_t n, const int64_t* off, const int64_t* cp, const int32_t* rs, const double* vs,
                               int32_t* rd, double* vd, int num_sms, cudaStream_t st) {
    own_compact<<<num_sms * 8, 256, 0, st>>>(n, off, cp, rs, vs, rd, vd);
    return cudaGetLastError();
}

cudaError_t own_transpose_launch(int64_t n, int64_t nnz, const int64_t* cp, const int32_t* r, const double* v,
                                 int64_t* rowcnt, int64_t* rp, int64_t* fill, int32_t* rc, double* rv, int num_sms,
                                 cudaStream_t st) {
    cudaMemsetAsync(rowcnt, 0, n * sizeof(int64_t), st);
    own_row_count<<<num_sms * 8, 256, 0, st>>>(nnz, r, rowcnt);
    own_scan<<<1, 1024, 0, st>>>(n, rowcnt, rp);
    cudaMemcpyAsync(fill, rp, n * sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
    own_row_fill<<<num_sms * 8, 256, 0, st>>>(n, cp, r, v, fill, rc, rv);
    return cudaGetLastError();
}

cudaError_t own_diag_launch(const OwnArgs& a, const int64_t* cp, const int32_t* r, const double* v, const int64_t* rp,
                            double* diag, int64_t* bound, cudaStream_t st) {
    cudaMemsetAsync(a.ticket, 0, sizeof(int32_t), st);
    trace_begin("ninv_own_diag", st);
    own_diag<<<own_grid(a.num_sms), kOwnThreads, 0, st>>>(a.n, cp, r, v, rp, a.dr, a.dp, a.part, diag, bound, a.gkeys,
                                                          a.gvals, a.gslice, a.ticket);
    trace_end(st);
    return cudaGetLastError();
}

cudaError_t own_product_launch(const OwnArgs& a, const int64_t* cp, const int32_t* r, const double* v,
                               const int64_t* rp, const int32_t* rc, const double* rv, const double* diag,
                               const int64_t* off, const int64_t* bound, int32_t* nr, double* nv, int64_t* cnt,
                               cudaStream_t st) {
    cudaMemsetAsync(a.ticket, 0, sizeof(int32_t), st);
    trace_begin("ninv_own_product", st);
    own_product<<<own_grid(a.num_sms), kOwnThreads, 0, st>>>(a.n, cp, r, v, rp, rc, rv, a.dr, a.dp, a.part, diag, off,
                                                             bound, a.delta, nr, nv, cnt, a.gkeys, a.gvals, a.gslice,
                                                             a.ticket);
    trace_end(st);
    return cudaGetLastError();
}

int own_table_slots(int64_t entries) { return (int)table_mask(entries) + 1; }
int own_grid_ctas(int num_sms) { return own_grid(num_sms); }

}  // namespace sinv
