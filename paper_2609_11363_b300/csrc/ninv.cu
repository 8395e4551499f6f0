// NInv (Section 2.2): truncated Neumann series of L^{-1}, Eq. (6), and the
// product (L^inv)^T D^{-1} L^inv of Eq. (8), evaluated on S only.
//
// With L = I - E, W = sum_{t=0}^{m} E^t is built by m Horner steps
//     W_t = I + E W_{t-1}      (column form: W_t[:, j] = e_j + sum_{k in struct(j)} E_kj W_{t-1}[:, k])
// on the fixed pattern P_W of the truncated series.  P_W is stored by columns
// with every column's rows grouped by the first power that reaches them, so
// the nonzeros of W_{t-1}[:, k] are exactly the prefix "groups 0..t-1" of
// column k and no step touches a structural zero.
//
// Horner step: one CTA owns one column j.  Its rows go into a shared-memory
// hash table (row -> slot).  Warp v handles the columns k of struct(j) with
// k = v mod 8 and adds E_kj W_{t-1}[r, k] into the slot of r with shared-memory
// atomics (native for FP32 and FP64 and as fast as a plain read-modify-write
// here; the lanes of one instruction always touch distinct rows).
//
// Product on S: N_ij = sum_r W_ri (D^{-1} W)_rj for (i, j) in S_lo.  One CTA
// owns column j: it tabulates y = (D^{-1} W)[:, j] on the rows of column j,
// then one warp per entry (i, j) streams column i of W and sums W_ri y_r over
// the rows found in the table.  The 2x2 blocks of D^{-1} couple a row with its
// partner: a row of column i outside column j still meets y through its
// partner; pattern entries carry a flag bit for rows of 2x2 blocks so that only
// those rows pay for the extra lookup.
//
// Columns too long for shared memory use the same code on a per-CTA slice of
// global scratch, with atomic accumulation.
#include <algorithm>

#include "device.cuh"
#include "hash.cuh"
#include "kernels.h"

namespace sinv {

namespace {

constexpr int kWarps = 8;                     // warps per CTA (Horner step and product)
constexpr int kThreads = kWarps * 32;
constexpr int kSlots = 4096;                  // hash slots in shared memory
constexpr int kEnt = 2730;                    // most table entries kept in shared memory (load <= 2/3)
constexpr int kUnroll = 8;                    // column entries per lane with loads in flight
constexpr int32_t kRowMask = 0x7FFFFFFF;      // row index bits of a pattern entry
constexpr int32_t kTwoFlag = (int32_t)0x80000000u;  // set when the row belongs to a 2x2 block of D

template <class T>
__global__ void ninv_init(const int64_t* __restrict__ Wcp, T* __restrict__ W, int64_t n) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        W[Wcp[j]] = T(1);  // group 0 of column j is row j
}

// D^{-1} per row: dr[r] = (D^{-1})_rr, dp[r] = (D^{-1})_{r, partner}, part[r] = partner or -1.
__global__ void ninv_dinv(int64_t n, const int32_t* __restrict__ dpos, const int8_t* __restrict__ pstart,
                          const double* __restrict__ Dval, double* __restrict__ dr, double* __restrict__ dp,
                          int32_t* __restrict__ part, int32_t* status) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const bool first = pstart[r] != 0;
        const bool two = first ? (r + 1 < n && pstart[r + 1] == 0) : true;
        const double* d = Dval + dpos[r];
        if (!two) {
            if (d[0] == 0.0) set_status(status, ST_SINGULAR);
            dr[r] = 1.0 / d[0];
            dp[r] = 0.0;
            part[r] = -1;
        } else {
            double det = d[0] * d[2] - d[1] * d[1];
            if (det == 0.0) set_status(status, ST_SINGULAR);
            dr[r] = (first ? d[2] : d[0]) / det;
            dp[r] = -d[1] / det;
            part[r] = (int32_t)(first ? r + 1 : r - 1);
        }
    }
}

template <class T>
__device__ __forceinline__ T fma_t(T a, T b, T c);
template <>
__device__ __forceinline__ double fma_t<double>(double a, double b, double c) { return fma(a, b, c); }
template <>
__device__ __forceinline__ float fma_t<float>(float a, float b, float c) { return fmaf(a, b, c); }

struct Scratch {
    int32_t* keys;   // per CTA: slots int32 keys
    void* acc;       // per CTA: slots accumulators / y values of 8 bytes
    int64_t slots;   // slots per CTA (0 when every column fits shared memory)
};

template <class T>
__global__ void __launch_bounds__(kThreads) ninv_horner(NinvArgs a, int t, const T* __restrict__ Wp, T* __restrict__ Wn,
                                                         int32_t* ticket, Scratch gs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sacc = reinterpret_cast<T*>(smem_raw);                    // kSlots accumulators, one per slot
    int32_t* skeys = reinterpret_cast<int32_t*>(sacc + kSlots);  // kSlots keys
    __shared__ int32_t s_j;
    const int G = a.m + 2;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) s_j = atomicAdd(ticket, 1);
        __syncthreads();
        const int64_t j = s_j;
        __syncthreads();
        if (j >= a.n) break;
        const int64_t base = a.Wcp[j];
        const int32_t nj = a.grp[j * G + t + 1];  // rows of groups 0..t
        const bool small = nj <= kEnt;
        const uint32_t mask = small ? (uint32_t)(kSlots - 1) : table_mask(nj);
        int32_t* keys = small ? skeys : gs.keys + (int64_t)blockIdx.x * gs.slots;
        T* acc = small ? sacc : reinterpret_cast<T*>(gs.acc) + (int64_t)blockIdx.x * gs.slots;
        for (uint32_t s = threadIdx.x; s <= mask; s += kThreads) {
            keys[s] = -1;
            acc[s] = T(0);
        }
        __syncthreads();
        for (int32_t e = threadIdx.x; e < nj; e += kThreads) table_insert(keys, mask, a.Wr[base + e] & kRowMask);
        __syncthreads();
        // sum_k E_kj W_{t-1}[:, k]: warp wid takes k = wid, wid+8, ...; lanes over column k's
        // groups 0..t-1, kUnroll entries per lane in flight; atomic adds into the row's slot
        for (int64_t q = a.Lcp[j] + wid; q < a.Lcp[j + 1]; q += kWarps) {
            const int32_t k = a.Lri[q];
            const T ekj = T(-a.Lval[a.Lcsr[q]]);
            const int64_t kb = a.Wcp[k];
            const int32_t nk = a.grp[(int64_t)k * G + t];
            for (int32_t e0 = 0; e0 < nk; e0 += 32 * kUnroll) {
                int32_t r[kUnroll];
                T v[kUnroll];
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) {
                    const int32_t e = e0 + u * 32 + lane;
                    r[u] = e < nk ? (a.Wr[kb + e] & kRowMask) : -1;
                    v[u] = e < nk ? Wp[kb + e] : T(0);
                }
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) {
                    if (r[u] < 0) continue;
                    const int32_t h = table_find(keys, mask, r[u]);
                    if (h >= 0) atomicAdd(acc + h, ekj * v[u]);
                    else set_status(a.status, ST_INTERNAL);  // row outside the pattern: never expected
                }
            }
        }
        __syncthreads();
        for (int32_t e = threadIdx.x; e < nj; e += kThreads) {
            const int32_t h = table_find(keys, mask, a.Wr[base + e] & kRowMask);
            const T v = acc[h] + (e == 0 ? T(1) : T(0));
            Wn[base + e] = (e != 0 && fabs((double)v) < a.delta) ? T(0) : v;  // drop below the tolerance
        }
        __syncthreads();
    }
}

// tlim: use the rows of groups 0..tlim of every column (the truncation after tlim
// Horner steps; tlim = m is the whole pattern)
template <class T>
__global__ void __launch_bounds__(kThreads) ninv_product(NinvArgs a, int tlim, const T* __restrict__ W,
                                                         const double* __restrict__ dr, const double* __restrict__ dp,
                                                         const int32_t* __restrict__ part, double* __restrict__ N,
                                                         int32_t* ticket, Scratch gs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* syv = reinterpret_cast<T*>(smem_raw);                     // y = (D^{-1} W)[:, j], one per slot
    int32_t* skeys = reinterpret_cast<int32_t*>(syv + kSlots);
    __shared__ int32_t s_j, s_flagged;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) {
            s_j = atomicAdd(ticket, 1);
            s_flagged = 0;
        }
        __syncthreads();
        const int64_t j = s_j;
        __syncthreads();
        if (j >= a.n) break;
        const int G = a.m + 2;
        const int64_t base = a.Wcp[j];
        const int32_t nj = a.grp[j * G + tlim + 1];
        // the table holds the rows of column j and, for its rows in 2x2 blocks, their partners
        int flagged = 0;
        for (int32_t e = threadIdx.x; e < nj; e += kThreads) flagged += (a.Wr[base + e] & kTwoFlag) ? 1 : 0;
        if (flagged) atomicAdd(&s_flagged, flagged);
        __syncthreads();
        const int32_t entries = nj + s_flagged;
        const bool small = entries <= kEnt;
        const uint32_t mask = small ? (uint32_t)(kSlots - 1) : table_mask(entries);
        int32_t* keys = small ? skeys : gs.keys + (int64_t)blockIdx.x * gs.slots;
        T* yv = small ? syv : reinterpret_cast<T*>(gs.acc) + (int64_t)blockIdx.x * gs.slots;
        for (uint32_t s = threadIdx.x; s <= mask; s += kThreads) {
            keys[s] = -1;
            yv[s] = T(0);
        }
        __syncthreads();
        for (int32_t e = threadIdx.x; e < nj; e += kThreads) table_insert(keys, mask, a.Wr[base + e] & kRowMask);
        __syncthreads();
        // y_r = sum_{r'} (D^{-1})_{r r'} W_{r' j}: row r adds (D^{-1})_rr W_rj to its own slot and,
        // in a 2x2 block with partner p, (D^{-1})_pr W_rj to p's slot (inserted if p is not in column j)
        for (int32_t e = threadIdx.x; e < nj; e += kThreads) {
            const int32_t rf = a.Wr[base + e];
            const int32_t r = rf & kRowMask;
            const double wv = (double)W[base + e];
            atomicAdd(yv + table_find(keys, mask, r), T(dr[r] * wv));
            if (rf & kTwoFlag) atomicAdd(yv + table_insert(keys, mask, part[r]), T(dp[r] * wv));
        }
        __syncthreads();
        // entries of S_lo in column j: the diagonal, the 2x2 partner row, struct(j)
        const bool two_first = a.pstart[j] != 0 && j + 1 < a.n && a.pstart[j + 1] == 0;
        const int64_t q0 = a.Lcp[j], q1 = a.Lcp[j + 1];
        const int64_t cnt = (q1 - q0) + 1 + (two_first ? 1 : 0);
        for (int64_t e = wid; e < cnt; e += kWarps) {
            int64_t i, spos;
            if (e == 0) {
                i = j;
                spos = a.Srp[j + 1] - 1;          // (j, j): last entry of row j
            } else if (two_first && e == 1) {
                i = j + 1;
                spos = a.Srp[j + 2] - 2;          // (j+1, j): before the diagonal of row j+1
            } else {
                const int64_t q = q0 + e - 1 - (two_first ? 1 : 0);
                i = a.Lri[q];
                // row i of S_lo starts with row i of L, so L(i, j) keeps its offset in the row
                spos = a.Srp[i] + ((int64_t)a.Lcsr[q] - a.Lrp[i]);
            }
            const int64_t ib = a.Wcp[i], ie = ib + a.grp[i * G + tlim + 1];
            T s = T(0);
            for (int64_t f0 = ib; f0 < ie; f0 += 32 * kUnroll) {
                int32_t r[kUnroll];
                T wv[kUnroll];
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) {
                    const int64_t f = f0 + u * 32 + lane;
                    r[u] = f < ie ? (a.Wr[f] & kRowMask) : -1;
                    wv[u] = f < ie ? W[f] : T(0);
                }
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) {
                    if (r[u] < 0) continue;
                    const int32_t h = table_find(keys, mask, r[u]);
                    if (h >= 0) s = fma_t<T>(wv[u], yv[h], s);
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) N[spos] = (double)s;
        }
        __syncthreads();
    }
}

template <class T>
constexpr size_t ninv_smem() { return (size_t)kSlots * (sizeof(int32_t) + sizeof(T)); }

int64_t global_slots(const NinvArgs& a) {
    if (a.max_col <= kEnt) return 0;
    return (int64_t)table_mask(2 * a.max_col) + 1;  // room for the partner rows too
}

}  // namespace

cudaError_t ninv_configure() {
    cudaError_t e;
    e = cudaFuncSetAttribute(ninv_horner<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ninv_smem<double>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(ninv_horner<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ninv_smem<float>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(ninv_product<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ninv_smem<double>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(ninv_product<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ninv_smem<float>());
}

static int ninv_grid(const NinvArgs& a) { return a.num_sms * 4; }

size_t ninv_work_bytes(const NinvArgs& a, int prec) {
    size_t ts = prec == 0 ? sizeof(double) : sizeof(float);
    size_t b = 2 * ((size_t)a.nnzW * ts + 256);                 // ping-pong W
    b += (size_t)a.n * (2 * sizeof(double) + sizeof(int32_t)) + 3 * 256;
    b += sizeof(int32_t) * 64 + 256;                            // tickets
    int64_t slots = global_slots(a);
    if (slots) b += (size_t)ninv_grid(a) * slots * (sizeof(int32_t) + sizeof(double)) + 2 * 256;
    return b + 4096;
}

template <class T>
static cudaError_t ninv_run(const NinvArgs& a, void* work, double* N_out, double* N_stack, cudaStream_t st) {
    char* p = reinterpret_cast<char*>(work);
    auto take = [&](size_t bytes) {
        char* r = p;
        p += (bytes + 255) & ~(size_t)255;
        return r;
    };
    T* W0 = reinterpret_cast<T*>(take((size_t)a.nnzW * sizeof(T)));
    T* W1 = reinterpret_cast<T*>(take((size_t)a.nnzW * sizeof(T)));
    double* dr = reinterpret_cast<double*>(take((size_t)a.n * sizeof(double)));
    double* dp = reinterpret_cast<double*>(take((size_t)a.n * sizeof(double)));
    int32_t* part = reinterpret_cast<int32_t*>(take((size_t)a.n * sizeof(int32_t)));
    int32_t* tickets = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * 64));
    const int grid = ninv_grid(a);
    Scratch gs{nullptr, nullptr, global_slots(a)};
    if (gs.slots) {
        gs.keys = reinterpret_cast<int32_t*>(take((size_t)grid * gs.slots * sizeof(int32_t)));
        gs.acc = take((size_t)grid * gs.slots * sizeof(double));
    }
    cudaError_t e = cudaMemsetAsync(tickets, 0, sizeof(int32_t) * 64, st);
    if (e != cudaSuccess) return e;
    trace_begin("ninv_dinv", st);
    ninv_dinv<<<a.num_sms * 4, 256, 0, st>>>(a.n, a.dpos, a.pstart, a.Dval, dr, dp, part, a.status);
    trace_end(st);
    trace_begin("ninv_init", st);
    ninv_init<T><<<a.num_sms * 4, 256, 0, st>>>(a.Wcp, W0, a.n);
    trace_end(st);
    T* cur = W0;
    T* nxt = W1;
    auto product = [&](int t, double* out, int32_t* tk) {
        trace_begin("ninv_product", st);
        ninv_product<T><<<grid, kThreads, ninv_smem<T>(), st>>>(a, t, cur, dr, dp, part, out, tk, gs);
        trace_end(st);
    };
    if (N_stack) product(0, N_stack, tickets + 62 - a.m);
    for (int t = 1; t <= a.m; ++t) {
        trace_begin("ninv_horner", st);
        ninv_horner<T><<<grid, kThreads, ninv_smem<T>(), st>>>(a, t, cur, nxt, tickets + t, gs);
        trace_end(st);
        std::swap(cur, nxt);
        if (N_stack && t < a.m) product(t, N_stack + (int64_t)t * a.nnzS, tickets + 62 - a.m + t);
    }
    product(a.m, N_stack ? N_stack + (int64_t)a.m * a.nnzS : N_out, tickets + 63);
    return cudaGetLastError();
}

void ninv_dinv_launch(const NinvArgs& a, double* dr, double* dp, int32_t* part, cudaStream_t st) {
    ninv_dinv<<<a.num_sms * 4, 256, 0, st>>>(a.n, a.dpos, a.pstart, a.Dval, dr, dp, part, a.status);
}

cudaError_t ninv_launch(const NinvArgs& a, int prec, void* work, double* N_out, cudaStream_t st, double* N_stack) {
    if (a.n == 0) return cudaSuccess;
    if (a.m > 30) return cudaErrorInvalidValue;
    if (prec == 0) return ninv_run<double>(a, work, N_out, N_stack, st);
    return ninv_run<float>(a, work, N_out, N_stack, st);
}

}  // namespace sinv
